"""Pins for the oracle's upwind DG sweep."""
import math

import numpy as np
import pytest

import smm_workloads as W
from oracle.transport import CycleError, Discretization
from tests.oracle_problems import disc_for, linear_problem, mms_problem


def test_sweep_equals_global_dense_solve():
    mesh, disc, q, pb = mms_problem(3, 2, 2, 4, seed=11, sigs=0.0)
    psi = disc.sweep(None, q, pb)
    for d in range(disc.nd):
        A = disc.global_ordinate_matrix(d)
        b = disc.global_ordinate_rhs(d, q[d], pb)
        ref = np.linalg.solve(A, b).reshape(disc.ne, disc.n)
        assert np.max(np.abs(psi[d] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("m,p,seed", [(1, 1, None), (2, 2, 5), (1, 3, 8)])
def test_linear_angular_flux_is_reproduced(m, p, seed):
    mesh, disc, q, pb, _ = linear_problem(4, m, p, 4, seed=seed, sigs=0.0)
    psi = disc.sweep(None, q, pb)
    for d, o in enumerate(disc.omega):
        ex = disc.interpolate(lambda x, y: W.linear_aniso_psi(x, y, o[0], o[1]))
        assert np.max(np.abs(psi[d] - ex)) < 1e-13


def test_element_balance():
    mesh, disc, q, pb = mms_problem(4, 3, 2, 4, seed=1, sigs=0.0)
    psi = disc.sweep(None, q, pb)
    for d in range(0, disc.nd, 3):
        for e, el in enumerate(disc.elems):
            out = inn = 0.0
            for f in range(4):
                fd = disc.faces[e][f]
                a = fd["nds"] @ disc.omega[d]
                out += np.sum(np.maximum(a, 0) * (fd["V"] @ psi[d, e]))
                up = disc.upwind_values(e, f, d, psi[d], pb)
                inn += np.sum(np.minimum(a, 0) * up)
            coll = disc.sigma_t[e] * np.sum(el.w * el.J * (el.V @ psi[d, e]))
            src = np.sum(el.w * el.J * (el.V @ q[d, e]))
            assert abs(out + inn + coll - src) < 1e-13 * max(1.0, abs(src))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_local_matrix_symmetric_part_positive(p):
    """x^T A x = 1/2 int_dK |Omega.n| x^2 + sigma_t |x|^2 > 0: LU without
    pivoting is safe for every local system."""
    mesh = W.structured_mesh(3, m=3, perturb_seed=3)
    for st in (0.2, 200.0):
        disc = disc_for(mesh, p, 8, st, 0.0)
        for e in range(disc.ne):
            for d in range(0, disc.nd, 7):
                A = disc.local_matrix(e, d)
                assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_cycle_detected():
    mesh = W.structured_mesh(2, 1, m=2, domain=(0.0, 2.0, 0.0, 1.0))
    nodes = mesh.nodes.copy()
    # middle control point of the shared face (x=1, y=0.5) bulged to x=1.2
    k = np.argmin(np.hypot(nodes[:, 0] - 1.0, nodes[:, 1] - 0.5))
    nodes[k, 0] = 1.2
    disc = Discretization(nodes, mesh.elem_nodes, 2, 1, 8, np.ones(2), np.zeros(2))
    assert min(el.J.min() for el in disc.elems) > 0
    with pytest.raises(CycleError):
        for d in range(disc.nd):
            disc.upwind_order(d, lag_cycles=False)
    # with lagging (the default) the mixed face is lagged in one direction
    assert sum(len(disc.upwind_order(d)[1]) for d in range(disc.nd)) > 0


def test_sweep_mms_order():
    errs = []
    for nx in (4, 8):
        mesh, disc, q, pb = mms_problem(nx, 3, 2, 4, seed=7, sigs=0.9)
        phi_ex = disc.interpolate(W.mms_phi)
        psi = disc.sweep(phi_ex, q, pb)
        phi = np.einsum("d,den->en", disc.wq, psi)
        errs.append(disc.l2_error(phi, W.mms_phi))
    assert math.log2(errs[0] / errs[1]) > 2.6

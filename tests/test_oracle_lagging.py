"""Pins of the oracle's cycle lagging (Sec. 6.2 lags the cycles of its
distorted mesh's upwind graphs; the ordering rule is stated in
oracle/transport.py).

On meshes whose faces turn enough for grazing ordinates to enter a face at
some points and leave it at others, the upwind graphs have cycles.  The
checks: nothing is lagged without cycles; a lagged sweep fed with the exact
solution of each ordinate's whole DG system (dense LU, no ordering at all)
returns that solution; repeated lagged sweeps converge to it; and the SMM
iteration with lagged sweeps converges to the dense solution of the coupled
transport + moment system.
"""
import math

import numpy as np
import pytest

import smm_workloads as W
from oracle.transport import CycleError, Discretization


def cyclic_mesh_problem(nx=5, m=2, p=1, sn=8, seed=1, c=0.5):
    mesh = W.structured_mesh(nx, m=m, perturb_seed=seed, wave_max=3, scale_by_k=False)
    ne = mesh.n_elem
    st = 1.0 + 0.5 * (np.arange(ne) % 3)
    disc = Discretization(mesh.nodes, mesh.elem_nodes, m, p, sn, st, c * st)
    rng = np.random.default_rng(5)
    q = rng.uniform(0.5, 1.5, (ne, disc.n))
    fpos = W.face_node_positions(mesh, p, W.boundary_faces(mesh))
    psibar = np.stack([1.0 + 0.3 * fpos[:, :, 0] * (1 + o[0]) for o in disc.omega])
    return mesh, disc, q, psibar


def test_meshes_without_cycles_lag_nothing():
    for mesh in (W.structured_mesh(4, m=1), W.structured_mesh(4, m=2, perturb_seed=3)):
        disc = Discretization(mesh.nodes, mesh.elem_nodes, mesh.m, 2, 8, np.ones(16), 0.5 * np.ones(16))
        assert all(not disc.upwind_order(d)[1] for d in range(disc.nd))


def test_cycles_are_lagged_or_rejected():
    _, disc, _, _ = cyclic_mesh_problem()
    lagged = [disc.upwind_order(d)[1] for d in range(disc.nd)]
    assert sum(map(len, lagged)) > 0
    with pytest.raises(CycleError):
        for d in range(disc.nd):
            disc.upwind_order(d, lag_cycles=False)
    # every element is visited once per ordinate, and a lagged face is an inflow face
    for d in range(disc.nd):
        order, lag = disc.upwind_order(d)
        assert sorted(order) == list(range(disc.ne))
        for e, f in lag:
            assert np.any(disc.faces[e][f]["nds"] @ disc.omega[d] < 0.0)


@pytest.mark.parametrize("case", [(5, 2, 1, 8, 1), (4, 2, 2, 12, 5)])
def test_lagged_sweep_fed_the_exact_solution_returns_it(case):
    mesh, disc, q, psibar = cyclic_mesh_problem(*case)
    phi = np.random.default_rng(2).uniform(0.5, 2.0, (disc.ne, disc.n))
    exact = disc.solve_global(phi, q, psibar)
    got = disc.sweep(phi, q, psibar, psi_lag=exact)
    assert np.max(np.abs(got - exact)) <= 1e-12 * np.max(np.abs(exact))
    # with zero lagged inflow the sweep differs (the lagged faces matter)
    assert np.max(np.abs(disc.sweep(phi, q, psibar) - exact)) > 1e-6 * np.max(np.abs(exact))


def test_repeated_lagged_sweeps_converge_to_the_exact_solution():
    mesh, disc, q, psibar = cyclic_mesh_problem()
    exact = disc.solve_global(None, q, psibar)
    psi = np.zeros_like(exact)
    errs = []
    for _ in range(30):
        psi = disc.sweep(None, q, psibar, psi_lag=psi)
        errs.append(np.max(np.abs(psi - exact)) / np.max(np.abs(exact)))
    assert errs[-1] < 1e-12 and errs[5] < errs[0]


def test_smm_iteration_with_lagging_reaches_the_coupled_solution():
    from oracle.smm import SMMProblem, coupled_dense_solve
    mesh, disc, q, psibar = cyclic_mesh_problem(4, 2, 1, 4, 1, c=0.9)
    prob = SMMProblem(disc, q, psibar)
    ref = coupled_dense_solve(SMMProblem(disc, q, psibar))
    phi, k, _ = prob.iterate(tol=1e-13, max_outer=300)
    assert np.max(np.abs(phi - ref)) <= 1e-10 * np.max(np.abs(ref))

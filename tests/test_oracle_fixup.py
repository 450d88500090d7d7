"""Pins for the oracle's zero and scale negative flux fixup (used inside the
sweep, Sec. 6.3)."""
import numpy as np
import pytest

import smm_workloads as W
from oracle.smm import SMMProblem
from oracle.transport import zero_and_scale
from tests.oracle_problems import disc_for


def thick_strip(nx=6, sig=30.0, p=2):
    """A strip of thick, purely absorbing cells lit from the left: the DG
    solution dips below zero where the flux attenuates steeply."""
    mesh = W.structured_mesh(nx, 1, m=1)
    disc = disc_for(mesh, p, 4, sig, 0.0)
    bf = W.boundary_faces(mesh)
    pb = np.zeros((disc.nd, len(bf), p + 1))
    for b, (e, f) in enumerate(bf):
        if f == 3:
            pb[:, b, :] = 1.0
    return disc, pb


def test_zero_and_scale_closed_form():
    rng = np.random.default_rng(0)
    A = rng.random((9, 9)) + 9.0 * np.eye(9)
    x = rng.standard_normal(9) + 0.8
    c = A.sum(axis=0)
    y = zero_and_scale(A, x)
    assert np.all(y >= 0.0) and np.all(y[x < 0] == 0.0)
    assert abs(c @ y - c @ x) < 1e-13 * abs(c @ x)
    assert np.allclose(y[x > 0] / x[x > 0], (c @ x) / (c @ np.maximum(x, 0)))
    xp = np.abs(x)
    assert np.array_equal(zero_and_scale(A, xp), xp)                     # no negativity: unchanged
    assert np.array_equal(zero_and_scale(A, -xp), np.zeros(9))           # nothing to keep: zero


def test_thick_strip_negativities_removed_with_balance_kept():
    disc, pb = thick_strip()
    q = np.zeros((disc.ne, disc.n))
    assert disc.sweep(None, q, pb).min() < -1e-3                         # the DG solution dips negative
    for d in range(disc.nd):
        psi = disc.sweep_ordinate(d, q, pb, fixup=True)
        assert psi.min() >= 0.0
        # every element balances with the (fixed) inflow its upwind neighbours pass on
        for e in range(disc.ne):
            A = disc.local_matrix(e, d)
            b = np.zeros(disc.n)
            for f in range(4):
                fd = disc.faces[e][f]
                neg = np.minimum(fd["nds"] @ disc.omega[d], 0.0)
                if np.any(neg < 0.0):
                    b -= fd["V"].T @ (neg * disc.upwind_values(e, f, d, psi, pb))
            assert abs(np.sum(A @ psi[e] - b)) <= 1e-12 * max(1.0, np.sum(np.abs(b)))


def test_fixup_is_identity_on_positive_solutions():
    """Optically thin cells (sigma_t h = 1/3) with a unit isotropic source and
    inflow: the DG solution is positive and the fixup leaves it untouched."""
    mesh = W.structured_mesh(3, m=2, perturb_seed=5)
    disc = disc_for(mesh, 2, 4, 1.0, 0.5)
    q = np.ones((disc.ne, disc.n))
    bf = W.boundary_faces(mesh)
    pb = np.ones((disc.nd, len(bf), 3))
    phi = np.ones((disc.ne, disc.n))
    a, b = disc.sweep(phi, q, pb), disc.sweep(phi, q, pb, fixup=True)
    assert a.min() > 0 and np.array_equal(a, b)


def test_smm_converges_with_fixup():
    """SMM closures need no positivity (Remark nofixup); with the fixup the
    iteration still converges, in about as many steps (Table cp_fixup)."""
    disc, pb = thick_strip(8, 50.0, 2)
    disc.sigma_s[:] = 0.9 * disc.sigma_t
    q = np.zeros((disc.ne, disc.n))
    phi0, k0, _ = SMMProblem(disc, q, pb).iterate(tol=1e-10, relative=True)
    phi1, k1, _ = SMMProblem(disc, q, pb, fixup=True).iterate(tol=1e-10, relative=True)
    assert abs(k1 - k0) <= 2, (k0, k1)
    assert np.max(np.abs(phi1 - phi0)) < 0.2 * np.max(np.abs(phi0))   # close, not equal: the fixup changes psi

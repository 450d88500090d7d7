"""Pins for the oracle's parallel block Jacobi sweep (Sec. 6.5): every tile
sweeps its own elements, taking inflow from other tiles from the previous
sweep."""
import numpy as np

from oracle.smm import SMMProblem
from tests.oracle_problems import mms_problem


def test_tiles_from_corner_centroids():
    mesh, disc, q, pb = mms_problem(8, 2, 1, 4, seed=3)
    t = disc.element_tiles(4)
    assert sorted(np.unique(t)) == list(range(16))
    assert all(np.sum(t == k) == 4 for k in range(16))          # 2x2 elements per tile on an 8x8 grid
    e = np.arange(64)
    assert np.array_equal(t, (e // 8 // 2) * 4 + (e % 8) // 2)


def test_lagged_exact_inflow_reproduces_the_exact_sweep():
    """Consistency: fed the exact sweep as its lagged data, the block Jacobi
    sweep returns the exact sweep."""
    mesh, disc, q, pb = mms_problem(6, 2, 2, 4, seed=5, sigs=0.5)
    phi = np.ones((disc.ne, disc.n))
    exact = disc.sweep(phi, q, pb)
    block = disc.element_tiles(3)
    again = disc.sweep(phi, q, pb, block=block, psi_lag=exact)
    assert np.max(np.abs(again - exact)) <= 1e-13 * np.max(np.abs(exact))
    # with zero lagged data the result differs (cross-tile inflow missing)
    first = disc.sweep(phi, q, pb, block=block, psi_lag=np.zeros_like(exact))
    assert np.max(np.abs(first - exact)) > 1e-3 * np.max(np.abs(exact))


def test_one_tile_is_the_exact_sweep():
    mesh, disc, q, pb = mms_problem(4, 1, 2, 4, seed=None, sigs=0.5)
    phi = np.ones((disc.ne, disc.n))
    block = disc.element_tiles(1)
    assert np.all(block == 0)
    assert np.array_equal(disc.sweep(phi, q, pb, block=block, psi_lag=np.zeros((disc.nd, disc.ne, disc.n))),
                          disc.sweep(phi, q, pb))


def test_block_jacobi_iteration_reaches_the_same_fixed_point_in_more_steps():
    mesh, disc, q, pb = mms_problem(8, 1, 1, 4, seed=None, sigs=0.5)
    phi1, k1, _ = SMMProblem(disc, q, pb).iterate(tol=1e-11, relative=True)
    phi4, k4, _ = SMMProblem(disc, q, pb, tiles=4).iterate(tol=1e-11, relative=True)
    assert np.max(np.abs(phi4 - phi1)) <= 1e-9 * np.max(np.abs(phi1))
    assert k4 > k1

"""Pins for the oracle's discrete SMM closures."""
import math

import numpy as np

import smm_workloads as W
from oracle import closures
from tests.oracle_problems import angular_source, disc_for, linear_problem


def test_linear_anisotropy_gives_zero_corrections():
    mesh, disc, q, pb, _ = linear_problem(3, 2, 2, 8, seed=4)
    psi = angular_source(disc, W.linear_aniso_psi)
    mom = closures.nodal_moments(disc, psi)
    assert np.max(np.abs(mom[3:])) < 1e-14
    assert np.max(np.abs(closures.beta(disc, psi))) < 1e-14
    # phi and J of psi = (phi + 3 Omega.J)/4pi
    phi = disc.interpolate(lambda x, y: W.LIN_A + W.LIN_B * x + W.LIN_C * y)
    assert np.max(np.abs(mom[0] - phi)) < 1e-13
    assert np.max(np.abs(mom[1] - W.LIN_JX)) < 1e-14 and np.max(np.abs(mom[2] - W.LIN_JY)) < 1e-14


def test_mms_pressure_with_corrected_offdiagonal():
    """Discrete P of the MMS flux equals alpha/3 I + (1/15)[[3T11+T22, 2T12],[2T21, T11+3T22]]:
    the paper prints the off-diagonal as T12/15; int Omx^2 Omy^2 = 4pi/15 makes it 2 T12/15."""
    mesh = W.structured_mesh(3, m=2, perturb_seed=2)
    disc = disc_for(mesh, 2, 8, 1.0, 0.5)
    psi = angular_source(disc, W.mms_psi)
    mom = closures.nodal_moments(disc, psi)
    pos = W.dg_node_positions(mesh, 2)
    F = W._mms_fields(pos[:, :, 0], pos[:, :, 1])
    t11, t22, t12 = 0.5 * F["s3"], 0.25 * F["s3"], F["s2"]
    phi = F["al"] + (t11 + t22) / 3
    assert np.max(np.abs(mom[0] - phi)) < 1e-13
    assert np.max(np.abs(mom[4] - 2 * t12 / 15)) < 1e-13
    assert np.max(np.abs(mom[4] - t12 / 15)) > 1e-3
    pxx = F["al"] / 3 + (3 * t11 + t22) / 15
    assert np.max(np.abs(mom[3] + phi / 3 - pxx)) < 1e-13


def test_isotropic_inflow_partial_current_and_eb0():
    mesh = W.structured_mesh(2, m=1)
    for sn in (4, 8, 12):
        disc = disc_for(mesh, 1, sn, 1.0, 0.5)
        c = 0.7
        pb = np.full((disc.nd, len(disc.bfaces), 2), c)
        jin = closures.j_in(disc, pb)
        for b, (e, f) in enumerate(disc.bfaces):
            nhat = disc.faces[e][f]["nds"][0] / np.linalg.norm(disc.faces[e][f]["nds"][0])
            on = disc.omega @ nhat
            ref = -c * np.sum(disc.wq[on < 0] * np.abs(on[on < 0]))
            assert np.allclose(jin[b], ref, atol=1e-14)
        eb = closures.eb0(disc, np.array([[1.0, 0.0]]))[0]
        # E_b0 -> 1/2 as N grows (int |Omega.n| dOmega = 2 pi)
        assert abs(eb - 0.5) < {4: 0.05, 8: 0.02, 12: 0.01}[sn]

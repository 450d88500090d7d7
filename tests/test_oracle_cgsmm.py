"""Pins for the oracle's continuous finite element SMM moment system (Sec. 5.1)."""
import math

import numpy as np
import pytest

import smm_workloads as W
from oracle import cgsmm, closures, ipsmm
from oracle.smm import SMMProblem, source_iteration
from tests.oracle_problems import angular_source, disc_for, inflow, linear_problem, mms_problem


@pytest.mark.parametrize("nx,ny,m,p,seed", [(3, 2, 1, 2, None), (4, 3, 2, 3, 5), (2, 2, 3, 4, 1)])
def test_numbering_counts_and_positions(nx, ny, m, p, seed):
    """A structured nx x ny mesh has (nx p + 1)(ny p + 1) continuous nodes, and
    the element nodes that share a global node sit at one physical point."""
    mesh = W.structured_mesh(nx, ny, m=m, perturb_seed=seed)
    disc = disc_for(mesh, p, 4, 1.0, 0.5)
    gid, ng = cgsmm.continuous_numbering(disc)
    assert ng == (nx * p + 1) * (ny * p + 1)
    pos = W.dg_node_positions(mesh, p).reshape(-1, 2)
    for g in range(ng):
        pts = pos[gid.ravel() == g]
        assert np.max(np.abs(pts - pts[0])) < 1e-13


def _random_closures(disc, seed):
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((3, disc.ne, disc.n))
    T = rng.standard_normal((3, disc.ne, disc.n))
    nf = len(disc.elems[0].fq_s)
    jin = rng.standard_normal((len(disc.bfaces), nf))
    beta = rng.standard_normal((len(disc.bfaces), nf))
    return Q, T, jin, beta


@pytest.mark.parametrize("seed", [None, 4])
def test_cg_system_is_ip_system_restricted_to_vp(seed):
    """Sec. 5.1: the CG method is Eq. ipsmm with test and trial space V_p, i.e.
    A_CG = P^T A_IP P and b_CG = P^T b_IP for the injection P: V_p -> Y_p."""
    mesh = W.structured_mesh(3, m=2, perturb_seed=seed)
    rng = np.random.default_rng(1)
    st = np.where(rng.random(9) < 0.5, 50.0, 0.5)
    disc = disc_for(mesh, 2, 4, st, 0.8 * st)
    gid, ng = cgsmm.continuous_numbering(disc)
    P = cgsmm.injection(gid, ng)
    A_cg = cgsmm.assemble_lhs(disc, gid, ng).toarray()
    A_ip = ipsmm.assemble_lhs(disc).toarray()
    R = (P.T @ A_ip @ P)
    assert np.max(np.abs(A_cg - R)) <= 1e-12 * np.max(np.abs(A_ip))
    Q, T, jin, beta = _random_closures(disc, 7)
    b_cg = cgsmm.assemble_rhs(disc, gid, ng, Q, T, jin, beta)
    b_ip = ipsmm.assemble_rhs(disc, Q, T, jin, beta)
    assert np.max(np.abs(b_cg - P.T @ b_ip)) <= 1e-12 * np.max(np.abs(b_ip))


def test_lhs_symmetric_positive_definite():
    mesh = W.structured_mesh(4, m=2, perturb_seed=6)
    rng = np.random.default_rng(0)
    st = np.where(rng.random(16) < 0.5, 200.0, 0.2)
    disc = disc_for(mesh, 2, 4, st, 0.9 * st)
    gid, ng = cgsmm.continuous_numbering(disc)
    A = cgsmm.assemble_lhs(disc, gid, ng).toarray()
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    np.linalg.cholesky(A)


@pytest.mark.parametrize("seed", [None, 3])
def test_linear_solution_is_the_fixed_point(seed):
    """psi = (phi + 3 Omega.J)/4pi with phi linear: T = beta = 0 and the CG
    moment solution is that phi, which is in V_p; the fixed point is exact."""
    mesh, disc, q, pb, phi_ex = linear_problem(4, 2, 2, 4, seed=seed)
    prob = cgsmm.SMMProblemCG(disc, q, pb)
    new, _ = prob.G(phi_ex)
    assert np.max(np.abs(new - phi_ex)) < 1e-12
    phi, k, _ = prob.iterate(tol=1e-12)
    assert np.max(np.abs(phi - phi_ex)) < 1e-11 and k < 30


@pytest.mark.parametrize("p,expect", [(1, 1.8), (2, 2.8)])
def test_moment_system_mms_order(p, expect):
    """Isolated moment-system MMS study with the CG system: closures, Q_0, Q_1
    and J_in from the MMS angular flux; L2 error of varphi at O(h^{p+1})."""
    errs = []
    for nx in (4, 8, 16) if p == 1 else (4, 8):
        mesh = W.structured_mesh(nx, m=3, perturb_seed=7)
        disc = disc_for(mesh, p, 4, 1.0, 0.9)
        psi = angular_source(disc, W.mms_psi)
        q = angular_source(disc, lambda x, y, ox, oy: W.mms_source(x, y, ox, oy, 1.0, 0.9))
        pb = inflow(mesh, disc, W.mms_psi)
        prob = cgsmm.SMMProblemCG(disc, q, pb)
        import scipy.sparse.linalg as spla
        x = spla.spsolve(prob.A.tocsc(), prob.rhs_from_psi(psi))
        errs.append(disc.l2_error((prob.P @ x).reshape(disc.ne, disc.n), W.mms_phi))
    assert math.log2(errs[-2] / errs[-1]) > expect


def test_cg_and_ip_fixed_points_approach_sn():
    """Both SMM discretizations differ from the S_N scalar flux by O(h^{p+1}),
    so from each other too."""
    diffs = []
    for nx in (4, 8):
        mesh, disc, q, pb = mms_problem(nx, 1, 2, 4, seed=None, sigs=0.5)
        phi_cg, _, _ = cgsmm.SMMProblemCG(disc, q, pb).iterate(tol=1e-12)
        phi_sn, _ = source_iteration(disc, q, pb, tol=1e-12)
        diffs.append(disc.l2_error(phi_cg - phi_sn, lambda x, y: 0.0 * x))
    assert math.log2(diffs[0] / diffs[1]) > 2.4


def test_rhs_sum_is_source_minus_boundary_terms():
    """u = 1 is in V_p: the RHS entries sum to int Q_0 - int_Gb (2 J_in + beta)."""
    mesh = W.structured_mesh(3, m=2, perturb_seed=1)
    disc = disc_for(mesh, 2, 4, 1.0, 0.5)
    gid, ng = cgsmm.continuous_numbering(disc)
    psi = angular_source(disc, W.mms_psi)
    q = angular_source(disc, lambda x, y, ox, oy: W.mms_source(x, y, ox, oy, 1.0, 0.5))
    pb = inflow(mesh, disc, W.mms_psi)
    Q = closures.source_moments(disc, q)
    T = closures.nodal_moments(disc, psi)[3:]
    jin, beta = closures.j_in(disc, pb), closures.beta(disc, psi)
    b = cgsmm.assemble_rhs(disc, gid, ng, Q, T, jin, beta)
    ref = disc.integrate(Q[0])
    for bi, (e, f) in enumerate(disc.bfaces):
        ds = np.linalg.norm(disc.faces[e][f]["nds"], axis=1)
        ref -= np.sum(ds * (2 * jin[bi] + beta[bi]))
    assert abs(b.sum() - ref) < 1e-12 * max(1.0, abs(ref))

"""Pins for the oracle's interior penalty SMM moment system (Eq. ipsmm)."""
import math

import numpy as np
import pytest

import smm_workloads as W
from oracle import closures, ipsmm
from oracle.smm import SMMProblem
from tests.oracle_problems import angular_source, disc_for, inflow, linear_problem


def _contrast_disc():
    mesh = W.structured_mesh(4, m=2, perturb_seed=6)
    rng = np.random.default_rng(0)
    st = np.where(rng.random(16) < 0.5, 200.0, 0.2)
    return mesh, disc_for(mesh, 2, 4, st, 0.9 * st)


def test_lhs_symmetric_positive_definite():
    mesh, disc = _contrast_disc()
    A = ipsmm.assemble_lhs(disc).toarray()
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    np.linalg.cholesky(A)


def test_lhs_column_sums_are_absorption_plus_marshak():
    """With u = 1 every jump and gradient term vanishes, so sum_i A_ij is
    int sigma_a phi_j + int_Gb E_b0 phi_j."""
    mesh, disc = _contrast_disc()
    A = ipsmm.assemble_lhs(disc).toarray()
    n = disc.n
    ref = np.zeros(disc.ne * n)
    for e in range(disc.ne):
        ref[e * n:(e + 1) * n] += (disc.sigma_t[e] - disc.sigma_s[e]) * disc.M[e].sum(0)
    for (e, f) in disc.bfaces:
        fd = disc.faces[e][f]
        ds = np.linalg.norm(fd["nds"], axis=1)
        E = closures.eb0(disc, fd["nds"] / ds[:, None])
        ref[e * n:(e + 1) * n] += (E * ds) @ fd["V"]
    assert np.allclose(A.sum(0), ref, atol=1e-12 * np.abs(A).max())


def test_rhs_sum_is_source_minus_boundary_terms():
    """Sum over all test functions (u = 1) of the RHS: int Q_0 - int_Gb (2 J_in + beta)."""
    mesh = W.structured_mesh(3, m=2, perturb_seed=1)
    disc = disc_for(mesh, 2, 4, 1.0, 0.5)
    psi = angular_source(disc, W.mms_psi)
    q = angular_source(disc, lambda x, y, ox, oy: W.mms_source(x, y, ox, oy, 1.0, 0.5))
    pb = inflow(mesh, disc, W.mms_psi)
    Q = closures.source_moments(disc, q)
    T = closures.nodal_moments(disc, psi)[3:]
    jin, beta = closures.j_in(disc, pb), closures.beta(disc, psi)
    b = ipsmm.assemble_rhs(disc, Q, T, jin, beta)
    ref = disc.integrate(Q[0])
    for bi, (e, f) in enumerate(disc.bfaces):
        ds = np.linalg.norm(disc.faces[e][f]["nds"], axis=1)
        ref -= np.sum(ds * (2 * jin[bi] + beta[bi]))
    assert abs(b.sum() - ref) < 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("seed", [None, 3])
def test_consistency_linear_solution(seed):
    """Closures and sources of psi = (phi + 3 Omega.J)/4pi with phi linear:
    the IP-SMM solution is that phi exactly."""
    mesh, disc, q, pb, phi_ex = linear_problem(4, 2, 2, 4, seed=seed)
    psi = angular_source(disc, W.linear_aniso_psi)
    prob = SMMProblem(disc, q, pb)
    x = ipsmm.solve(prob.A, prob.rhs_from_psi(psi)).reshape(disc.ne, disc.n)
    assert np.max(np.abs(x - phi_ex)) < 1e-12


@pytest.mark.parametrize("p,expect", [(1, 1.8), (2, 2.8), (3, 3.6)])
def test_moment_system_mms_order(p, expect):
    """Paper's isolated moment-system MMS study: closures, Q_0, Q_1 and J_in
    from the MMS angular flux (S4) on a curved order-3 mesh; L2 error of
    varphi converges at O(h^{p+1})."""
    errs = []
    sizes = (4, 8, 16) if p == 1 else (4, 8)
    for nx in sizes:
        mesh = W.structured_mesh(nx, m=3, perturb_seed=7)
        disc = disc_for(mesh, p, 4, 1.0, 0.9)
        psi = angular_source(disc, W.mms_psi)
        q = angular_source(disc, lambda x, y, ox, oy: W.mms_source(x, y, ox, oy, 1.0, 0.9))
        pb = inflow(mesh, disc, W.mms_psi)
        prob = SMMProblem(disc, q, pb)
        x = ipsmm.solve(prob.A, prob.rhs_from_psi(psi)).reshape(disc.ne, disc.n)
        errs.append(disc.l2_error(x, W.mms_phi))
    assert math.log2(errs[-2] / errs[-1]) > expect


def test_rhs_tensor_terms_are_the_diffusion_form_for_isotropic_T():
    """For T = tau phi I, with phi any broken (discontinuous) function that
    vanishes on the boundary faces, the three T-terms of Eq. ipsmm's
    right-hand side (volume divergence, face average of div T . n against
    [u], face average of grad u against [T n]) discretize div((1/sigma_t)
    div T) = 3 tau div(D grad phi) exactly as the left-hand side's diffusion
    terms do: they equal -3 tau times its penalty-free form (sigma_a = 0 here,
    element-wise sigma_t)."""
    from oracle.fem import face_nodes
    mesh = W.structured_mesh(4, 3, m=2, perturb_seed=6)
    ne = mesh.n_elem
    st = 1.0 + 0.5 * (np.arange(ne) % 3)
    disc = disc_for(mesh, 2, 4, st, st)
    rng = np.random.default_rng(5)
    phi = rng.uniform(-1.0, 1.0, (ne, disc.n))
    for (e, f) in disc.bfaces:
        phi[e, face_nodes(disc.p, f)] = 0.0
    tau = 0.7
    A0 = ipsmm.assemble_lhs(disc, kappa_scale=0.0)
    nb, nfq = len(disc.bfaces), len(disc.elems[0].fq_s)
    z = np.zeros((nb, nfq))
    b = ipsmm.assemble_rhs(disc, np.zeros((3, ne, disc.n)), np.stack([tau * phi, 0.0 * phi, tau * phi]), z, z)
    want = -3.0 * tau * (A0 @ phi.ravel())
    assert np.max(np.abs(b - want)) <= 1e-12 * np.max(np.abs(want))

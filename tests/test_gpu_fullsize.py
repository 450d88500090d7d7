"""GPU parity at the full bench configuration, on sampled outputs.

Workload: the curved manufactured-solution problem on a 128x128 mesh of
geometry order 3, DG order 4, S8 (40 ordinates), sigma_t = 1, c = 0.9, with
the library's default (bench) configuration: FP64 sweep with cached local
inverses, multigrid-preconditioned CG.  The oracle cannot sweep 16.4 M angular
unknowns in seconds, so it checks sampled outputs one at a time on a patch of
at most 3x3 elements around each sampled element (the patch holds every
element a sampled quantity depends on):

- sweep: the oracle's local DG solve of (element, ordinate), fed the GPU's
  upwind angular flux (or the inflow data), reproduces the GPU's psi;
- moments: the quadrature sums of the GPU's psi reproduce its moments;
- moment solve: the GPU's solution satisfies the sampled element's rows of
  the oracle's IP-SMM system (Eq. ipsmm) built from the GPU's closures;
- converged scalar flux: agrees with the manufactured phi (Sec. 6.1) to the
  discretization error, a property that holds at any size.
"""
import numpy as np
import pytest

import smm_workloads as W
from tests.parity_inputs import problem, sources

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NX, M, P_ORDER, SN = 128, 3, 4, 8


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_07386_gb300 as P
    from paper_2304_07386_gb300 import build as B
    B.build()
    prob = problem(NX, m=M, p=P_ORDER, sn=SN, seed=0, sigt=1.0, c=0.9, kind="mms")
    om, _ = P.smm_quadrature(SN)
    q, inflow = sources(prob, om)
    mesh = prob["mesh"]
    h = P.smm_create(mesh.nodes, mesh.elem_nodes, M, P_ORDER, SN, prob["sigma_t"], prob["sigma_s"], q,
                     inflow=inflow, options=P.smm_default_options())
    info = h.info()
    ne, nd, n = info.n_elem, info.n_ord, info.n_dof_elem
    phi = torch.zeros(ne * n, dtype=torch.float64, device="cuda")
    for _ in range(3):                                       # the bench's step state
        P.smm_iterate(h, phi, 1e-300, 1, relative=True, raise_on_error=False)
    phi3 = phi.clone()
    P.smm_sweep(h, phi3)
    psi = torch.zeros(ne * nd * n, dtype=torch.float64, device="cuda")
    P.smm_get_psi(h, psi)
    mom = torch.zeros(6 * ne * n, dtype=torch.float64, device="cuda")
    beta = torch.zeros(info.n_bface * info.n_fq, dtype=torch.float64, device="cuda")
    P.smm_moments(h, mom, beta)
    sol = phi3.clone()
    cg_iters = P.smm_moment_solve(h, sol)
    yield dict(P=P, h=h, prob=prob, ne=ne, nd=nd, n=n, phi3=phi3.cpu().numpy().reshape(ne, n),
               psi=psi.cpu().numpy().reshape(ne, nd, n), mom=mom.cpu().numpy().reshape(6, ne, n),
               sol=sol.cpu().numpy().reshape(ne, n), cg_iters=cg_iters)
    h.destroy()


def samples():
    rng = np.random.default_rng(2024)
    edge = [(0, 0), (NX - 1, 0), (0, NX - 1), (NX - 1, NX - 1), (NX // 2, 0), (0, NX // 3), (NX - 1, 77),
            (51, NX - 1)]
    inner = [tuple(v) for v in rng.integers(1, NX - 1, size=(10, 2))]
    return [j * NX + i for i, j in edge + inner]


def patch(F, E):
    """Oracle discretization of the elements within one index of E (clipped at
    the domain boundary); returns (disc, element list, index of E, psibar)."""
    from oracle.transport import Discretization
    prob = F["prob"]
    mesh = prob["mesh"]
    i0, j0 = E % NX, E // NX
    els = [j * NX + i for j in range(max(0, j0 - 1), min(NX, j0 + 2)) for i in range(max(0, i0 - 1), min(NX, i0 + 2))]
    disc = Discretization(mesh.nodes, mesh.elem_nodes[els], M, P_ORDER, SN, prob["sigma_t"][els],
                          prob["sigma_s"][els])
    c = els.index(E)
    # inflow data on the patch's boundary faces that lie on the domain boundary (others never reach E)
    pos = prob["pos"]
    psibar = np.zeros((disc.nd, len(disc.bfaces), P_ORDER + 1))
    for b, (e, f) in enumerate(disc.bfaces):
        g = els[e]
        gi, gj = g % NX, g // NX
        on_domain = (f == 0 and gj == 0) or (f == 1 and gi == NX - 1) or (f == 2 and gj == NX - 1) or \
                    (f == 3 and gi == 0)
        if not on_domain:
            continue
        a = np.arange(P_ORDER + 1)
        k = P_ORDER + 1
        idx = [a, a * k + P_ORDER, P_ORDER * k + a, a * k][f]
        xy = pos[g, idx]
        for d in range(disc.nd):
            psibar[d, b] = W.mms_psi(xy[:, 0], xy[:, 1], disc.omega[d, 0], disc.omega[d, 1])
    return disc, els, c, psibar


def patch_source(F, disc, els):
    """MMS source q_d at the patch elements' nodes, [nd][len(els)][n]."""
    prob = F["prob"]
    pos = prob["pos"][els]
    st, ss = prob["sigma_t"][els], prob["sigma_s"][els]
    return np.stack([W.mms_source(pos[:, :, 0], pos[:, :, 1], o[0], o[1], st[:, None], ss[:, None])
                     for o in disc.omega])


def test_sampled_sweep_tasks_match_oracle_local_solves(full):
    F = full
    for E in samples():
        disc, els, c, psibar = patch(F, E)
        q = patch_source(F, disc, els)
        scat = (disc.sigma_s / (4.0 * np.pi))[:, None] * F["phi3"][els]
        psi_patch = F["psi"][els].transpose(1, 0, 2)               # [nd][len(els)][n], GPU values
        for d in range(disc.nd):
            A = disc.local_matrix(c, d)
            b = disc.M[c] @ (scat[c] + q[d][c])
            for f in range(4):
                fd = disc.faces[c][f]
                neg = np.minimum(fd["nds"] @ disc.omega[d], 0.0)
                if np.any(neg < 0.0):
                    up = disc.upwind_values(c, f, d, psi_patch[d], psibar)
                    b = b - fd["V"].T @ (neg * up)
            x = np.linalg.solve(A, b)
            gpu = F["psi"][E, d]
            assert np.max(np.abs(gpu - x)) <= 1e-11 * max(np.max(np.abs(x)), 1e-300), (E, d)


def test_sampled_moments_match_quadrature_sums(full):
    from oracle import closures
    F = full
    for E in samples():
        disc, els, c, _ = patch(F, E)
        mom_o = closures.nodal_moments(disc, F["psi"][els].transpose(1, 0, 2))[:, c]
        mom_g = F["mom"][:, E]
        scale = np.max(np.abs(mom_o[0]))
        assert np.max(np.abs(mom_g - mom_o)) <= 1e-11 * scale, E


def test_moment_solve_satisfies_sampled_ipsmm_rows(full):
    from oracle import closures, ipsmm
    F = full
    n = F["n"]
    assert 0 < F["cg_iters"] < 200
    for E in samples():
        disc, els, c, psibar = patch(F, E)
        q = patch_source(F, disc, els)
        A = ipsmm.assemble_lhs(disc).tocsr()
        Q = closures.source_moments(disc, q)
        T = F["mom"][3:6][:, els]
        psi_patch = F["psi"][els].transpose(1, 0, 2)
        b = ipsmm.assemble_rhs(disc, Q, T, closures.j_in(disc, psibar), closures.beta(disc, psi_patch))
        x = F["sol"][els].ravel()
        rows = slice(c * n, (c + 1) * n)
        r = A[rows] @ x - b[rows]
        scale = np.max(np.abs(b[rows])) + np.max(np.abs(A[rows] @ x))
        assert np.max(np.abs(r)) <= 1e-8 * scale, (E, np.max(np.abs(r)) / scale)


def test_converged_flux_matches_manufactured_solution(full):
    F = full
    P, h = F["P"], F["h"]
    ne, n = F["ne"], F["n"]
    x = torch.zeros(ne * n, dtype=torch.float64, device="cuda")
    rc, stats = P.smm_iterate(h, x, 1e-10, 100, relative=True)
    assert rc == 0 and stats["outer_iterations"] < 40
    pos = F["prob"]["pos"]
    exact = W.mms_phi(pos[:, :, 0], pos[:, :, 1])
    err = np.max(np.abs(x.cpu().numpy().reshape(ne, n) - exact)) / np.max(np.abs(exact))
    # discretization error of p = 4 on h = 1/128 (order p+1), far below any path error
    assert err < 1e-7, err

"""GPU parity at the full size of the thick/thin workload, on sampled outputs.

Workload: 256x256 straight quads on [0,8]^2, 8x8 blocks of 32x32 elements,
each thick (sigma_t = 200, c = 0.999) or thin (sigma_t = 0.2, c = 0.5)
(seed 0), isotropic source 1 per steradian in the lowest-index thin block,
vacuum boundaries, p = 3, S12 (84 ordinates): 88.1 M angular unknowns per
sweep, in the library's default configuration (FP64-accuracy sweep with
cached local inverses as FP32 pairs, multigrid CG), the state of the fourth
outer step from varphi = 0.  The oracle checks sampled outputs one at a time
on the patch of at most 3x3 elements around each sampled element: the local
DG solve of every ordinate fed the GPU's upwind flux, the moments as
quadrature sums of the GPU's flux, and the sampled element's rows of the
IP-SMM system (Eq. ipsmm) built from the GPU's closures.  The samples sit on
block corners and edges (material jumps of 1000 in sigma_t), on the domain
edges and inside blocks.
"""
import numpy as np
import pytest

import smm_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NX, BLOCKS, P_ORDER, SN, LENGTH = 256, 8, 3, 12, 8.0


def inputs():
    mesh = W.structured_mesh(NX, m=1, domain=(0.0, LENGTH, 0.0, LENGTH))
    st, ss, blk, thick = W.block_materials(NX, BLOCKS, 0)
    src_blk = int(np.flatnonzero(~thick)[0])
    q = np.repeat((blk == src_blk).astype(np.float64)[:, None], (P_ORDER + 1) ** 2, axis=1)
    return mesh, st, ss, q


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2304_07386_gb300 as P
    from paper_2304_07386_gb300 import build as B
    B.build()
    mesh, st, ss, q = inputs()
    h = P.smm_create(mesh.nodes, mesh.elem_nodes, 1, P_ORDER, SN, st, ss, q, options=P.smm_default_options())
    info = h.info()
    ne, nd, n = info.n_elem, info.n_ord, info.n_dof_elem
    phi = torch.zeros(ne * n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        P.smm_iterate(h, phi, 1e-300, 1, relative=True, raise_on_error=False)
    phi3 = phi.clone()
    P.smm_sweep(h, phi3)
    psi = torch.zeros(ne * nd * n, dtype=torch.float64, device="cuda")
    P.smm_get_psi(h, psi)
    mom = torch.zeros(6 * ne * n, dtype=torch.float64, device="cuda")
    P.smm_moments(h, mom)
    sol = phi3.clone()
    cg_iters = P.smm_moment_solve(h, sol)
    yield dict(mesh=mesh, st=st, ss=ss, q=q, ne=ne, nd=nd, n=n, phi3=phi3.cpu().numpy().reshape(ne, n),
               psi=psi.cpu().numpy().reshape(ne, nd, n), mom=mom.cpu().numpy().reshape(6, ne, n),
               sol=sol.cpu().numpy().reshape(ne, n), cg_iters=cg_iters)
    h.destroy()


def samples():
    b = NX // BLOCKS
    rng = np.random.default_rng(7)
    corners = [(b - 1, b - 1), (b, b), (3 * b, 5 * b - 1), (4 * b - 1, 2 * b)]    # block corners
    edges = [(b // 2, 3 * b), (5 * b - 1, b // 3), (2 * b, 6 * b + 7)]            # block edges
    domain = [(0, 0), (NX - 1, 0), (0, NX - 1), (NX - 1, NX - 1), (NX // 2, 0), (0, 77), (NX - 1, 130)]
    inner = [tuple(v) for v in rng.integers(1, NX - 1, size=(6, 2))]
    return [j * NX + i for i, j in corners + edges + domain + inner]


def patch(F, E):
    """Oracle discretization of the elements within one index of E (clipped
    at the domain boundary); returns (disc, element list, index of E)."""
    from oracle.transport import Discretization
    mesh = F["mesh"]
    i0, j0 = E % NX, E // NX
    els = [j * NX + i for j in range(max(0, j0 - 1), min(NX, j0 + 2)) for i in range(max(0, i0 - 1), min(NX, i0 + 2))]
    disc = Discretization(mesh.nodes, mesh.elem_nodes[els], 1, P_ORDER, SN, F["st"][els], F["ss"][els])
    return disc, els, els.index(E)


def test_sampled_sweep_tasks_match_oracle_local_solves(full):
    F = full
    for E in samples():
        disc, els, c = patch(F, E)
        psibar = np.zeros((disc.nd, len(disc.bfaces), P_ORDER + 1))     # vacuum
        scat = (disc.sigma_s / (4.0 * np.pi))[:, None] * F["phi3"][els]
        psi_patch = F["psi"][els].transpose(1, 0, 2)
        for d in range(disc.nd):
            A = disc.local_matrix(c, d)
            b = disc.M[c] @ (scat[c] + F["q"][els][c])
            for f in range(4):
                fd = disc.faces[c][f]
                neg = np.minimum(fd["nds"] @ disc.omega[d], 0.0)
                if np.any(neg < 0.0):
                    up = disc.upwind_values(c, f, d, psi_patch[d], psibar)
                    b = b - fd["V"].T @ (neg * up)
            x = np.linalg.solve(A, b)
            gpu = F["psi"][E, d]
            scale = max(np.max(np.abs(x)), 1e-300)
            assert np.max(np.abs(gpu - x)) <= 1e-11 * scale, (E, d, np.max(np.abs(gpu - x)) / scale)


def test_sampled_moments_match_quadrature_sums(full):
    from oracle import closures
    F = full
    for E in samples():
        disc, els, c = patch(F, E)
        mom_o = closures.nodal_moments(disc, F["psi"][els].transpose(1, 0, 2))[:, c]
        mom_g = F["mom"][:, E]
        scale = np.max(np.abs(mom_o[0]))
        assert np.max(np.abs(mom_g - mom_o)) <= 1e-11 * scale, E


def test_moment_solve_satisfies_sampled_ipsmm_rows(full):
    """The CG stops when ||r||_2 <= 1e-12 ||b||_2 over the whole system, which
    bounds every row's residual by sqrt(N) 1e-12 ||b||_inf ~ 1e-9 ||b||_inf.
    The flux here spans many orders of magnitude (thick blocks attenuate it
    by ~1e-12 towards the far corners), so each sampled row is checked
    against 1e-8 of its own scale plus 1e-8 of the largest row scale, taken
    at the element where the solution peaks (near the source)."""
    from oracle import closures, ipsmm
    F = full
    n = F["n"]
    assert 0 < F["cg_iters"] < 200

    def row_residual(E):
        disc, els, c = patch(F, E)
        psibar = np.zeros((disc.nd, len(disc.bfaces), P_ORDER + 1))
        q = np.broadcast_to(F["q"][els], (disc.nd,) + F["q"][els].shape)
        A = ipsmm.assemble_lhs(disc).tocsr()
        Q = closures.source_moments(disc, q)
        T = F["mom"][3:6][:, els]
        psi_patch = F["psi"][els].transpose(1, 0, 2)
        b = ipsmm.assemble_rhs(disc, Q, T, closures.j_in(disc, psibar), closures.beta(disc, psi_patch))
        x = F["sol"][els].ravel()
        rows = slice(c * n, (c + 1) * n)
        r = A[rows] @ x - b[rows]
        return np.max(np.abs(r)), np.max(np.abs(b[rows])) + np.max(np.abs(A[rows] @ x))

    peak = int(np.argmax(np.max(np.abs(F["sol"]), axis=1)))
    r_peak, global_scale = row_residual(peak)
    assert r_peak <= 1e-8 * global_scale, (peak, r_peak / global_scale)
    for E in samples():
        r, scale = row_residual(E)
        assert r <= 1e-8 * (scale + global_scale), (E, r / scale, r / global_scale)

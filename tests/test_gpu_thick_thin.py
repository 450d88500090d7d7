"""Multi-material thick/thin workload (Sec. 6.3's 1000x contrast): [0,8]^2,
8x8 (or 4x4) blocks, each thick (sigma_t = 200, c = 0.999) or thin
(sigma_t = 0.2, c = 0.5) by a seeded coin, unit isotropic source in the
lowest-index thin block, vacuum boundaries, p = 3, S12.

- small mesh: converged GPU scalar flux equals the oracle's;
- full 256x256 mesh: the iteration converges, and the converged solution
  satisfies the IP-SMM particle balance that testing Eq. ipsmm with v = 1
  gives (every jump and gradient term drops out):
      int sigma_a phi + int_dD (E_b0 phi + beta) ds = int Q_0 = 4 pi |source block|,
  a property that holds at any size.
"""
import math

import numpy as np
import pytest

import smm_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

L, P_ORDER, SN = 8.0, 3, 12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_07386_gb300 import build as B
    B.build()


def workload(nx, blocks, seed=0):
    mesh = W.structured_mesh(nx, m=1, domain=(0.0, L, 0.0, L))
    st, ss, blk, thick = W.block_materials(nx, blocks, seed)
    src_blk = int(np.flatnonzero(~thick)[0])
    n = (P_ORDER + 1) ** 2
    q = np.repeat((blk == src_blk).astype(np.float64)[:, None], n, axis=1)
    return mesh, st, ss, q, thick


def solve_gpu(mesh, st, ss, q, tol):
    import paper_2304_07386_gb300 as P
    h = P.smm_create(mesh.nodes, mesh.elem_nodes, 1, P_ORDER, SN, st, ss, q, options=P.smm_default_options())
    info = h.info()
    x = torch.zeros(info.n_elem * info.n_dof_elem, dtype=torch.float64, device="cuda")
    rc, stats = P.smm_iterate(h, x, tol, 200, relative=True)
    return h, info, x.cpu().numpy().reshape(info.n_elem, info.n_dof_elem), rc, stats


def test_thick_thin_small_matches_oracle():
    from oracle.smm import SMMProblem
    from oracle.transport import Discretization
    mesh, st, ss, q, thick = workload(8, 4, seed=1)
    assert thick.any() and (~thick).any()
    h, info, phi_g, rc, stats = solve_gpu(mesh, st, ss, q, 1e-12)
    h.destroy()
    assert rc == 0
    disc = Discretization(mesh.nodes, mesh.elem_nodes, 1, P_ORDER, SN, st, ss)
    phi_o, _, hist = SMMProblem(disc, q).iterate(tol=1e-13, relative=True)
    err = np.max(np.abs(phi_g - phi_o)) / np.max(np.abs(phi_o))
    assert err < 1e-9, err
    its = 1 + next(k for k, dv in enumerate(hist) if dv < 1e-12)   # the oracle's count at the GPU's tolerance
    assert abs(stats["outer_iterations"] - its) <= 1, (stats["outer_iterations"], its)


def test_thick_thin_full_size_converges_and_balances():
    import paper_2304_07386_gb300 as P
    nx, blocks = 256, 8
    mesh, st, ss, q, thick = workload(nx, blocks)
    h, info, phi, rc, stats = solve_gpu(mesh, st, ss, q, 1e-8)
    try:
        assert rc == 0 and stats["outer_iterations"] <= 100, stats
        print("thick/thin 256^2 p=3 S12: outer", stats["outer_iterations"], "CG per outer",
              stats["cg_total"] / stats["outer_iterations"], "max", stats["cg_max"])
        ne, n, p1 = info.n_elem, info.n_dof_elem, P_ORDER + 1
        mom = torch.zeros(6 * ne * n, dtype=torch.float64, device="cuda")
        beta = torch.zeros(info.n_bface * info.n_fq, dtype=torch.float64, device="cuda")
        P.smm_moments(h, mom, beta)
        beta = beta.cpu().numpy().reshape(info.n_bface, info.n_fq)
    finally:
        h.destroy()
    hx = L / nx
    gll = W.gauss_lobatto_points(p1)     # nodes on [0, 1]; weights from exactness on degree < p+1
    V = np.vander(gll, p1, increasing=True).T                # V[k][a] = x_a^k
    wl = np.linalg.solve(V, 1.0 / np.arange(1, p1 + 1))       # int_0^1 x^k = sum_a w_a x_a^k
    w2 = np.outer(wl, wl).ravel()                             # node i = iy * p1 + ix
    absorb = hx * hx * np.sum((st - ss)[:, None] * phi * w2[None, :])
    om, wq = P.smm_quadrature(SN)
    eb0 = np.sum(wq * np.abs(om[:, 0])) / (4.0 * math.pi)     # the same for x and y normals (octant symmetry)
    assert abs(eb0 - np.sum(wq * np.abs(om[:, 1])) / (4.0 * math.pi)) < 1e-14
    edge = 0.0
    e = np.arange(ne)
    i, j = e % nx, e // nx
    a = np.arange(p1)
    for f, sel, idx in ((0, j == 0, a), (1, i == nx - 1, a * p1 + P_ORDER), (2, j == nx - 1, P_ORDER * p1 + a),
                        (3, i == 0, a * p1)):
        edge += hx * np.sum(phi[sel][:, idx] * wl[None, :])
    leak = eb0 * edge + hx * np.sum(beta * gauss_weights(info.n_fq)[None, :])
    q0 = 4.0 * math.pi * 1.0
    assert abs(absorb + leak - q0) < 1e-8 * q0, (absorb, leak, q0)


def gauss_weights(k):
    """Gauss-Legendre weights on [0, 1] (numpy's rule, rescaled)."""
    _, w = np.polynomial.legendre.leggauss(k)
    return w / 2.0

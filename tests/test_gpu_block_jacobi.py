"""GPU parallel block Jacobi sweep (Sec. 6.5) vs the oracle: two consecutive
sweeps (the second lagging the first across tiles) to 1e-11 for both local
solvers, and the SMM iteration to the oracle's fixed point (1e-9) with the
same outer-iteration count (within one)."""
import numpy as np
import pytest

from tests.parity_inputs import oracle_disc, problem, sources

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_07386_gb300 import build as B
    B.build()


def make_gpu(prob, tiles, solver):
    import paper_2304_07386_gb300 as P
    om, _ = P.smm_quadrature(prob["sn"])
    q, inflow = sources(prob, om)
    opt = P.smm_default_options()
    opt.sweep_tiles = tiles
    opt.sweep_solver = solver
    opt.tol_cg = 1e-13
    mesh = prob["mesh"]
    return P.smm_create(mesh.nodes, mesh.elem_nodes, mesh.m, prob["p"], prob["sn"], prob["sigma_t"], prob["sigma_s"],
                        q, inflow=inflow, options=opt)


@pytest.mark.parametrize("solver", [0, 1], ids=["lu", "cached_inverse"])
@pytest.mark.parametrize("case", [(8, 2, 2, 4, 3, 4), (12, 3, 3, 8, 5, 3), (9, 1, 4, 4, None, 2)],
                         ids=lambda c: "x".join(map(str, c)))
def test_block_jacobi_sweeps_match_oracle(case, solver):
    import paper_2304_07386_gb300 as P
    import smm_workloads as W
    nx, m, p, sn, seed, tiles = case
    prob = problem(nx, m=m, p=p, sn=sn, seed=seed, kind="mms", c=0.6)
    h = make_gpu(prob, tiles, solver)
    disc = oracle_disc(prob)
    q, inflow = sources(prob, disc.omega)
    block = disc.element_tiles(tiles)
    phi = W.mms_phi(prob["pos"][:, :, 0], prob["pos"][:, :, 1])
    info = h.info()
    lag = np.zeros((disc.nd, disc.ne, disc.n))
    for _ in range(2):
        P.smm_sweep(h, torch.as_tensor(phi.ravel(), device="cuda"))
        psi = torch.zeros(info.n_elem * info.n_ord * info.n_dof_elem, dtype=torch.float64, device="cuda")
        P.smm_get_psi(h, psi)
        psi_g = psi.cpu().numpy().reshape(info.n_elem, info.n_ord, info.n_dof_elem).transpose(1, 0, 2)
        psi_o = disc.sweep(phi, q, inflow, block=block, psi_lag=lag)
        assert np.max(np.abs(psi_g - psi_o)) <= 1e-11 * np.max(np.abs(psi_o))
        lag = psi_o
    h.destroy()


def test_block_jacobi_iteration_matches_oracle():
    import paper_2304_07386_gb300 as P
    from oracle.smm import SMMProblem
    prob = problem(8, m=2, p=2, sn=4, seed=3, kind="mms", c=0.6)
    disc = oracle_disc(prob)
    q, inflow = sources(prob, disc.omega)
    phi_o, k_o, _ = SMMProblem(disc, q, inflow, tiles=4).iterate(tol=1e-12, relative=True)
    phi_exact, k_exact, _ = SMMProblem(disc, q, inflow).iterate(tol=1e-12, relative=True)
    h = make_gpu(prob, 4, 1)
    x = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    rc, stats = P.smm_iterate(h, x, 1e-12, 200, relative=True)
    info = h.info()
    h.destroy()
    xg = x.cpu().numpy().reshape(disc.ne, disc.n)
    assert rc == 0 and abs(stats["outer_iterations"] - k_o) <= 1
    assert np.max(np.abs(xg - phi_o)) <= 1e-9 * np.max(np.abs(phi_o))
    assert np.max(np.abs(xg - phi_exact)) <= 1e-9 * np.max(np.abs(phi_exact))   # same fixed point as the exact sweep
    assert k_o > k_exact and info.n_levels < 15

"""GPU continuous finite element SMM moment system (Sec. 5.1) vs the oracle.

The library's continuous path (options.moment_discretization = SMM_MOMENT_CG)
against oracle.cgsmm: the moment solve alone with the oracle's closures, and
the converged SMM fixed point, on straight and curved meshes, p = 1..4, ragged
sizes.  Tolerance 1e-9 relative (CG at 1e-13 on systems with condition numbers
up to ~1e6), outer-iteration counts within one.
"""
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


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def make_gpu(prob, **kw):
    import paper_2304_07386_gb300 as P
    om, _ = P.smm_quadrature(prob["sn"])
    q, inflow = sources(prob, om)
    opt = P.smm_default_options()
    opt.moment_discretization = P.smm.SMM_MOMENT_CG
    opt.tol_cg = 1e-13
    for k, v in kw.items():
        setattr(opt, k, v)
    mesh = prob["mesh"]
    return P.smm_create(mesh.nodes, mesh.elem_nodes, mesh.m, prob["p"], prob["sn"], prob["sigma_t"], prob["sigma_s"],
                        q, inflow=inflow, options=opt)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


CASES = [
    # (nx, ny, m, p, sn, seed, kind)
    (5, 3, 2, 1, 4, 3, "mms"),
    (4, 4, 2, 2, 8, 5, "mms"),
    (3, 5, 3, 3, 4, 7, "mms"),
    (3, 3, 3, 4, 4, 2, "mms"),
    (12, 9, 1, 2, 4, None, "iso"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[:5])))
def test_cg_moment_solve_matches_oracle(case):
    import scipy.sparse.linalg as spla
    import paper_2304_07386_gb300 as P
    from oracle import cgsmm, closures
    import smm_workloads as W
    nx, ny, m, p, sn, seed, kind = case
    prob = problem(nx, ny, m=m, p=p, sn=sn, seed=seed, kind=kind, c=0.6)
    h = make_gpu(prob)
    disc = oracle_disc(prob)
    q, inflow = sources(prob, disc.omega)
    phi = W.mms_phi(prob["pos"][:, :, 0], prob["pos"][:, :, 1])
    psi = disc.sweep(phi, q, inflow)
    op = cgsmm.SMMProblemCG(disc, q, inflow)
    x_o = op.P @ spla.spsolve(op.A.tocsc(), op.rhs_from_psi(psi))
    mom = closures.nodal_moments(disc, psi)
    beta = closures.beta(disc, psi)
    P.smm_set_moments(h, dev(mom), dev(beta))
    x = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    its = P.smm_moment_solve(h, x)
    h.destroy()
    x_g = x.cpu().numpy()
    assert rel(x_g, x_o) < 1e-9, rel(x_g, x_o)
    assert 0 < its < 200
    # a V_p function: equal values at the element nodes of every global node
    gid = op.gid.ravel()
    for g in range(op.nglob):
        vals = x_g[gid == g]
        assert np.max(vals) - np.min(vals) <= 1e-12 * np.max(np.abs(x_g))


@pytest.mark.parametrize("case", CASES[:4], ids=lambda c: "x".join(map(str, c[:5])))
def test_cg_fixed_point_matches_oracle(case):
    import paper_2304_07386_gb300 as P
    from oracle import cgsmm
    nx, ny, m, p, sn, seed, kind = case
    prob = problem(nx, ny, m=m, p=p, sn=sn, seed=seed, kind=kind, c=0.6)
    h = make_gpu(prob)
    disc = oracle_disc(prob)
    q, inflow = sources(prob, disc.omega)
    phi_o, k_o, _ = cgsmm.SMMProblemCG(disc, q, inflow).iterate(tol=1e-12, relative=True)
    x = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    rc, stats = P.smm_iterate(h, x, 1e-12, 100, relative=True)
    h.destroy()
    assert rc == 0
    assert rel(x.cpu().numpy().reshape(disc.ne, disc.n), phi_o) < 1e-9
    assert abs(stats["outer_iterations"] - k_o) <= 1


def test_cg_multigrid_iterations_bounded_in_h():
    """The V-cycle keeps CG iteration counts nearly flat under refinement."""
    import paper_2304_07386_gb300 as P
    counts = []
    for nx in (16, 32, 64):
        prob = problem(nx, m=1, p=2, sn=4, kind="iso", c=0.9)
        h = make_gpu(prob, tol_cg=1e-10)
        x = torch.zeros(prob["mesh"].n_elem * 9, dtype=torch.float64, device="cuda")
        P.smm_sweep(h, x)
        counts.append(P.smm_moment_solve(h, x))
        h.destroy()
    assert counts[-1] < 1.6 * counts[0] + 5, counts

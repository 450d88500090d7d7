"""GPU (C ABI, sm_103a kernels) vs. oracle parity.

Tolerances: FP64 path 1e-11 relative (max norm over the array, relative to
its max magnitude) per sweep and for the moments; 1e-9 on converged scalar
fluxes.  The FP32-refined path is compared to the FP64 oracle at the
tolerance its stopping test implies (stated in each test).
"""
import math

import numpy as np
import pytest

import smm_workloads as W
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
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def make_gpu(prob, precision=0, **kw):
    import paper_2304_07386_gb300 as P
    om, w = P.smm_quadrature(prob["sn"])
    q, inflow = sources(prob, om)
    opt = P.smm_default_options()
    opt.sweep_precision = precision
    for k, v in kw.items():
        setattr(opt, k, v)
    mesh = prob["mesh"]
    h = P.smm_create(mesh.nodes, mesh.elem_nodes, mesh.m, prob["p"], prob["sn"], prob["sigma_t"], prob["sigma_s"],
                     q, inflow=inflow, options=opt)
    return h


def make_oracle(prob, kappa_scale=1.0):
    from oracle.smm import SMMProblem
    disc = oracle_disc(prob)
    q, inflow = sources(prob, disc.omega)
    return disc, SMMProblem(disc, q, inflow, kappa_scale), q, inflow


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


CASES = [
    # (nx, ny, m, p, sn, seed, kind)
    (5, 3, 2, 1, 4, 3, "mms"),
    (4, 4, 2, 2, 8, 5, "mms"),
    (3, 5, 3, 3, 4, 7, "mms"),
    (3, 3, 3, 4, 4, 2, "mms"),
    (1, 1, 1, 2, 6, None, "mms"),
    (7, 1, 1, 1, 12, None, "iso"),
]


@pytest.mark.parametrize("solver", [0, 1], ids=["lu", "cached_inverse"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[:5])))
def test_sweep_and_moments_fp64(case, solver):
    import paper_2304_07386_gb300 as P
    from oracle import closures
    nx, ny, m, p, sn, seed, kind = case
    prob = problem(nx, ny, m=m, p=p, sn=sn, seed=seed, kind=kind, c=0.6)
    h = make_gpu(prob, sweep_solver=solver)
    disc, op, q, inflow = make_oracle(prob)
    phi = W.mms_phi(prob["pos"][:, :, 0], prob["pos"][:, :, 1])
    P.smm_sweep(h, dev(phi))
    info = h.info()
    psi_g = torch.zeros(info.n_elem * info.n_ord * info.n_dof_elem, dtype=torch.float64, device="cuda")
    P.smm_get_psi(h, psi_g)
    psi_g = psi_g.cpu().numpy().reshape(info.n_elem, info.n_ord, info.n_dof_elem).transpose(1, 0, 2)
    psi_o = disc.sweep(phi, q, inflow)
    assert rel(psi_g, psi_o) < 1e-11
    mom = torch.zeros(6 * info.n_elem * info.n_dof_elem, dtype=torch.float64, device="cuda")
    beta = torch.zeros(info.n_bface * info.n_fq, dtype=torch.float64, device="cuda")
    P.smm_moments(h, mom, beta)
    mom_o = closures.nodal_moments(disc, psi_o)
    mom_g = mom.cpu().numpy().reshape(6, info.n_elem, info.n_dof_elem)
    for c in range(6):
        assert rel(mom_g[c], mom_o[c]) < 1e-11 or np.max(np.abs(mom_g[c] - mom_o[c])) < 1e-12 * np.max(np.abs(mom_o[0]))
    beta_o = closures.beta(disc, psi_o)
    assert np.max(np.abs(beta.cpu().numpy().reshape(beta_o.shape) - beta_o)) < 1e-11 * np.max(np.abs(mom_o[0]))


@pytest.mark.parametrize("solver", [0, 1], ids=["lu", "cached_inverse"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_sweep_with_three_inflow_faces_on_a_fan_mesh(p, solver):
    """Trapezoids widening upwards: ordinates pointing up enter some elements
    through three faces.  Flux and moments against the oracle at 1e-11, as
    above."""
    import paper_2304_07386_gb300 as P
    from oracle import closures
    prob = problem(5, 4, m=1, p=p, sn=8, kind="mms", c=0.6, fan=1.5)
    h = make_gpu(prob, sweep_solver=solver)
    disc, op, q, inflow = make_oracle(prob)
    assert any(sum(bool(np.all(disc.faces[e][f]["nds"] @ disc.omega[d] < 0.0)) for f in range(4)) == 3
               for e in range(disc.ne) for d in range(disc.nd))
    phi = W.mms_phi(prob["pos"][:, :, 0], prob["pos"][:, :, 1])
    P.smm_sweep(h, dev(phi))
    info = h.info()
    psi_g = torch.zeros(info.n_elem * info.n_ord * info.n_dof_elem, dtype=torch.float64, device="cuda")
    P.smm_get_psi(h, psi_g)
    psi_g = psi_g.cpu().numpy().reshape(info.n_elem, info.n_ord, info.n_dof_elem).transpose(1, 0, 2)
    psi_o = disc.sweep(phi, q, inflow)
    assert rel(psi_g, psi_o) < 1e-11
    mom = torch.zeros(6 * info.n_elem * info.n_dof_elem, dtype=torch.float64, device="cuda")
    P.smm_moments(h, mom)
    mom_o = closures.nodal_moments(disc, psi_o)
    assert np.max(np.abs(mom.cpu().numpy().reshape(6, info.n_elem, -1) - mom_o)) < 1e-11 * np.max(np.abs(mom_o[0]))
    h.destroy()


@pytest.mark.parametrize("precond", [0, 1], ids=["block_jacobi", "multigrid"])
@pytest.mark.parametrize("case", CASES[:4] + [(12, 9, 2, 2, 4, 4, "mms")], ids=lambda c: "x".join(map(str, c[:5])))
def test_moment_solve_fp64(case, precond):
    import paper_2304_07386_gb300 as P
    from oracle import ipsmm
    nx, ny, m, p, sn, seed, kind = case
    prob = problem(nx, ny, m=m, p=p, sn=sn, seed=seed, kind=kind, c=0.6)
    h = make_gpu(prob, tol_cg=1e-14, precond=precond)
    disc, op, q, inflow = make_oracle(prob)
    P.smm_sweep(h, None)
    psi_o = disc.sweep(None, q, inflow)
    x_o = ipsmm.solve(op.A, op.rhs_from_psi(psi_o))
    phi = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    P.smm_moment_solve(h, phi)
    assert rel(phi.cpu().numpy(), x_o) < 1e-9


@pytest.mark.parametrize("case", [CASES[1], CASES[2]], ids=lambda c: "x".join(map(str, c[:5])))
def test_iterate_fp64_converged_flux(case):
    import paper_2304_07386_gb300 as P
    nx, ny, m, p, sn, seed, kind = case
    prob = problem(nx, ny, m=m, p=p, sn=sn, seed=seed, kind=kind, c=0.6)
    h = make_gpu(prob, tol_cg=1e-14)
    disc, op, q, inflow = make_oracle(prob)
    phi_o, k_o, _ = op.iterate(tol=1e-12)
    phi = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    rc, st = P.smm_iterate(h, phi, 1e-12, 200)
    assert rel(phi.cpu().numpy(), phi_o.ravel()) < 1e-9
    assert abs(st["outer_iterations"] - k_o) <= 1


@pytest.mark.parametrize("solver", [0, 1], ids=["lu", "cached_inverse"])
def test_fp32_refined_reaches_fp64_fixed_point(solver):
    """FP32 local solves corrected from an FP64 residual: the converged flux
    matches the FP64 oracle to the 1e-10 relative stopping tolerance (x10)."""
    import paper_2304_07386_gb300 as P
    prob = problem(4, 4, m=2, p=2, sn=8, seed=5, kind="mms", c=0.6)
    h = make_gpu(prob, precision=1, tol_cg=1e-14, sweep_solver=solver)
    disc, op, q, inflow = make_oracle(prob)
    phi_o, _, _ = op.iterate(tol=1e-13)
    phi = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    rc, st = P.smm_iterate(h, phi, 1e-10, 200, relative=True)
    assert rel(phi.cpu().numpy(), phi_o.ravel()) < 1e-9


def test_linear_solution_reproduced_on_gpu():
    import paper_2304_07386_gb300 as P
    prob = problem(4, 3, m=2, p=2, sn=4, seed=3, kind="linear", c=0.5)
    h = make_gpu(prob, tol_cg=1e-14)
    phi_ex = W.LIN_A + W.LIN_B * prob["pos"][:, :, 0] + W.LIN_C * prob["pos"][:, :, 1]
    phi = torch.zeros(phi_ex.size, dtype=torch.float64, device="cuda")
    P.smm_iterate(h, phi, 1e-13, 100)
    assert np.max(np.abs(phi.cpu().numpy() - phi_ex.ravel())) < 1e-11


def test_thick_diffusion_limit_counts_match_oracle():
    import paper_2304_07386_gb300 as P
    for eps in (1e-1, 1e-3):
        prob = problem(8, 8, m=1, p=2, sn=4, sigt=1.0 / eps, c=(1.0 / eps - eps) * eps, kind="iso")
        prob_q = np.full(prob["pos"].shape[:2], eps)
        mesh = prob["mesh"]
        opt = P.smm_default_options()
        opt.tol_cg = 1e-14
        h = P.smm_create(mesh.nodes, mesh.elem_nodes, 1, 2, 4, prob["sigma_t"], prob["sigma_s"], prob_q, options=opt)
        disc, op, _, _ = make_oracle(prob)
        from oracle.smm import SMMProblem
        op = SMMProblem(disc, prob_q)
        phi_o, k_o, _ = op.iterate(tol=1e-6)
        phi = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
        rc, st = P.smm_iterate(h, phi, 1e-6, 100)
        assert st["outer_iterations"] == k_o
        assert rel(phi.cpu().numpy(), phi_o.ravel()) < 1e-8


def test_cycle_rejected_without_lagging():
    """A bowed shared face that is inflow at some points and outflow at others
    for some S8 ordinates: with cycle lagging off it is SMM_ERR_CYCLE, with
    lagging (the default) the handle lags it."""
    import paper_2304_07386_gb300 as P
    mesh = W.structured_mesh(2, 1, m=2, domain=(0.0, 2.0, 0.0, 1.0))
    nodes = mesh.nodes.copy()
    k = np.argmin(np.hypot(nodes[:, 0] - 1.0, nodes[:, 1] - 0.5))
    nodes[k, 0] = 1.2
    opt = P.smm_default_options()
    opt.cycle_lagging = 0
    with pytest.raises(P.SMMError) as ei:
        P.smm_create(nodes, mesh.elem_nodes, 2, 1, 8, np.ones(2), np.zeros(2), np.ones((2, 4)), options=opt)
    assert ei.value.status == 5
    h = P.smm_create(nodes, mesh.elem_nodes, 2, 1, 8, np.ones(2), np.zeros(2), np.ones((2, 4)))
    assert h.info().n_lagged > 0


def test_multigrid_cuts_cg_iterations():
    """The V-cycle preconditioner needs far fewer CG iterations than
    element-block Jacobi on a fine mesh, for the same converged answer."""
    import paper_2304_07386_gb300 as P
    prob = problem(24, 24, m=1, p=2, sn=4, kind="iso", c=0.9)
    its, sols = [], []
    for precond in (0, 1):
        h = make_gpu(prob, tol_cg=1e-12, precond=precond)
        P.smm_sweep(h, None)
        phi = torch.zeros(prob["mesh"].n_elem * 9, dtype=torch.float64, device="cuda")
        its.append(P.smm_moment_solve(h, phi))
        sols.append(phi.cpu().numpy())
    assert its[1] * 8 < its[0], its
    assert rel(sols[1], sols[0]) < 1e-9


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_anderson_reaches_oracle_fixed_point(depth):
    """Anderson-accelerated SMM (the paper's outer solver) converges to the same
    fixed point as the oracle's plain iteration, in no more outer steps than
    the plain GPU iteration."""
    import paper_2304_07386_gb300 as P
    prob = problem(6, 5, m=2, p=2, sn=4, seed=2, kind="mms", c=0.95)
    disc, op, q, inflow = make_oracle(prob)
    phi_o, _, _ = op.iterate(tol=1e-13)
    its = []
    for d in (0, depth):
        h = make_gpu(prob, tol_cg=1e-14, anderson_depth=d)
        phi = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
        rc, st = P.smm_iterate(h, phi, 1e-11, 200)
        assert rel(phi.cpu().numpy(), phi_o.ravel()) < 1e-9
        its.append(st["outer_iterations"])
    assert its[1] <= its[0], its


@pytest.mark.parametrize("anderson", [0, 2])
def test_adaptive_inner_tolerance_reaches_oracle_fixed_point(anderson):
    """Moment solves to max(tol_cg, 1e-2 d_{k-1}) (d the previous step's
    relative difference) instead of tol_cg: the same fixed point as the
    oracle's, in fewer CG iterations than every solve to tol_cg; and the
    batched iterate with the same option matches the single iterate."""
    import paper_2304_07386_gb300 as P
    prob = problem(6, 5, m=2, p=2, sn=4, seed=2, kind="mms", c=0.95)
    disc, op, q, inflow = make_oracle(prob)
    phi_o, _, _ = op.iterate(tol=1e-13)
    cg = []
    for eta in (0.0, 1e-2):
        h = make_gpu(prob, tol_cg=1e-14, anderson_depth=anderson, cg_tol_adaptive=eta)
        phi = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
        rc, st = P.smm_iterate(h, phi, 1e-11, 200, relative=True)
        assert rel(phi.cpu().numpy(), phi_o.ravel()) < 1e-9
        cg.append(st["cg_total"])
        h.destroy()
    assert cg[1] < cg[0], cg
    hb = make_gpu(prob, tol_cg=1e-14, anderson_depth=anderson, cg_tol_adaptive=1e-2)
    b = P.smm.smm_batch_create([hb])
    xb = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    P.smm.smm_batch_iterate(b, [xb], 1e-11, 200, relative=True)
    assert rel(xb.cpu().numpy(), phi_o.ravel()) < 1e-9
    b.destroy()
    hb.destroy()


def test_extrapolated_cg_start_reaches_oracle_fixed_point_in_fewer_cg_iterations():
    """Each outer step's CG started from varphi_k + rho (varphi_k - varphi_{k-1})
    (the default) instead of varphi_k: the oracle's fixed point, the same
    outer steps within one, fewer CG iterations; the batched iterate too."""
    import paper_2304_07386_gb300 as P
    prob = problem(6, 5, m=2, p=2, sn=4, seed=2, kind="mms", c=0.95)
    disc, op, q, inflow = make_oracle(prob)
    phi_o, _, _ = op.iterate(tol=1e-13)
    res = []
    for ex in (0, 1):
        h = make_gpu(prob, tol_cg=1e-14, cg_guess_extrapolate=ex)
        phi = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
        rc, st = P.smm_iterate(h, phi, 1e-11, 200, relative=True)
        assert rel(phi.cpu().numpy(), phi_o.ravel()) < 1e-9
        res.append((st["outer_iterations"], st["cg_total"]))
        h.destroy()
    assert abs(res[1][0] - res[0][0]) <= 1 and res[1][1] < res[0][1], res
    hb = make_gpu(prob, tol_cg=1e-14, cg_guess_extrapolate=1)
    b = P.smm.smm_batch_create([hb])
    xb = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
    stats = P.smm.smm_batch_iterate(b, [xb], 1e-11, 200, relative=True)
    assert rel(xb.cpu().numpy(), phi_o.ravel()) < 1e-9 and stats[0]["cg_total"] < res[0][1]
    b.destroy()
    hb.destroy()


BATCH = [
    # (nx, ny, m, p, sn, seed)
    (4, 4, 1, 1, 4, None),
    (6, 5, 2, 2, 8, 3),
    (3, 3, 3, 3, 4, 7),
    (5, 4, 2, 4, 6, 2),
    (7, 3, 1, 2, 12, None),
]


@pytest.mark.parametrize("orders", ["p1_to_4", "p1_to_3"])
@pytest.mark.parametrize("precision,solver", [(0, 1), (0, 0), (1, 1)], ids=["fp64_cached", "fp64_lu", "fp32_cached"])
def test_batched_sweep_matches_single_problems(precision, solver, orders):
    """Uneven problems (mesh size, p, S_N, geometry order) in one launch give
    the same angular fluxes as their single sweeps (a batch without p = 4
    runs the kernel compiled without that order's path)."""
    import paper_2304_07386_gb300 as P
    cases = [c for c in BATCH if orders == "p1_to_4" or c[3] <= 3]
    probs = [problem(nx, ny, m=m, p=p, sn=sn, seed=seed, kind="mms", c=0.6) for (nx, ny, m, p, sn, seed) in cases]
    phis = [dev(W.mms_phi(pr["pos"][:, :, 0], pr["pos"][:, :, 1]).ravel()) for pr in probs]
    singles, hs = [], []
    for pr, ph in zip(probs, phis):
        h = make_gpu(pr, precision=precision, sweep_solver=solver)
        P.smm_sweep(h, ph)
        info = h.info()
        buf = torch.zeros(info.n_elem * info.n_ord * info.n_dof_elem, dtype=torch.float64, device="cuda")
        P.smm_get_psi(h, buf)
        singles.append(buf.cpu().numpy())
        hs.append(make_gpu(pr, precision=precision, sweep_solver=solver))
    b = P.smm.smm_batch_create(hs)
    sched = b.schedule()
    assert sched["n_tasks"] == sum(h.info().n_elem * h.info().n_ord for h in hs)
    # (the refined FP32 sweep corrects the flux left by the tuning sweeps; both
    # it and the single sweep approximate the same FP64 result to FP32 accuracy)
    P.smm.smm_batch_sweep(b, phis)
    for h, ref in zip(hs, singles):
        info = h.info()
        buf = torch.zeros(info.n_elem * info.n_ord * info.n_dof_elem, dtype=torch.float64, device="cuda")
        P.smm_get_psi(h, buf)
        tol = 1e-13 if precision == 0 else 1e-6
        assert rel(buf.cpu().numpy(), ref) < tol


def test_batched_iterate_matches_oracle():
    import paper_2304_07386_gb300 as P
    probs = [problem(nx, ny, m=m, p=p, sn=sn, seed=seed, kind="mms", c=0.6) for (nx, ny, m, p, sn, seed) in BATCH[:3]]
    hs = [make_gpu(pr, tol_cg=1e-14) for pr in probs]
    b = P.smm.smm_batch_create(hs)
    phis = [torch.zeros(h.info().n_elem * h.info().n_dof_elem, dtype=torch.float64, device="cuda") for h in hs]
    stats = P.smm.smm_batch_iterate(b, phis, 1e-12, 100)
    for pr, ph, st in zip(probs, phis, stats):
        disc, op, q, inflow = make_oracle(pr)
        ref, k, _ = op.iterate(tol=1e-12)
        assert rel(ph.cpu().numpy(), ref.ravel()) < 1e-9
        assert abs(st["outer_iterations"] - k) <= 1


def test_moment_solve_from_smooth_moments_on_a_fine_curved_mesh():
    """The right-hand side's pair products where they cancel most: smooth T
    (K and the face gradient operators annihilate constants, so K T is small
    next to its terms) on a curved 32x32 p = 4 mesh, with a seeded beta on the
    boundary.  The moment solve from these moments matches the oracle's solve
    of the same IP-SMM system (Eq. ipsmm)."""
    import paper_2304_07386_gb300 as P
    from oracle import closures, ipsmm
    prob = problem(32, 32, m=3, p=4, sn=4, seed=5, kind="iso", c=0.6)
    h = make_gpu(prob, tol_cg=1e-13)
    try:
        disc = oracle_disc(prob)
        q, inflow = sources(prob, disc.omega)
        x, y = prob["pos"][:, :, 0], prob["pos"][:, :, 1]
        T = np.stack([np.sin(2 * x + 1) * np.cos(1.5 * y - 1), 0.5 * np.cos(2 * x - y), 0.8 * np.sin(x + 2 * y) + 0.3])
        jin = closures.j_in(disc, inflow)
        beta = np.random.default_rng(11).uniform(-0.1, 0.1, jin.shape)
        mom = np.concatenate([np.ones((1,) + x.shape), np.zeros((2,) + x.shape), T])
        P.smm_set_moments(h, dev(mom), dev(beta))
        phi = torch.zeros(disc.ne * disc.n, dtype=torch.float64, device="cuda")
        its = P.smm_moment_solve(h, phi)
        assert 0 < its < 200
        b = ipsmm.assemble_rhs(disc, closures.source_moments(disc, q), T, jin, beta)
        x_o = ipsmm.solve(ipsmm.assemble_lhs(disc), b)
        assert rel(phi.cpu().numpy(), x_o) < 1e-9, rel(phi.cpu().numpy(), x_o)
    finally:
        h.destroy()


def test_multigrid_with_the_vertex_level_on_grid_kernels():
    """A vertex level of more than 32,768 rows (here 201 x 201) runs its
    stages as grid kernels around the cluster launch; the V-cycle must still
    cut the CG iterations far below element-block Jacobi's and give the same
    solution of the moment system."""
    import paper_2304_07386_gb300 as P
    prob = problem(200, 200, m=1, p=1, sn=4, kind="iso", c=0.9)
    its, sols = [], []
    for precond in (0, 1):
        h = make_gpu(prob, tol_cg=1e-12, precond=precond)
        P.smm_sweep(h, None)
        phi = torch.zeros(prob["mesh"].n_elem * 4, dtype=torch.float64, device="cuda")
        its.append(P.smm_moment_solve(h, phi))
        sols.append(phi.cpu().numpy())
        h.destroy()
    assert its[1] < 40 and its[1] * 8 < its[0], its
    assert rel(sols[1], sols[0]) < 1e-9

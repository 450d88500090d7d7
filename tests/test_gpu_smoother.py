"""Level-0 smoother of the IP-SMM multigrid preconditioner.

The smoother changes only the preconditioner inside flexible CG, so every
choice must solve the same moment system: damped element-block Jacobi and the
Chebyshev polynomial smoother with 1..4 steps (which exercises the two-buffer
rotation of the three-term recurrence) reach the same solution within the CG
tolerance, and that solution satisfies the oracle's IP-SMM system (Eq. ipsmm)
to the same tolerance.  On a 32x32 mesh the degree-3 Chebyshev smoother takes
fewer CG iterations than two Jacobi steps.  The CG loop run as one device-side
graph and as host-checked chunks of the one-iteration graph executes the same
kernels: the same solution bit for bit and the same iteration count.
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


def solve(prob, smoother, steps, phi, device_loop=1):
    """Sweep from phi, then the moment solve; returns (solution, CG iterations)."""
    import paper_2304_07386_gb300 as P
    om, _ = P.smm_quadrature(prob["sn"])
    q, inflow = sources(prob, om)
    opt = P.smm_default_options()
    opt.mg_smoother = smoother
    opt.mg_smooth_steps = steps
    opt.cg_device_loop = device_loop
    opt.tol_cg = 1e-13
    mesh = prob["mesh"]
    h = P.smm_create(mesh.nodes, mesh.elem_nodes, mesh.m, prob["p"], prob["sn"], prob["sigma_t"], prob["sigma_s"],
                     q, inflow=inflow, options=opt)
    try:
        x = torch.as_tensor(np.ascontiguousarray(phi.ravel()), device="cuda")
        P.smm_sweep(h, x)
        its = P.smm_moment_solve(h, x)
        return x.cpu().numpy(), its
    finally:
        h.destroy()


def test_smoothers_solve_the_same_system():
    import scipy.sparse.linalg as spla
    import paper_2304_07386_gb300 as P
    from oracle import closures, ipsmm
    import smm_workloads as W
    prob = problem(9, 7, m=2, p=3, sn=4, seed=3, kind="mms", c=0.8)
    phi = W.mms_phi(prob["pos"][:, :, 0], prob["pos"][:, :, 1])
    # the oracle's solution of the same moment system (closures from the oracle's sweep of phi)
    disc = oracle_disc(prob)
    q, inflow = sources(prob, disc.omega)
    psi = disc.sweep(phi, q, inflow)
    Q = closures.source_moments(disc, q)
    mom = closures.nodal_moments(disc, psi)
    b = ipsmm.assemble_rhs(disc, Q, mom[3:], closures.j_in(disc, inflow), closures.beta(disc, psi))
    x_o = spla.spsolve(ipsmm.assemble_lhs(disc).tocsc(), b)
    scale = np.max(np.abs(x_o))
    for smoother, steps in ((P.smm.SMM_SMOOTHER_JACOBI, 2), (P.smm.SMM_SMOOTHER_CHEBYSHEV, 1),
                            (P.smm.SMM_SMOOTHER_CHEBYSHEV, 2), (P.smm.SMM_SMOOTHER_CHEBYSHEV, 3),
                            (P.smm.SMM_SMOOTHER_CHEBYSHEV, 4), (P.smm.SMM_SMOOTHER_JACOBI, 4)):
        x, its = solve(prob, smoother, steps, phi)
        assert 0 < its < 200, (smoother, steps, its)
        err = np.max(np.abs(x - x_o)) / scale
        assert err < 1e-9, (smoother, steps, err)


def test_chebyshev_needs_fewer_iterations():
    import paper_2304_07386_gb300 as P
    prob = problem(32, m=1, p=3, sn=4, kind="iso", c=0.9)
    phi = np.ones((prob["mesh"].n_elem, 16))
    _, its_j = solve(prob, P.smm.SMM_SMOOTHER_JACOBI, 2, phi)
    _, its_c = solve(prob, P.smm.SMM_SMOOTHER_CHEBYSHEV, 3, phi)
    assert its_c < its_j, (its_c, its_j)


def test_device_loop_matches_host_loop():
    import paper_2304_07386_gb300 as P
    prob = problem(20, 13, m=2, p=4, sn=4, seed=9, kind="mms", c=0.9)
    phi = np.ones((prob["mesh"].n_elem, 25))
    x_dev, its_dev = solve(prob, P.smm.SMM_SMOOTHER_CHEBYSHEV, 3, phi, device_loop=1)
    x_host, its_host = solve(prob, P.smm.SMM_SMOOTHER_CHEBYSHEV, 3, phi, device_loop=0)
    assert its_dev == its_host, (its_dev, its_host)
    assert np.array_equal(x_dev, x_host)

"""The C ABI's boundary calls on the GPU: the transport scalar flux returned by
a sweep, the fixed-point iteration on a host array, the checkpoint calls, the
bounded dependency wait running out, and the guess check with Anderson
acceleration.

Tolerances as in test_gpu_parity.py: 1e-11 relative (max norm over the array,
relative to its max magnitude) for a sweep's results, 1e-9 for converged
scalar fluxes; restored and host-array runs are compared bit for bit with the
run they must reproduce.
"""
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


def make_gpu(prob, **kw):
    import paper_2304_07386_gb300 as P
    om, _ = P.smm_quadrature(prob["sn"])
    q, inflow = sources(prob, om)
    opt = P.smm_default_options()
    for k, v in kw.items():
        setattr(opt, k, v)
    mesh = prob["mesh"]
    return P.smm_create(mesh.nodes, mesh.elem_nodes, mesh.m, prob["p"], prob["sn"], prob["sigma_t"],
                        prob["sigma_s"], q, inflow=inflow, options=opt)


def make_oracle(prob):
    from oracle.smm import SMMProblem
    disc = oracle_disc(prob)
    q, inflow = sources(prob, disc.omega)
    return disc, SMMProblem(disc, q, inflow), q, inflow


def zeros(n):
    return torch.zeros(n, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("solver", [0, 1], ids=["lu", "cached_inverse"])
def test_sweep_returns_the_transport_scalar_flux(solver):
    """smm_sweep's optional output is phi_T = sum_d w_d psi_d of that sweep
    (Eq. correction_tensor_disc's zeroth moment), on the host or the device."""
    import paper_2304_07386_gb300 as P
    from oracle import closures
    prob = problem(5, 3, m=2, p=2, sn=8, seed=3, kind="mms", c=0.6)
    h = make_gpu(prob, sweep_solver=solver)
    disc, op, q, inflow = make_oracle(prob)
    phi = W.mms_phi(prob["pos"][:, :, 0], prob["pos"][:, :, 1])
    n_phi = disc.ne * disc.n
    out_dev = zeros(n_phi)
    out_host = np.zeros(n_phi)
    P.smm_sweep(h, torch.as_tensor(phi.ravel(), device="cuda"), out_dev)
    P.smm_sweep(h, torch.as_tensor(phi.ravel(), device="cuda"), out_host)
    ref = closures.nodal_moments(disc, disc.sweep(phi, q, inflow))[0]
    assert rel(out_dev.cpu().numpy(), ref.ravel()) < 1e-11
    assert np.array_equal(out_host, out_dev.cpu().numpy())
    mom = zeros(6 * n_phi)
    P.smm_moments(h, mom)
    assert np.array_equal(mom[:n_phi].cpu().numpy(), out_host)


def test_iterate_on_a_host_array_equals_the_device_run():
    """smm_iterate accepts the iterate in host memory (copied in once, out
    once): the same steps, bit for bit, as on a device array, and the oracle's
    fixed point."""
    import paper_2304_07386_gb300 as P
    prob = problem(4, 4, m=2, p=2, sn=8, seed=5, kind="mms", c=0.6)
    disc, op, q, inflow = make_oracle(prob)
    phi_o, _, _ = op.iterate(tol=1e-12)
    h = make_gpu(prob, tol_cg=1e-14)
    x_dev = zeros(disc.ne * disc.n)
    rc_d, st_d = P.smm_iterate(h, x_dev, 1e-12, 200)
    h2 = make_gpu(prob, tol_cg=1e-14)
    x_host = np.zeros(disc.ne * disc.n)
    rc_h, st_h = P.smm_iterate(h2, x_host, 1e-12, 200)
    assert rc_d == rc_h == 0
    assert st_h["outer_iterations"] == st_d["outer_iterations"]
    assert np.array_equal(x_host, x_dev.cpu().numpy())
    assert rel(x_host, phi_o.ravel()) < 1e-9
    # NOT_CONVERGED still hands the last iterate back to the host array
    x3 = np.zeros(disc.ne * disc.n)
    rc, st = P.smm_iterate(h2, x3, 1e-30, 2, raise_on_error=False)
    assert rc == 7 and st["outer_iterations"] == 2 and np.max(np.abs(x3)) > 0


@pytest.mark.parametrize("mode", ["fp32_refined", "anderson2", "tiles", "extrapolate"])
def test_restored_state_reproduces_the_next_iterates_bit_for_bit(mode):
    """A state saved after three outer steps and restored into a fresh handle
    built from the same data gives, bit for bit, the next two iterates of the
    saved handle -- for each mode whose next step reads the state: the
    FP32-refined sweep (it corrects the stored angular flux), Anderson depth 2
    with resume_history (the history ring and its length), the block Jacobi
    sweep (it lags the stored flux across tile borders), the extrapolated CG
    start with resume_history (the previous input and the last two
    differences).  Without the restore the fresh handle's steps differ, so
    the state is what carries them."""
    import paper_2304_07386_gb300 as P
    prob = problem(6, 5, m=2, p=2, sn=4, seed=2, kind="mms", c=0.95)
    kw = dict(tol_cg=1e-14)
    if mode == "fp32_refined":
        kw["sweep_precision"] = 1
    elif mode == "anderson2":
        kw.update(anderson_depth=2, resume_history=1)
    elif mode == "extrapolate":
        kw.update(cg_guess_extrapolate=1, resume_history=1)
    else:
        kw["sweep_tiles"] = 2
    n_phi = prob["mesh"].n_elem * 9
    a = make_gpu(prob, **kw)
    x = zeros(n_phi)
    rc, _ = P.smm_iterate(a, x, 1e-30, 3, raise_on_error=False)
    assert rc == 7
    x3 = x.clone()
    host_state = P.smm_get_state(a)
    dev_state = torch.zeros(P.smm_state_size(a), dtype=torch.uint8, device="cuda")
    P.smm_get_state(a, dev_state)
    assert np.array_equal(dev_state.cpu().numpy(), host_state)
    P.smm_iterate(a, x, 1e-30, 2, raise_on_error=False)
    x5 = x.cpu().numpy()
    for buf in (host_state, dev_state):
        b = make_gpu(prob, **kw)
        P.smm_set_state(b, buf)
        y = x3.clone()
        P.smm_iterate(b, y, 1e-30, 2, raise_on_error=False)
        assert np.array_equal(y.cpu().numpy(), x5)
    c = make_gpu(prob, **kw)
    y = x3.clone()
    P.smm_iterate(c, y, 1e-30, 2, raise_on_error=False)
    assert not np.array_equal(y.cpu().numpy(), x5)
    if mode in ("anderson2", "extrapolate"):
        # with resume_history a run split 3 + 2 takes the steps of one 5-step run
        d = make_gpu(prob, **kw)
        z = zeros(n_phi)
        P.smm_iterate(d, z, 1e-30, 5, raise_on_error=False)
        assert np.array_equal(z.cpu().numpy(), x5)


def test_state_of_another_shape_is_rejected():
    import paper_2304_07386_gb300 as P
    a = make_gpu(problem(4, 4, m=1, p=2, sn=4, kind="iso"))
    b = make_gpu(problem(4, 5, m=1, p=2, sn=4, kind="iso"))
    with pytest.raises(P.SMMError) as ei:
        P.smm_set_state(b, P.smm_get_state(a))
    assert ei.value.status == 1
    with pytest.raises(P.SMMError) as ei:
        P.smm_get_state(a, np.zeros(16, dtype=np.uint8))
    assert ei.value.status == 1


@pytest.mark.parametrize("solver", [0, 1], ids=["lu", "cached_inverse"])
def test_expired_dependency_wait_returns_timeout_and_the_handle_recovers(solver):
    """The bounded dependency wait run out on the device: with a 1 ns bound
    every wait that does not find its upwind flag within its first polls gives
    up, and on a 64 x 64 mesh (127 upwind levels per quadrant) some must wait.
    The call returns SMM_ERR_DEVICE_TIMEOUT (8) instead of hanging, and on the
    same handle, with the bound restored, the next sweep matches the oracle:
    the aborted sweep's flags belong to an old epoch and are ignored."""
    import paper_2304_07386_gb300 as P
    prob = problem(64, 64, m=1, p=1, sn=8, kind="iso", c=0.6)
    h = make_gpu(prob, sweep_solver=solver)
    P.smm_set_spin_timeout(h, 1e-9)
    with pytest.raises(P.SMMError) as ei:
        P.smm_sweep(h, None)
    assert ei.value.status == 8
    x = zeros(prob["mesh"].n_elem * 4)
    rc, _ = P.smm_iterate(h, x, 1e-8, 3, raise_on_error=False)
    assert rc == 8
    P.smm_set_spin_timeout(h, 2.0)
    disc, op, q, inflow = make_oracle(prob)
    phi = np.random.default_rng(4).uniform(0.5, 1.5, (disc.ne, disc.n))
    for _ in range(2):
        P.smm_sweep(h, torch.as_tensor(phi.ravel(), device="cuda"))
        info = h.info()
        psi = zeros(info.n_elem * info.n_ord * info.n_dof_elem)
        P.smm_get_psi(h, psi)
        got = psi.cpu().numpy().reshape(info.n_elem, info.n_ord, info.n_dof_elem).transpose(1, 0, 2)
        assert rel(got, disc.sweep(phi, q, inflow)) < 1e-11


def test_rejected_guess_with_anderson_reaches_the_oracle_fixed_point():
    """guess_check with Anderson depth 2: a guess far off (1e3 everywhere) is
    rejected after the first step, the iteration restarts from zero with an
    empty history (no step from the rejected guess is mixed in), and it reaches
    the oracle's fixed point in the zero guess's outer steps plus the rejected
    one."""
    import paper_2304_07386_gb300 as P
    prob = problem(6, 5, m=2, p=2, sn=4, seed=2, kind="mms", c=0.95)
    disc, op, q, inflow = make_oracle(prob)
    phi_o, _, _ = op.iterate(tol=1e-13)
    h0 = make_gpu(prob, tol_cg=1e-14, anderson_depth=2)
    x0 = zeros(disc.ne * disc.n)
    _, st0 = P.smm_iterate(h0, x0, 1e-11, 200)
    h = make_gpu(prob, tol_cg=1e-14, anderson_depth=2, guess_check=1)
    # run once first so that the history ring holds values from another solve
    y = zeros(disc.ne * disc.n)
    P.smm_iterate(h, y, 1e-11, 200)
    x = torch.full((disc.ne * disc.n,), 1e3, dtype=torch.float64, device="cuda")
    rc, st = P.smm_iterate(h, x, 1e-11, 200)
    assert rc == 0 and st["guess_rejected"] == 1
    assert rel(x.cpu().numpy(), phi_o.ravel()) < 1e-9
    assert st["outer_iterations"] == st0["outer_iterations"] + 1
    assert np.array_equal(x.cpu().numpy(), x0.cpu().numpy())

"""Learned initial guess: the library's BF16 network kernels against the
NumPy oracle (forward and gradients), and a held-out test of what a network
trained on the method's own solutions gains over the zero guess."""
import numpy as np
import pytest

import smm_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_07386_gb300 import build as B
    B.build()


@pytest.mark.parametrize("seed", [0, 1, 3])
def test_network_reproduces_the_oracle_bit_for_bit_on_exact_cases(seed):
    """Forward output, loss and every parameter gradient, element by element
    and layer by layer (tests/cnn_exact.py: cases on which every FP32 sum of
    the library's arithmetic is exact in any order, certified from the
    oracle's values), must equal the oracle's exactly."""
    import paper_2304_07386_gb300 as P
    from oracle import cnn
    from tests import cnn_exact
    params, x, t, n_out = cnn_exact.case(seed)
    cnn_exact.certify(params, x, t, n_out)
    B, _, H, Wd = x.shape
    net = P.smm.Guess(H, Wd, n_out, B, seed=3)
    assert net.n_params == params.size
    net.set_params(params.astype(np.float32))
    xd = torch.as_tensor(x.astype(np.float32), device="cuda")
    td = torch.as_tensor(t.astype(np.float32), device="cuda")
    y = torch.zeros((B, n_out, H, Wd), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    loss_o, g_o, _, it = cnn.loss_and_grad(params, x, t, n_out, bf=True, intermediates=True)
    assert np.array_equal(y.cpu().numpy().astype(np.float64), it["y"])
    loss, g = net.gradients(xd, td)
    assert loss == loss_o
    bad = [name for name, sl in cnn_exact.blocks(n_out) if not np.array_equal(g[sl].astype(np.float64), g_o[sl])]
    assert not bad, bad


def test_network_forward_and_gradients_match_oracle_elementwise():
    """General inputs (weights ~ N(0, 0.2^2), normal inputs and targets): the
    library's FP32 sums round differently from the oracle's FP64 ones, by about
    2^-24 K of a sum of K terms, and where such a difference crosses a BF16
    rounding boundary a stored activation or stored gradient moves by one
    BF16 unit (at most 2^-7 of its value), moving what follows it by about
    that fraction.  So
    every output value is checked against 1e-2 of its channel's largest
    magnitude, and every gradient entry against 1e-2 of its layer block's
    (weights and bias of each layer separately); the loss to 1e-3."""
    import paper_2304_07386_gb300 as P
    from oracle import cnn
    from tests import cnn_exact
    H, Wd, n_out, B = 8, 6, 4, 2
    net = P.smm.Guess(H, Wd, n_out, B, seed=3)
    assert net.n_params == cnn.num_params(n_out)
    for seed in (1, 2):
        rng = np.random.default_rng(seed)
        params = (rng.standard_normal(net.n_params) * 0.2).astype(np.float32)
        net.set_params(params)
        x = rng.standard_normal((B, 3, H, Wd)).astype(np.float32)
        t = rng.standard_normal((B, n_out, H, Wd)).astype(np.float32)
        xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
        y = torch.zeros((B, n_out, H, Wd), dtype=torch.float32, device="cuda")
        net.forward(xd, y)
        y_ref, _ = cnn.forward(params.astype(np.float64), x.astype(np.float64), n_out, bf=True)
        scale = np.max(np.abs(y_ref), axis=(0, 2, 3), keepdims=True)
        assert np.all(np.abs(y.cpu().numpy() - y_ref) <= 1e-2 * scale)
        loss, g = net.gradients(xd, td)
        loss_ref, g_ref = cnn.loss_and_grad(params.astype(np.float64), x.astype(np.float64), t.astype(np.float64),
                                            n_out, bf=True)
        assert abs(loss - loss_ref) < 1e-3 * loss_ref
        for name, sl in cnn_exact.blocks(n_out):
            assert np.all(np.abs(g[sl] - g_ref[sl]) <= 1e-2 * np.max(np.abs(g_ref[sl]))), name


def test_two_million_parameter_network_matches_oracle_elementwise():
    """The network at the widths of the two-million-parameter configuration
    (c1 = 64, c2 = 384: 1,846,473 parameters), He-initialized by the library
    with non-zero biases, on a 12 x 10 grid: forward output and every gradient
    entry against the oracle (bf=True) as in the test above.  Its reductions
    have up to 3,456 terms (9 taps x 384 channels) per output and span several
    64 x 64 tiles of the tensor-core passes in both the pixel and channel
    directions."""
    import paper_2304_07386_gb300 as P
    from oracle import cnn
    H, Wd, n_out, B, c1, c2 = 12, 10, 9, 3, 64, 384
    net = P.smm.Guess(H, Wd, n_out, B, seed=5, c1=c1, c2=c2)
    assert net.n_params == cnn.num_params(n_out, c1, c2) == 1_846_473
    rng = np.random.default_rng(7)
    params = net.get_params()
    off = 0
    for ci, co, k, _ in cnn.layer_specs(n_out, c1, c2):
        off += co * ci * k * k
        params[off:off + co] = rng.standard_normal(co).astype(np.float32) * 0.1
        off += co
    net.set_params(params)
    x = rng.standard_normal((B, 3, H, Wd)).astype(np.float32)
    t = rng.standard_normal((B, n_out, H, Wd)).astype(np.float32)
    xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
    y = torch.zeros((B, n_out, H, Wd), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    p64 = params.astype(np.float64)
    y_ref, _ = cnn.forward(p64, x.astype(np.float64), n_out, bf=True, c1=c1, c2=c2)
    scale = np.max(np.abs(y_ref), axis=(0, 2, 3), keepdims=True)
    assert np.all(np.abs(y.cpu().numpy() - y_ref) <= 1e-2 * scale)
    loss, g = net.gradients(xd, td)
    loss_ref, g_ref = cnn.loss_and_grad(p64, x.astype(np.float64), t.astype(np.float64), n_out, bf=True, c1=c1, c2=c2)
    assert abs(loss - loss_ref) < 1e-3 * loss_ref
    off = 0
    for i, (ci, co, k, _) in enumerate(cnn.layer_specs(n_out, c1, c2)):
        for name, n in (("weights", co * ci * k * k), ("bias", co)):
            sl = slice(off, off + n)
            off += n
            assert np.all(np.abs(g[sl] - g_ref[sl]) <= 1e-2 * np.max(np.abs(g_ref[sl]))), (i, name)


def test_two_million_parameter_network_at_full_size_on_sampled_pixels():
    """The forward pass at the full-size configuration (128 x 128, batch 16,
    widths 64 / 384: the launch shapes the bench trains with) against the
    oracle on crops.  An output pixel depends only on inputs within 7 pixels
    (3x3 layers, the stride-2 layer and the nearest up-sampling; crops start at
    even offsets so the half-resolution grid lines up), so the oracle's forward
    pass on a 48 x 48 crop gives the exact full-size output on every pixel at
    least 8 pixels from a crop edge that lies inside the image
    (test_oracle_cnn.py checks this on the oracle alone: exact from a margin
    of 6, not at 5).  Crops at two
    corners and the centre of the first and last sample; each value within 1e-2
    of its channel's largest magnitude, as in the small-grid test."""
    import paper_2304_07386_gb300 as P
    from oracle import cnn
    H = Wd = 128
    n_out, B, c1, c2, S, margin = 9, 16, 64, 384, 48, 8
    net = P.smm.Guess(H, Wd, n_out, B, seed=11, c1=c1, c2=c2)
    rng = np.random.default_rng(13)
    params = net.get_params()
    off = 0
    for ci, co, k, _ in cnn.layer_specs(n_out, c1, c2):
        off += co * ci * k * k
        params[off:off + co] = rng.standard_normal(co).astype(np.float32) * 0.1
        off += co
    net.set_params(params)
    x = rng.standard_normal((B, 3, H, Wd)).astype(np.float32)
    y = torch.zeros((B, n_out, H, Wd), dtype=torch.float32, device="cuda")
    net.forward(torch.as_tensor(x, device="cuda"), y)
    y = y.cpu().numpy()
    p64 = params.astype(np.float64)
    checked = 0
    for b in (0, B - 1):
        for oy, ox in ((0, 0), (40, 40), (H - S, Wd - S)):
            crop = x[b:b + 1, :, oy:oy + S, ox:ox + S].astype(np.float64)
            ref, _ = cnn.forward(p64, crop, n_out, bf=True, c1=c1, c2=c2)
            y0 = 0 if oy == 0 else margin
            y1 = S if oy + S == H else S - margin
            x0 = 0 if ox == 0 else margin
            x1 = S if ox + S == Wd else S - margin
            r = ref[0, :, y0:y1, x0:x1]
            g = y[b, :, oy + y0:oy + y1, ox + x0:ox + x1]
            scale = np.max(np.abs(r), axis=(1, 2), keepdims=True)
            assert np.all(np.abs(g - r) <= 1e-2 * scale), (b, oy, ox, float(np.max(np.abs(g - r) / scale)))
            checked += r.size
    assert checked > 6 * n_out * 32 * 32


def _solve(P, nx, seed, phi0=None, check=False, p=2, sn=4, tol=1e-8):
    mesh, st, ss, qe = W.learned_guess_problem(nx, seed)
    n = (p + 1) ** 2
    opt = P.smm_default_options()
    opt.tol_cg = 1e-12
    opt.guess_check = int(check)
    h = P.smm_create(mesh.nodes, mesh.elem_nodes, 1, p, sn, st, ss, np.repeat(qe[:, None], n, axis=1), options=opt)
    phi = torch.zeros(nx * nx * n, dtype=torch.float64, device="cuda")
    if phi0 is not None:
        phi.copy_(torch.as_tensor(phi0, device="cuda"))
    rc, stats = P.smm_iterate(h, phi, tol, 200, relative=True)
    mom = torch.zeros(6 * nx * nx * n, dtype=torch.float64, device="cuda")
    P.smm_moments(h, mom)
    h.destroy()
    return phi.cpu().numpy(), mom.cpu().numpy(), stats, (st, ss, qe)


def test_trained_guess_saves_outer_iterations_on_held_out_problems():
    import paper_2304_07386_gb300 as P
    from paper_2304_07386_gb300 import guess as G
    nx, p, n = 16, 2, 9
    X, Y = [], []
    for seed in range(96):
        phi, mom, _, (st, ss, qe) = _solve(P, nx, seed, tol=1e-10)
        X.append(G.features(st, ss, qe, nx))
        Y.append(G.targets(phi, nx, n))
    X, Y = np.stack(X), np.stack(Y)
    xn, yn = G.Normalizer(X), G.Normalizer(Y)
    net = P.smm.Guess(nx, nx, n, 16, seed=0)
    Xd = torch.as_tensor(xn.fwd(X), device="cuda")
    Yd = torch.as_tensor(yn.fwd(Y), device="cuda")
    losses = G.train(net, Xd, Yd, steps=800, batch=16, lr=3e-3)
    assert np.mean(losses[-50:]) < 0.25 * np.mean(losses[:10])
    base, learned, rejected = [], [], 0
    for seed in range(1000, 1008):
        _, _, s0, (st, ss, qe) = _solve(P, nx, seed)
        xg = torch.as_tensor(xn.fwd(G.features(st, ss, qe, nx)[None]), device="cuda")
        phi0 = G.predict_phi(net, xg, yn, nx, n)
        phi1, _, s1, _ = _solve(P, nx, seed, phi0=phi0, check=True)
        ref, _, _, _ = _solve(P, nx, seed, tol=1e-11)
        assert np.max(np.abs(phi1 - ref)) < 1e-6 * np.max(np.abs(ref))
        base.append(s0["outer_iterations"])
        learned.append(s1["outer_iterations"])
        rejected += s1["guess_rejected"]
    print("zero guess", base, "learned", learned, "rejected", rejected)
    assert np.mean(learned) < np.mean(base)

"""Pins for the NumPy reference of the learned-guess network: gradients
against central finite differences (FP64), BF16 rounding, shapes."""
import numpy as np
import pytest

from oracle import cnn


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 0.0])
    r = cnn.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0  # halfway rounds to even
    assert r[2] == 1.0 + 2 ** -7
    assert abs(r[3] + 3.140625) < 1e-12 and r[4] == 0.0


@pytest.mark.parametrize("c1,c2", [(cnn.C1, cnn.C2), (16, 48)])
def test_gradients_match_finite_differences(c1, c2):
    rng = np.random.default_rng(0)
    n_out = 4
    npar = cnn.num_params(n_out, c1, c2)
    p = rng.standard_normal(npar) * 0.2
    x = rng.standard_normal((2, 3, 6, 4))
    t = rng.standard_normal((2, n_out, 6, 4))
    loss, g = cnn.loss_and_grad(p, x, t, n_out, c1=c1, c2=c2)
    y, _ = cnn.forward(p, x, n_out, c1=c1, c2=c2)
    assert y.shape == (2, n_out, 6, 4)
    idx = rng.choice(npar, 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(npar)
        e[i] = h
        fd = (cnn.loss_and_grad(p + e, x, t, n_out, c1=c1, c2=c2)[0] -
              cnn.loss_and_grad(p - e, x, t, n_out, c1=c1, c2=c2)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_widths_set_the_parameter_count():
    """Two million parameters at c1 = 64, c2 = 384 (9 (3 c1 + c1 c2 + c2^2 + c2 c1 + 2 c1^2) weights of the 3x3
    layers, c1 n_out of the head, and one bias per output channel)."""
    n_out, c1, c2 = 9, 64, 384
    w = 9 * (3 * c1 + c1 * c2 + c2 * c2 + c2 * c1 + 2 * c1 * c1) + c1 * n_out
    b = c1 + c2 + c2 + c1 + c1 + n_out
    assert cnn.num_params(n_out, c1, c2) == w + b == 1_846_473


def test_outputs_depend_only_on_nearby_inputs():
    """The receptive field behind the full-size GPU network test's crops: the
    forward pass on a crop at an even offset equals the full image's on every
    pixel at least 6 pixels from an interior crop edge, and not at 5 (so the
    test's margin of 8 is a real bound, not a coincidence of the data)."""
    rng = np.random.default_rng(0)
    n_out, c1, c2, S = 4, 16, 32, 48
    p = rng.standard_normal(cnn.num_params(n_out, c1, c2)) * 0.3
    x = rng.standard_normal((1, 3, 64, 64))
    full, _ = cnn.forward(p, x, n_out, c1=c1, c2=c2)
    for oy, ox in ((0, 0), (8, 8), (16, 16)):
        crop, _ = cnn.forward(p, x[:, :, oy:oy + S, ox:ox + S], n_out, c1=c1, c2=c2)
        for m, exact in ((8, True), (6, True), (5, False)):
            y0, x0 = (0 if oy == 0 else m), (0 if ox == 0 else m)
            y1, x1 = (S if oy + S == 64 else S - m), (S if ox + S == 64 else S - m)
            same = np.array_equal(crop[0, :, y0:y1, x0:x1], full[0, :, oy + y0:oy + y1, ox + x0:ox + x1])
            assert same == exact, (oy, ox, m)

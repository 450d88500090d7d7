"""Pins for the NumPy reference of the learned-guess network: gradients
against central finite differences (FP64), BF16 rounding, shapes."""
import numpy as np

from oracle import cnn


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 0.0])
    r = cnn.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0  # halfway rounds to even
    assert r[2] == 1.0 + 2 ** -7
    assert abs(r[3] + 3.140625) < 1e-12 and r[4] == 0.0


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    n_out = 4
    npar = cnn.num_params(n_out)
    p = rng.standard_normal(npar) * 0.2
    x = rng.standard_normal((2, 3, 6, 4))
    t = rng.standard_normal((2, n_out, 6, 4))
    loss, g = cnn.loss_and_grad(p, x, t, n_out)
    y, _ = cnn.forward(p, x, n_out)
    assert y.shape == (2, n_out, 6, 4)
    idx = rng.choice(npar, 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(npar)
        e[i] = h
        fd = (cnn.loss_and_grad(p + e, x, t, n_out)[0] - cnn.loss_and_grad(p - e, x, t, n_out)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])

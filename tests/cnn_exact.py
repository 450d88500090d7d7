"""Inputs on which the learned-guess network can be checked bit for bit (test
infrastructure).

The library evaluates the network of oracle/cnn.py with BF16 weights and
stored activations and FP32 accumulation, in an order of its own; the oracle
evaluates it in FP64 with the same BF16 roundings (bf=True).  In general the
two differ by rounding, and a rounding difference in a stored activation
moves everything after it.  On the inputs built here they cannot differ at
all, so the device must reproduce the oracle exactly:

- weights are -1, 0 or +1 (sparse), biases, inputs and targets small
  integers: every forward product and sum is an integer far below 2^24, so
  every FP32 partial sum is exact in any order, and both sides round the same
  exact pre-activation to BF16;
- the output gradient 2 (y - t) / n has n = 512, so every backward value is a
  multiple of 2^-8, and certify() checks that each backward sum (input,
  weight and bias gradients of every layer) has sum |terms| < 2^15: every
  FP32 partial sum of it is then exact in any order;
- the loss's sum of squares is an integer below 2^24;
- a few targets are large odd integers, so some output gradients are not
  BF16 numbers and the rounding of the stored gradients is exercised.

The inputs come from a seeded generator here; certify() reads only the
oracle's values.
"""
from __future__ import annotations

import numpy as np

from oracle import cnn

B, H, W, N_OUT = 2, 8, 8, 4          # output gradient 2 (y - t) / n with n = 512
DENSITY = (0.3, 0.05, 0.05, 0.05, 0.04, 0.2)   # fraction of non-zero weights per layer


def case(seed):
    """(params, x, target, n_out) as float64 arrays of integer values."""
    rng = np.random.default_rng(seed)
    parts = []
    for (ci, co, k, _), d in zip(cnn.layer_specs(N_OUT), DENSITY):
        parts.append(rng.choice([-1.0, 0.0, 1.0], size=co * ci * k * k, p=[d / 2, 1 - d, d / 2]))
        parts.append(rng.integers(-1, 2, size=co).astype(float))
    x = rng.integers(0, 3, size=(B, 3, H, W)).astype(float)
    t = rng.integers(-8, 9, size=(B, N_OUT, H, W)).astype(float)
    # a few large odd targets: their output gradients 2 (y - t) / n need more
    # than BF16's 8 significant bits, so the rounding of the stored gradient
    # is exercised
    pos = rng.choice(t.size, size=6, replace=False)
    t.ravel()[pos] = rng.choice([-1.0, 1.0], size=6) * (2 * rng.integers(150, 250, size=6) + 1)
    return np.concatenate(parts), x, t, N_OUT


def certify(params, x, t, n_out):
    """Raise AssertionError unless every FP32 operation of the library's
    evaluation of this case is exact (see the module docstring).  Returns the
    largest sum |terms| met."""
    loss, g, c, it = cnn.loss_and_grad(params, x, t, n_out, bf=True, intermediates=True)
    L = c["L"]
    assert np.all(np.abs(params) < 8) and np.all(params == np.round(params))
    ins = [c["x0"], c["a1"], c["a2"], c["u3"], c["cat"], c["a5"]]
    gouts = [it["g1"], it["g2"], it["g3"], it["g4"], it["g5"], it["gy"]]
    strides = [1, 2, 1, 1, 1, 1]
    worst = 0.0
    for i in range(6):
        w, b, k, _ = L[i]
        fwd = cnn.conv(np.abs(ins[i]), np.abs(w), np.abs(b), strides[i])
        assert np.all(ins[i] == np.round(ins[i])) and fwd.max() < 2.0 ** 23
        gs = gouts[i] * 256.0
        assert np.all(gs == np.round(gs)), "backward values must be multiples of 2^-8"
        gx, gw, gb = cnn.conv_grads(np.abs(ins[i]), np.abs(w), strides[i], np.abs(gouts[i]))
        worst = max(worst, gx.max(), gw.max(), gb.max())
    assert worst < 2.0 ** 15
    up = np.abs(it["gu3"]).reshape(B, -1, H // 2, 2, W // 2, 2).sum(axis=(3, 5))
    assert up.max() < 2.0 ** 15
    assert np.sum((it["y"] - t) ** 2) < 2.0 ** 24
    return worst


def blocks(n_out):
    """(name, slice) of each layer's weight and bias block in the flat parameter vector."""
    names = ["conv0 (3->24)", "conv1 stride 2 (24->32)", "conv2 (32->32)", "conv3 after up-sampling (32->24)",
             "conv4 on the skip concatenation (48->24)", "head 1x1 (24->n_out)"]
    out, off = [], 0
    for name, (ci, co, k, _) in zip(names, cnn.layer_specs(n_out)):
        nw = co * ci * k * k
        out.append((name + " weights", slice(off, off + nw)))
        out.append((name + " bias", slice(off + nw, off + nw + co)))
        off += nw + co
    return out

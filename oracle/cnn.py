"""Plain NumPy reference of the learned-guess network (oracle, test infrastructure).

The network is not part of the paper's method; it only proposes a starting
point for the SMM iteration.  This module restates the library's
encoder-decoder in FP64 with explicit loops over the 3x3 (or 1x1) taps so
its forward pass and gradients can be checked by finite differences and then
used to check the GPU's hand-written kernels:

  a1 = relu(conv(x, 3 -> 24));  a2 = relu(conv_s2(a1, 24 -> 32));
  a3 = relu(conv(a2, 32 -> 32)); a4 = relu(conv(up2(a3), 32 -> 24));
  a5 = relu(conv([a4, a1], 48 -> 24)); y = conv1x1(a5, 24 -> n_out);
  loss = mean((y - target)^2).

The widths 24 and 32 are the defaults; C1 and C2 are parameters (c1, c2)
of every function, so the same network at about two million parameters
(c1 = 64, c2 = 384) is the same code.

Parameters are one flat vector, layer by layer: weights [cout][cin][k][k],
then biases [cout].  ``bf=True`` rounds weights, the input, every stored
activation and every stored backward gradient to bfloat16 (round to nearest
even), as the GPU does: the tensor-core kernels read both operands of every
product in BF16, so the gradient that enters a layer's backward products
(2 (y - t) / n at the head, and each layer's gradient after its ReLU mask)
is stored in BF16.  The skip part of a1's gradient stays in FP32 until it
is added to the main part; the sum is then rounded.
"""
from __future__ import annotations

import numpy as np

C1, C2, CIN = 24, 32, 3


def layer_specs(n_out, c1=C1, c2=C2):
    """(cin, cout, k, stride) per layer."""
    return [(CIN, c1, 3, 1), (c1, c2, 3, 2), (c2, c2, 3, 1), (c2, c1, 3, 1), (2 * c1, c1, 3, 1), (c1, n_out, 1, 1)]


def num_params(n_out, c1=C1, c2=C2):
    return sum(co * ci * k * k + co for ci, co, k, _ in layer_specs(n_out, c1, c2))


def unpack(params, n_out, c1=C1, c2=C2):
    out, off = [], 0
    for ci, co, k, s in layer_specs(n_out, c1, c2):
        w = params[off:off + co * ci * k * k].reshape(co, ci, k, k)
        off += co * ci * k * k
        b = params[off:off + co]
        off += co
        out.append((w, b, k, s))
    return out


def bf16(x):
    """Round to bfloat16 (nearest even), returned as float64."""
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def conv(x, w, b, stride):
    """Zero-padded 'same' convolution (pad k//2), output size H/stride."""
    B, C, H, W = x.shape
    co, ci, k, _ = w.shape
    pad = k // 2
    Ho, Wo = (H + stride - 1) // stride, (W + stride - 1) // stride
    xp = np.zeros((B, C, H + 2 * pad, W + 2 * pad))
    xp[:, :, pad:pad + H, pad:pad + W] = x
    y = np.zeros((B, co, Ho, Wo)) + b[None, :, None, None]
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride]
            y += np.einsum("bchw,oc->bohw", patch, w[:, :, ky, kx])
    return y


def conv_grads(x, w, stride, gy):
    """Gradients of conv w.r.t. its input and weights, and of the bias."""
    B, C, H, W = x.shape
    co, ci, k, _ = w.shape
    pad = k // 2
    Ho, Wo = gy.shape[2], gy.shape[3]
    xp = np.zeros((B, C, H + 2 * pad, W + 2 * pad))
    xp[:, :, pad:pad + H, pad:pad + W] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride]
            gw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", gy, patch)
            gxp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride] += np.einsum("bohw,oc->bchw", gy, w[:, :, ky, kx])
    return gxp[:, :, pad:pad + H, pad:pad + W], gw, gy.sum(axis=(0, 2, 3))


def forward(params, x, n_out, bf=False, c1=C1, c2=C2):
    q = bf16 if bf else (lambda v: v)
    L = unpack(params, n_out, c1, c2)
    Lq = [(q(w), b, k, s) for (w, b, k, s) in L]
    x0 = q(x)
    a1 = q(np.maximum(conv(x0, Lq[0][0], Lq[0][1], 1), 0.0))
    a2 = q(np.maximum(conv(a1, Lq[1][0], Lq[1][1], 2), 0.0))
    a3 = q(np.maximum(conv(a2, Lq[2][0], Lq[2][1], 1), 0.0))
    u3 = np.repeat(np.repeat(a3, 2, axis=2), 2, axis=3)
    a4 = q(np.maximum(conv(u3, Lq[3][0], Lq[3][1], 1), 0.0))
    cat = np.concatenate([a4, a1], axis=1)
    a5 = q(np.maximum(conv(cat, Lq[4][0], Lq[4][1], 1), 0.0))
    y = conv(a5, Lq[5][0], Lq[5][1], 1)
    return y, dict(x0=x0, a1=a1, a2=a2, a3=a3, u3=u3, a4=a4, cat=cat, a5=a5, L=Lq)


def loss_and_grad(params, x, target, n_out, bf=False, intermediates=False, c1=C1, c2=C2):
    """Loss and the flat parameter gradient; with intermediates=True also the
    forward cache and the gradients w.r.t. each layer's output before its
    ReLU mask is applied (keys gy, gu5, gucat, gu3, gu2, gu1: the gradient
    that reaches a5, [a4, a1], u3, a2, a1 from the layer above)."""
    q = bf16 if bf else (lambda v: v)
    y, c = forward(params, x, n_out, bf, c1, c2)
    r = y - target
    loss = float(np.mean(r * r))
    gy = q(2.0 * r / r.size)
    L = c["L"]
    grads = []
    gu5, gw5, gb5 = conv_grads(c["a5"], L[5][0], 1, gy)
    g5 = q(gu5 * (c["a5"] > 0))
    gcat, gw4, gb4 = conv_grads(c["cat"], L[4][0], 1, g5)
    g4 = q(gcat[:, :c1] * (c["a4"] > 0))
    g1_skip = gcat[:, c1:] * (c["a1"] > 0)
    gu3, gw3, gb3 = conv_grads(c["u3"], L[3][0], 1, g4)
    gsum3 = gu3.reshape(gu3.shape[0], gu3.shape[1], gu3.shape[2] // 2, 2, gu3.shape[3] // 2, 2).sum(axis=(3, 5))
    g3 = q(gsum3 * (c["a3"] > 0))
    gu2, gw2, gb2 = conv_grads(c["a2"], L[2][0], 1, g3)
    g2 = q(gu2 * (c["a2"] > 0))
    gu1, gw1, gb1 = conv_grads(c["a1"], L[1][0], 2, g2)
    g1 = q(gu1 * (c["a1"] > 0) + g1_skip)
    _, gw0, gb0 = conv_grads(c["x0"], L[0][0], 1, g1)
    for gw, gb in ((gw0, gb0), (gw1, gb1), (gw2, gb2), (gw3, gb3), (gw4, gb4), (gw5, gb5)):
        grads.append(gw.ravel())
        grads.append(gb)
    if intermediates:
        inter = dict(gy=gy, gu5=gu5, g5=g5, gucat=gcat, g4=g4, g1_skip=g1_skip, gu3=gu3, gsum3=gsum3, g3=g3, gu2=gu2,
                     g2=g2, gu1=gu1, g1=g1, y=y)
        return loss, np.concatenate(grads), c, inter
    return loss, np.concatenate(grads)

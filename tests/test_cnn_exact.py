"""CPU checks of the exact network cases (tests/cnn_exact.py) that the GPU
network test compares bit for bit: the exactness certificate holds for the
seeds the GPU test uses; an evaluation in the library's arithmetic (BF16
weights, stored activations and stored backward gradients, FP32
accumulation), written here in NumPy
float32 with its own summation order, reproduces the oracle exactly on them;
and plausible mistakes planted in that evaluation -- one per kind of layer
(the 1x1 head, the skip concatenation, the stride-2 convolution, the
up-sampling, a ReLU mask, a bias) -- each change some output value or
gradient entry, so the GPU test would catch the same mistake in a kernel."""
import numpy as np
import pytest

from oracle import cnn
from tests import cnn_exact

SEEDS = [0, 1, 3]


def _bf(v):
    return cnn.bf16(v).astype(np.float32)


def _conv32(x, w, b, stride):
    B, C, H, W = x.shape
    co, ci, k, _ = w.shape
    pad = k // 2
    Ho, Wo = (H + stride - 1) // stride, (W + stride - 1) // stride
    xp = np.zeros((B, C, H + 2 * pad, W + 2 * pad), np.float32)
    xp[:, :, pad:pad + H, pad:pad + W] = x
    y = np.zeros((B, co, Ho, Wo), np.float32) + b[None, :, None, None].astype(np.float32)
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride]
            y += np.einsum("bchw,oc->bohw", patch, w[:, :, ky, kx]).astype(np.float32)
    return y


def _conv_grads32(x, w, stride, gy, wrong_stride=False):
    B, C, H, W = x.shape
    co, ci, k, _ = w.shape
    pad = k // 2
    Ho, Wo = gy.shape[2], gy.shape[3]
    xp = np.zeros((B, C, H + 2 * pad, W + 2 * pad), np.float32)
    xp[:, :, pad:pad + H, pad:pad + W] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w, dtype=np.float32)
    s_w = 1 if wrong_stride else stride
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, :, ky:ky + s_w * Ho:s_w, kx:kx + s_w * Wo:s_w]
            gw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", gy, patch)
            gxp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride] += \
                np.einsum("bohw,oc->bchw", gy, w[:, :, ky, kx]).astype(np.float32)
    return gxp[:, :, pad:pad + H, pad:pad + W], gw, gy.sum(axis=(0, 2, 3), dtype=np.float32)


def _emulate(params, x, t, n_out, mistake=None):
    """(y, loss, flat gradient) in the library's arithmetic, with an optional planted mistake."""
    L = [(_bf(w), b.astype(np.float32), k, s) for (w, b, k, s) in cnn.unpack(params, n_out)]
    if mistake == "conv3_bias_dropped":
        L[3] = (L[3][0], np.zeros_like(L[3][1]), L[3][2], L[3][3])
    x0 = _bf(x)
    a1 = _bf(np.maximum(_conv32(x0, L[0][0], L[0][1], 1), 0))
    a2 = _bf(np.maximum(_conv32(a1, L[1][0], L[1][1], 2), 0))
    a3 = _bf(np.maximum(_conv32(a2, L[2][0], L[2][1], 1), 0))
    u3 = np.repeat(np.repeat(a3, 2, axis=2), 2, axis=3)
    a4 = _bf(np.maximum(_conv32(u3, L[3][0], L[3][1], 1), 0))
    cat = np.concatenate([a4, a1], axis=1)
    a5 = _bf(np.maximum(_conv32(cat, L[4][0], L[4][1], 1), 0))
    y = _conv32(a5, L[5][0], L[5][1], 1)
    r = (y - t.astype(np.float32)).astype(np.float32)
    loss = float(np.sum(r * r, dtype=np.float32)) / r.size
    gy = (np.float32(2.0) * r / np.float32(r.size)).astype(np.float32)
    if mistake != "gradient_kept_in_fp32":
        gy = _bf(gy)
    gu5, gw5, gb5 = _conv_grads32(a5, L[5][0], 1, gy)
    if mistake == "head_bias_misses_a_sample":
        gb5 = gy[:-1].sum(axis=(0, 2, 3), dtype=np.float32)
    g5 = _bf(gu5 if mistake == "a5_mask_dropped" else gu5 * (a5 > 0))
    gcat, gw4, gb4 = _conv_grads32(cat, L[4][0], 1, g5)
    C1 = cnn.C1
    g4 = _bf(gcat[:, :C1] * (a4 > 0))
    g1_skip = gcat[:, C1:] * (a1 > 0)
    gu3, gw3, gb3 = _conv_grads32(u3, L[3][0], 1, g4)
    if mistake == "upsampling_backward_takes_one_of_four":
        gs3 = 4.0 * gu3[:, :, ::2, ::2]
    else:
        gs3 = gu3.reshape(gu3.shape[0], gu3.shape[1], gu3.shape[2] // 2, 2, gu3.shape[3] // 2, 2).sum(axis=(3, 5))
    g3 = _bf(gs3 * (a3 > 0))
    gu2, gw2, gb2 = _conv_grads32(a2, L[2][0], 1, g3)
    g2 = _bf(gu2 * (a2 > 0))
    gu1, gw1, gb1 = _conv_grads32(a1, L[1][0], 2, g2, wrong_stride=mistake == "stride2_weight_grad_at_stride1")
    g1 = gu1 * (a1 > 0)
    if mistake != "skip_gradient_dropped":
        g1 = (g1 + g1_skip).astype(np.float32)
    g1 = _bf(g1)
    _, gw0, gb0 = _conv_grads32(x0, L[0][0], 1, g1)
    g = np.concatenate([v.ravel() for v in (gw0, gb0, gw1, gb1, gw2, gb2, gw3, gb3, gw4, gb4, gw5, gb5)])
    return y, loss, g


@pytest.mark.parametrize("seed", SEEDS)
def test_certified_cases_are_reproduced_exactly_in_any_order(seed):
    params, x, t, n_out = cnn_exact.case(seed)
    cnn_exact.certify(params, x, t, n_out)
    loss_o, g_o, _, it = cnn.loss_and_grad(params, x, t, n_out, bf=True, intermediates=True)
    y, loss, g = _emulate(params.astype(np.float32), x.astype(np.float32), t.astype(np.float32), n_out)
    assert np.array_equal(y, it["y"]) and loss == loss_o and np.array_equal(g, g_o)
    # the cases exercise every layer: each block has non-zero gradient entries
    for name, sl in cnn_exact.blocks(n_out):
        assert np.count_nonzero(g_o[sl]) > 0, name


@pytest.mark.parametrize("mistake", ["gradient_kept_in_fp32", "conv3_bias_dropped", "head_bias_misses_a_sample", "a5_mask_dropped",
                                     "upsampling_backward_takes_one_of_four", "stride2_weight_grad_at_stride1",
                                     "skip_gradient_dropped"])
def test_planted_mistakes_change_the_exact_results(mistake):
    params, x, t, n_out = cnn_exact.case(SEEDS[0])
    loss_o, g_o, _, it = cnn.loss_and_grad(params, x, t, n_out, bf=True, intermediates=True)
    y, loss, g = _emulate(params.astype(np.float32), x.astype(np.float32), t.astype(np.float32), n_out, mistake)
    assert not (np.array_equal(y, it["y"]) and np.array_equal(g, g_o)), mistake

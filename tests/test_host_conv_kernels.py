"""CPU test of the learned-guess network's tensor-core kernels (cnn.cu),
compiled for the host with tests/host_kernel_shim.h and emulations of
mma.sync.m16n8k16 and ldmatrix.x4 (plain and transposed) in the register
layouts the PTX ISA documents, and of cp.async as an immediate copy or zero
fill (tests/conv_emu.cpp).  One convolution layer per case -- the first layer's
3 padded input channels, a stride-2 layer, the skip concatenation, the 1x1
head, several output tiles, ragged pixel counts -- through the forward pass
(with and without ReLU), the input gradient (ReLU masks, an FP32 addend,
BF16 and FP32 outputs; for a stride-2 layer one launch per parity class of
input pixels over the taps that reach an output pixel, as the library does), and the weight and bias gradients through their
split partials, against the oracle's convolution and its gradients.  The
values are small integers and multiples of 2^-8, so every sum is exact in
any order and the comparison is exact."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle import cnn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_07386_gb300", "csrc")


def extract(src, signature):
    """The definition starting at `signature` (with a template line just above
    it), through its closing brace."""
    i = src.index(signature)
    line_start = src.rfind("\n", 0, i - 1) + 1
    if src.startswith("template", line_start):
        i = line_start
    depth, k = 0, src.index("{", i)
    while True:
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            return src[i:k + 1]
        k += 1


@pytest.fixture(scope="module")
def conv_emu(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("conv_emu")
    src = open(os.path.join(CSRC, "cnn.cu")).read()
    consts = "\n".join(re.findall(r"^constexpr int k[A-Za-z]+ = .*$", src, flags=re.M))
    parts = [consts,
             extract(src, "struct ConvGeom {") + ";",
             extract(src, "struct GradPart {") + ";",
             extract(src, "struct GemmArgs {") + ";",
             "enum { kFwd = 0, kBwdData = 1, kBwdWeight = 2 };",
             extract(src, "__device__ __forceinline__ float bf("),
             extract(src, "__global__ void __launch_bounds__(kGemmThreads, 5) conv_gemm_kernel("),
             extract(src, "__device__ __forceinline__ int real_channel("),
             extract(src, "__global__ void repack_kernel("),
             extract(src, "__global__ void bias_partial_kernel("),
             extract(src, "__global__ void grad_reduce_kernel("),
             extract(src, "void weight_splits("),
             extract(src, "int class_taps(")]
    (d / "conv_kernels.inc").write_text("\n\n".join(parts))
    exe = d / "conv_emu"
    subprocess.run([cxx, "-std=c++20", "-O1", "-ffp-contract=off", "-pthread", "-I", str(d), "-I",
                    os.path.join(ROOT, "tests"), os.path.join(ROOT, "tests", "conv_emu.cpp"), "-o", str(exe)],
                   check=True)
    return str(exe)


def _p16(c):
    return (c + 15) // 16 * 16


def _bits(a):
    """float64 values already in BF16 -> uint16 bits"""
    return (a.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def _from_bits(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _nhwc(x, cp):
    """[B][C][H][W] -> [B][H][W][cp] with zero pad channels"""
    B, C, H, W = x.shape
    out = np.zeros((B, H, W, cp))
    out[..., :C] = x.transpose(0, 2, 3, 1)
    return out


# (B, Hin, Win, k, stride, ca, cb, cout)
CASES = [(2, 8, 8, 3, 1, 3, 0, 24),       # first layer: 3 real of 16 stored input channels
         (1, 6, 10, 3, 2, 24, 0, 20),     # stride 2, ragged pixel count, padded channels
         (2, 6, 6, 3, 1, 24, 24, 24),     # skip concatenation
         (2, 10, 6, 1, 1, 24, 0, 9),      # 1x1 head
         (1, 12, 12, 3, 1, 40, 0, 72),    # two output-channel tiles, 160-pixel rows
         (3, 16, 16, 3, 2, 16, 0, 32)]    # three pixel tiles of the weight gradient


@pytest.mark.parametrize("case", CASES)
def test_conv_kernels_match_oracle_exactly(conv_emu, tmp_path, case):
    B, H, W, k, s, ca, cb, cout = case
    rng = np.random.default_rng(hash(case) % 2 ** 32)
    Ka, Kb, Np = _p16(ca), (_p16(cb) if cb else 0), _p16(cout)
    Ho, Wo = (H + s - 1) // s, (W + s - 1) // s
    xa = rng.integers(0, 3, size=(B, ca, H, W)).astype(float)
    xb = rng.integers(0, 3, size=(B, cb, H, W)).astype(float)
    w = rng.choice([-1.0, 0.0, 1.0], size=(cout, ca + cb, k, k), p=[0.3, 0.4, 0.3])
    b = rng.integers(-2, 3, size=cout).astype(float)
    gy = rng.integers(-8, 9, size=(B, cout, Ho, Wo)) / 256.0
    ma = rng.integers(0, 2, size=(B, ca, H, W)).astype(float)
    mb = rng.integers(0, 2, size=(B, cb, H, W)).astype(float)
    add = rng.integers(-8, 9, size=(B, ca, H, W)) / 256.0
    _bits(_nhwc(xa, Ka)).tofile(tmp_path / "in_a.bf16")
    _bits(_nhwc(ma, Ka)).tofile(tmp_path / "act_a.bf16")
    _nhwc(add, Ka).astype(np.float32).tofile(tmp_path / "add_a.f32")
    if cb:
        _bits(_nhwc(xb, Kb)).tofile(tmp_path / "in_b.bf16")
        _bits(_nhwc(mb, Kb)).tofile(tmp_path / "act_b.bf16")
    _bits(_nhwc(gy, Np)).tofile(tmp_path / "gout.bf16")
    w.astype(np.float32).tofile(tmp_path / "w.f32")
    b.astype(np.float32).tofile(tmp_path / "bias.f32")
    env = dict(os.environ, BIAS_CHUNK="40")
    subprocess.run([conv_emu, str(tmp_path), *map(str, case)], check=True, timeout=600, env=env)

    x = np.concatenate([xa, xb], axis=1)
    pre = cnn.conv(x, w, b, s)
    fwd = _from_bits(np.fromfile(tmp_path / "fwd.bf16", np.uint16)).reshape(B, Ho, Wo, Np)
    assert np.array_equal(fwd, _nhwc(cnn.bf16(np.maximum(pre, 0.0)), Np))
    nchw = np.fromfile(tmp_path / "fwd_nchw.f32", np.float32).reshape(B, cout, Ho, Wo)
    assert np.array_equal(nchw, pre)

    gx, gw, gb = cnn.conv_grads(x, w, s, gy)
    gin_a = _from_bits(np.fromfile(tmp_path / "gin_a.bf16", np.uint16)).reshape(B, H, W, Ka)
    assert np.array_equal(gin_a, _nhwc(cnn.bf16(gx[:, :ca] * ma + add), Ka))
    if cb:
        gin_b = np.fromfile(tmp_path / "gin_b.f32", np.float32).reshape(B, H, W, Kb)
        assert np.array_equal(gin_b, _nhwc(gx[:, ca:] * mb, Kb))
    assert np.array_equal(np.fromfile(tmp_path / "gw.f32", np.float32).reshape(gw.shape), gw)
    assert np.array_equal(np.fromfile(tmp_path / "gb.f32", np.float32), gb)
    assert np.count_nonzero(gw) > 0 and np.count_nonzero(gx) > 0

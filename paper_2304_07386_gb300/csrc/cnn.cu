// Learned initial guess: a convolutional encoder-decoder on the element grid,
// trained and run with this file's own kernels (BF16 weights, activations and
// stored gradients, FP32 accumulation on the tensor cores, FP32 master weights
// and Adam state).
//
// Network (all convolutions 3x3, zero padding 1, except the last 1x1):
//   a1 = relu(conv(x, 3 -> C1))                 full resolution
//   a2 = relu(conv_stride2(a1, C1 -> C2))       half resolution
//   a3 = relu(conv(a2, C2 -> C2))               half resolution
//   a4 = relu(conv(up2(a3), C2 -> C1))          full resolution (nearest up-sampling)
//   a5 = relu(conv([a4, a1], 2 C1 -> C1))       skip connection by channel concatenation
//   y  = conv1x1(a5, C1 -> n_out)
// with widths C1, C2 chosen at create (24 / 32 for the small network, 64 / 384
// for about two million parameters).  Loss: mean squared error.
//
// Every convolution pass is an implicit GEMM on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulators): activations and
// gradients live in HBM as [batch][y][x][channel] with the channel count
// padded to a multiple of 16 (pad channels hold zero), so that 8 consecutive
// reduction indices (one tap, 8 channels) are one 16-byte load.
//   forward      out[pixel][co]  = sum_{tap, c} in[pixel + tap][c] Wf[co][tap, c]
//   input grad   gin[pixel][c]   = sum_{tap, co} gout[pixel - tap][co] Wb[c][tap, co]
//   weight grad  gw[co][tap, c]  = sum_{pixel} gout[pixel][co] in[pixel + tap][c]
// The first two gather their A rows (pixels) and read the repacked BF16
// weights (Wf, Wb, rebuilt from the FP32 masters after every update); the
// third reduces over pixels in split chunks whose FP32 partials are summed in
// a fixed order, so every result is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/smm.h"
#include "kernels.cuh"

namespace {

constexpr int kIn = 3;
constexpr int kBM = 64, kBN = 64, kBK = 32, kLds = kBK + 8;  // block tile; smem row of kLds BF16
constexpr int kLdt = kBM + 8;  // weight grad: smem row (one pixel) of kLdt BF16 channels
constexpr int kGemmThreads = 128;                          // four warps, each a 32 x 32 piece
constexpr int kStages = 3;                                 // shared-memory stages of the copy pipeline
constexpr int kWgradBlocks = 2 * 5 * 152;                  // weight grad: two waves of five CTAs per SM

smm_status fail(smm_status s, const std::string& msg) {
    smm::set_last_error(msg.c_str());
    return s;
}

inline int pad16(int c) { return (c + 15) / 16 * 16; }

// A convolution pass as the GEMM kernel sees it.  Input channels come from up
// to two tensors (the skip concatenation): part a has ca real channels stored
// with Ka (padded) per pixel, part b cb / Kb; Kc = Ka + Kb.  Output channels:
// cout real, Np = pad16(cout) stored.
struct ConvGeom {
    int B, Hin, Win, Hout, Wout;
    int ksz, stride, pad, taps;
    int ca, Ka, cb, Kb, Kc, cout, Np;
};

// Epilogue of an input-gradient pass for the channels of one input part:
// v = acc; v *= (act > 0) if act; v += add if add; stored to out_bf (BF16) or
// out_f (FP32), ld channels per pixel.
struct GradPart {
    const __nv_bfloat16* act;
    const float* add;
    __nv_bfloat16* out_bf;
    float* out_f;
    int ld;
};

struct GemmArgs {
    ConvGeom g;
    int M, N, K;
    const __nv_bfloat16* in_a;  // forward / weight grad: the input parts
    const __nv_bfloat16* in_b;
    const __nv_bfloat16* gout;  // input / weight grad: the output gradient (Np channels)
    const __nv_bfloat16* wt;    // forward: Wf [Np][taps*Kc]; input grad: Wb [Kc][taps*Np]
    // forward epilogue
    const float* bias;
    int relu;
    __nv_bfloat16* out_bf;  // [pixel][Np]
    float* out_nchw;        // [b][cout][y][x] (the head)
    // input-grad epilogue
    GradPart part[2];
    // weight grad: FP32 partials [split][Np][taps*Kc], kchunk pixels per split
    float* wpart;
    int kchunk;
    // row length of wt (taps * Kc or taps * Np)
    int wt_ld;
    // input grad of a strided layer, one launch per parity class of input pixels: rows are the pixels
    // (b, stride qy + py, stride qx + px), the reduction runs over the ntap taps tapk[] that reach an
    // output pixel from that class (K = ntap * Np).  cls = 0: every pixel and every tap.
    int cls, py, px, ntap;
    int tapk[9];
};

enum { kFwd = 0, kBwdData = 1, kBwdWeight = 2 };

// D += A B on a 16 x 8 x 16 tile: A row-major BF16 pairs, B column-major BF16
// pairs, FP32 accumulators (the register layout of mma.sync.m16n8k16).
__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Four 8 x 8 BF16 matrices from shared memory: lane l gives the address of row
// l % 8 of matrix l / 8 (16 contiguous bytes); register j of lane t receives
// row t / 4, columns 2 (t % 4) and 2 (t % 4) + 1 of matrix j (ldmatrix.x4), or
// with .trans rows 2 (t % 4), 2 (t % 4) + 1 of column t / 4.
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const __nv_bfloat16* p) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t* r, const __nv_bfloat16* p) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// 16 bytes global -> shared without a register stop (cp.async, L2 only); with valid == false nothing is
// read and the 16 bytes are zero-filled (src must still be a valid global address).  The copies of one
// thread form groups (commit); wait_group<N> returns once at most N of its newest groups are pending.
__device__ __forceinline__ void cp_async16(__nv_bfloat16* dst, const __nv_bfloat16* src, bool valid) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// One 64 x 64 tile of a convolution pass per block (blockIdx.z: the weight
// gradient's pixel split).  The reduction runs in steps of 32 through a
// pipeline of kStages shared-memory stages: each thread copies its 16-byte
// pieces of step st + kStages - 1 with cp.async (zero-filled at the image
// border and past the end) while the products of step st run; one barrier
// per step.  Forward and input gradient keep
// both operands as rows of 32 reduction indices ([m][k], [n][k]); the weight
// gradient, whose reduction index is the pixel, keeps them as rows of
// channels ([k][m], [k][n]) and reads its fragments transposed.
template <int MODE>
__global__ void __launch_bounds__(kGemmThreads, 5) conv_gemm_kernel(const GemmArgs args) {
    __shared__ __align__(16) __nv_bfloat16 sA[kStages][kBM * kLds];
    __shared__ __align__(16) __nv_bfloat16 sB[kStages][kBN * kLds];
    const ConvGeom& g = args.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    int k_begin = 0, k_end = args.K;
    if (MODE == kBwdWeight) {
        k_begin = blockIdx.z * args.kchunk;
        k_end = min(args.K, k_begin + args.kchunk);
    }
    const int hw_out = g.Hout * g.Wout, hw_in = g.Hin * g.Win;

    // The reduction index of this thread's chunks advances by kBK per step; its decomposition is kept
    // up to date without divisions.  Forward / input grad: every chunk of the thread has k = k0 + 8 (tid % 4),
    // split into (tap ti of the launch's taps, channel c < Kd); ctap = ky ksz + kx is the tap itself (ti, or
    // tapk[ti] for a parity class); the two A rows (pixels) are fixed.  Weight grad: both chunks have pixel
    // kk = k0 + tid % 32, split into (b, oy, ox); the channels of the two B chunks (tap, c) are fixed.
    const int Kd = MODE == kFwd ? g.Kc : g.Np;
    const bool cls = MODE == kBwdData && args.cls;
    int rb_[2] = {0, 0}, ry_[2] = {0, 0}, rx_[2] = {0, 0};
    bool rok[2] = {false, false};
    int cc = 0, ti = 0, ctap = 0, cky = 0, ckx = 0;  // forward / input grad: channel and tap of k
    int pb = 0, poy = 0, pox = 0;                  // weight grad: pixel kk
    int nky[2] = {0, 0}, nkx[2] = {0, 0}, nc[2] = {0, 0};
    bool nok[2] = {false, false};
    if (MODE != kBwdWeight) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int m = m0 + ((tid + i * kGemmThreads) >> 2);
            rok[i] = m < args.M;
            if (cls) {
                const int wd = g.Win / g.stride, hw = (g.Hin / g.stride) * wd;
                rb_[i] = m / hw;
                ry_[i] = (m % hw) / wd * g.stride + args.py;
                rx_[i] = m % wd * g.stride + args.px;
            } else {
                const int hw = MODE == kFwd ? hw_out : hw_in, wd = MODE == kFwd ? g.Wout : g.Win;
                rb_[i] = m / hw;
                ry_[i] = (m % hw) / wd;
                rx_[i] = m % wd;
            }
        }
        const int k = k_begin + (tid & 3) * 8;
        ti = k / Kd;
        cc = k - ti * Kd;
        ctap = cls ? args.tapk[ti < args.ntap ? ti : 0] : ti;
        cky = ctap / g.ksz;
        ckx = ctap - cky * g.ksz;
    } else {
        const int kk = k_begin + (tid & 31), rem = kk % hw_out;
        pb = kk / hw_out;
        poy = rem / g.Wout;
        pox = rem - poy * g.Wout;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int n = n0 + ((tid + i * kGemmThreads) >> 5) * 8, tap = n / g.Kc;
            nok[i] = n < args.N;
            nc[i] = n - tap * g.Kc;
            nky[i] = tap / g.ksz;
            nkx[i] = tap - nky[i] * g.ksz;
        }
    }
    auto advance = [&]() {
        if (MODE != kBwdWeight) {
            cc += kBK;
            while (cc >= Kd) {
                cc -= Kd;
                ++ti;
                if (cls) {
                    ctap = args.tapk[ti < args.ntap ? ti : 0];
                    cky = ctap / g.ksz;
                    ckx = ctap - cky * g.ksz;
                } else {
                    ++ctap;
                    if (++ckx == g.ksz) {
                        ckx = 0;
                        ++cky;
                    }
                }
            }
        } else {
            pox += kBK;
            while (pox >= g.Wout) {
                pox -= g.Wout;
                if (++poy == g.Hout) {
                    poy = 0;
                    ++pb;
                }
            }
        }
    };
    auto src_of = [&](size_t pix, int c) {
        return c < g.Ka ? args.in_a + pix * g.Ka + c : args.in_b + pix * g.Kb + (c - g.Ka);
    };

    // copies of the reduction step starting at k0 (the state above describes k0) into stage sg
    auto load = [&](int k0, int sg) {
        const __nv_bfloat16* any = args.wt ? args.wt : args.gout;  // a valid address for zero-filled pieces
        if (MODE != kBwdWeight) {
            const int kc = (tid & 3) * 8, k = k0 + kc;
            const bool kin = k < k_end;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = (tid + i * kGemmThreads) >> 2;
                const __nv_bfloat16* src = any;
                bool ok = false;
                if (MODE == kFwd) {
                    const int iy = ry_[i] * g.stride + cky - g.pad, ix = rx_[i] * g.stride + ckx - g.pad;
                    ok = kin && rok[i] && iy >= 0 && iy < g.Hin && ix >= 0 && ix < g.Win;
                    if (ok) src = src_of(((size_t)rb_[i] * g.Hin + iy) * g.Win + ix, cc);
                } else {
                    int oy = ry_[i] + g.pad - cky, ox = rx_[i] + g.pad - ckx;
                    ok = kin && rok[i] && oy >= 0 && ox >= 0;
                    if (g.stride != 1) {
                        ok = ok && oy % g.stride == 0 && ox % g.stride == 0;
                        oy /= g.stride;
                        ox /= g.stride;
                    }
                    ok = ok && oy < g.Hout && ox < g.Wout;
                    if (ok) src = args.gout + (((size_t)rb_[i] * g.Hout + oy) * g.Wout + ox) * g.Np + cc;
                }
                cp_async16(&sA[sg][r * kLds + kc], src, ok);
                const int n = n0 + r;
                const bool nok_ = kin && n < args.N;
                cp_async16(&sB[sg][r * kLds + kc], nok_ ? args.wt + (size_t)n * args.wt_ld + ctap * Kd + cc : any,
                           nok_);
            }
        } else {
            const int p = tid & 31, kk = k0 + p;
            const bool kin = kk < k_end;
            const __nv_bfloat16* grow = args.gout + (size_t)(kin ? kk : 0) * g.Np;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int j8 = ((tid + i * kGemmThreads) >> 5) * 8;
                const bool aok = kin && m0 + j8 < args.M;
                cp_async16(&sA[sg][p * kLdt + j8], aok ? grow + m0 + j8 : any, aok);
                const int iy = poy * g.stride + nky[i] - g.pad, ix = pox * g.stride + nkx[i] - g.pad;
                const bool bok = kin && nok[i] && iy >= 0 && iy < g.Hin && ix >= 0 && ix < g.Win;
                cp_async16(&sB[sg][p * kLdt + j8],
                           bok ? src_of(((size_t)pb * g.Hin + iy) * g.Win + ix, nc[i]) : any, bok);
            }
        }
    };

    float acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.0f;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32, gq = lane >> 2, tq = lane & 3;

    const int nsteps = k_end > k_begin ? (k_end - k_begin + kBK - 1) / kBK : 0;
    // prologue: steps 0 .. kStages - 2 in flight (one commit group per step, empty past the end)
#pragma unroll
    for (int sg = 0; sg < kStages - 1; ++sg) {
        if (sg < nsteps) {
            if (sg > 0) advance();
            load(k_begin + sg * kBK, sg);
        }
        cp_async_commit();
    }
    for (int st = 0; st < nsteps; ++st) {
        const int cur = st % kStages;
        cp_async_wait<kStages - 2>();  // this thread's pieces of step st have landed
        __syncthreads();               // everyone's have; everyone is done with step st - 1's stage
        {
            const int nx = st + kStages - 1;
            if (nx < nsteps) {
                advance();
                load(k_begin + nx * kBK, nx % kStages);
            }
            cp_async_commit();
        }
#pragma unroll
        for (int ks = 0; ks < kBK; ks += 16) {
            // A of rows wm + 16 mi: matrices (rows 0-7 | 8-15) x (k 0-7 | 8-15) in the order a0..a3;
            // B of columns wn + 8 nj, two n8 tiles per load: (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, ...)
            uint32_t af[2][4], bq[4][2];
            const int r8 = lane & 7, j1 = (lane >> 3) & 1, j2 = lane >> 4;
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                if (MODE != kBwdWeight)
                    ldsm_x4(af[mi], &sA[cur][(wm + mi * 16 + r8 + 8 * j1) * kLds + ks + 8 * j2]);
                else
                    ldsm_x4_trans(af[mi], &sA[cur][(ks + 8 * j2 + r8) * kLdt + wm + mi * 16 + 8 * j1]);
            }
#pragma unroll
            for (int nj = 0; nj < 4; nj += 2) {
                uint32_t r[4];
                if (MODE != kBwdWeight)
                    ldsm_x4(r, &sB[cur][(wn + nj * 8 + r8 + 8 * j2) * kLds + ks + 8 * j1]);
                else
                    ldsm_x4_trans(r, &sB[cur][(ks + 8 * j1 + r8) * kLdt + wn + nj * 8 + 8 * j2]);
                bq[nj][0] = r[0];
                bq[nj][1] = r[1];
                bq[nj + 1][0] = r[2];
                bq[nj + 1][1] = r[3];
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16_16816(acc[mi][ni], af[mi], bq[ni]);
        }
    }
    cp_async_wait<0>();

    // epilogue: accumulator e of tile (mi, ni) is row gq + 8 (e >> 1), column 2 tq + (e & 1)
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = m0 + wm + mi * 16 + gq + 8 * (e >> 1);
                const int col = n0 + wn + ni * 8 + 2 * tq + (e & 1);
                if (row >= args.M || col >= args.N) continue;
                float v = acc[mi][ni][e];
                if (MODE == kFwd) {
                    if (col < g.cout) v += args.bias[col];
                    if (args.relu) v = fmaxf(v, 0.0f);
                    if (args.out_bf) args.out_bf[(size_t)row * g.Np + col] = __float2bfloat16(v);
                    if (args.out_nchw && col < g.cout) {
                        const int b = row / hw_out, rem = row - b * hw_out;
                        args.out_nchw[((size_t)b * g.cout + col) * hw_out + rem] = v;
                    }
                } else if (MODE == kBwdData) {
                    const int pi = col < g.Ka ? 0 : 1, lc = pi ? col - g.Ka : col;
                    const GradPart& P = args.part[pi];
                    size_t pix = (size_t)row;
                    if (cls) {
                        const int wd = g.Win / g.stride, hw = (g.Hin / g.stride) * wd;
                        const int b = row / hw, qy = (row % hw) / wd, qx = row % wd;
                        pix = ((size_t)b * g.Hin + qy * g.stride + args.py) * g.Win + qx * g.stride + args.px;
                    }
                    const size_t idx = pix * P.ld + lc;
                    if (P.act && !(bf(P.act[idx]) > 0.0f)) v = 0.0f;
                    if (P.add) v += P.add[idx];
                    if (P.out_bf) P.out_bf[idx] = __float2bfloat16(v);
                    if (P.out_f) P.out_f[idx] = v;
                } else {
                    args.wpart[((size_t)blockIdx.z * g.Np + row) * args.N + col] = v;
                }
            }
}

// x [b][3][y][x] FP32 -> [b][y][x][16] BF16 (channels 3..15 zero)
__global__ void pack_input_kernel(int B, int H, int W, const float* __restrict__ in, __nv_bfloat16* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long hw = (long long)H * W, tot = (long long)B * hw * 16;
    if (t >= tot) return;
    const int c = (int)(t & 15);
    const long long pix = t >> 4, b = pix / hw, rem = pix - b * hw;
    out[t] = __float2bfloat16(c < kIn ? in[(b * kIn + c) * hw + rem] : 0.0f);
}

// nearest up-sampling of [b][h][w][C] to [b][2h][2w][C], 8 channels per thread
__global__ void upsample_kernel(int B, int H, int W, int C, const __nv_bfloat16* __restrict__ in,
                                __nv_bfloat16* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c8 = C / 8;
    const long long tot = (long long)B * 4 * H * W * c8;
    if (t >= tot) return;
    const int j = (int)(t % c8);
    const long long pix = t / c8;
    const int x = (int)(pix % (2 * W)), y = (int)((pix / (2 * W)) % (2 * H));
    const long long b = pix / (4LL * H * W);
    reinterpret_cast<uint4*>(out)[t] =
        reinterpret_cast<const uint4*>(in)[((b * H + y / 2) * W + x / 2) * c8 + j];
}

// g[b][y][x][c] = bf16((a[b][y][x][c] > 0) * sum of the four up-sampled gradients gup[b][2y+i][2x+j][c])
__global__ void upsample_bwd_kernel(int B, int H, int W, int C, const float* __restrict__ gup,
                                    const __nv_bfloat16* __restrict__ act, __nv_bfloat16* __restrict__ g) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)B * H * W * C;
    if (t >= tot) return;
    const int c = (int)(t % C);
    const long long pix = t / C;
    const int x = (int)(pix % W), y = (int)((pix / W) % H);
    const long long b = pix / ((long long)H * W);
    const float* r0 = gup + ((b * 2 * H + 2 * y) * 2 * W + 2 * x) * C + c;
    const float* r1 = r0 + (size_t)2 * W * C;
    float s = (r0[0] + r0[C]) + (r1[0] + r1[C]);
    if (!(bf(act[t]) > 0.0f)) s = 0.0f;
    g[t] = __float2bfloat16(s);
}

// gy[b][y][x][co] = bf16(2 (y - target) / count) (layouts: y, target [b][n_out][y][x]; gy with ld
// channels per pixel); partial sums of (y - target)^2 per block
__global__ void mse_kernel(int B, int nout, int hw, int ld, const float* __restrict__ y, const float* __restrict__ tgt,
                           __nv_bfloat16* __restrict__ gy, float* __restrict__ part) {
    __shared__ float sh[256];
    const long long n = (long long)B * nout * hw;
    float acc = 0.0f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float r = y[t] - tgt[t];
        const long long b = t / ((long long)nout * hw), rem = t % hw;
        const int co = (int)((t / hw) % nout);
        gy[(b * hw + rem) * ld + co] = __float2bfloat16(2.0f * r / (float)n);
        acc += r * r;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// real input channel of padded channel c (or -1 for a pad channel)
__device__ __forceinline__ int real_channel(const ConvGeom& g, int c) {
    if (c < g.Ka) return c < g.ca ? c : -1;
    const int cb = c - g.Ka;
    return cb < g.cb ? g.ca + cb : -1;
}

// Wf[n][tap*Kc + c] and Wb[c][tap*Np + n] in BF16 from the FP32 master w[co][ci][tap] (zero where n or c pads)
__global__ void repack_kernel(ConvGeom g, const float* __restrict__ w, __nv_bfloat16* __restrict__ wf,
                              __nv_bfloat16* __restrict__ wb) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)g.Np * g.taps * g.Kc;
    if (t >= tot) return;
    const int c = (int)(t % g.Kc), tap = (int)((t / g.Kc) % g.taps), n = (int)(t / ((long long)g.Kc * g.taps));
    const int ci = real_channel(g, c), cin = g.ca + g.cb;
    const float v = (n < g.cout && ci >= 0) ? w[((size_t)n * cin + ci) * g.taps + tap] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16(v);
    wf[t] = h;
    wb[((size_t)c * g.taps + tap) * g.Np + n] = h;
}

// bias-gradient partials: part[chunk][c] = sum of gout[pixel][c] over the chunk's pixels (64 channels per block)
__global__ void bias_partial_kernel(int npix, int np, int chunk, const __nv_bfloat16* __restrict__ gout,
                                    float* __restrict__ part) {
    __shared__ float sh[4][64];
    const int cl = threadIdx.x & 63, grp = threadIdx.x >> 6, c = blockIdx.x * 64 + cl;
    const int p0 = blockIdx.y * chunk, p1 = min(npix, p0 + chunk);
    float acc = 0.0f;
    if (c < np)
        for (int p = p0 + grp; p < p1; p += 4) acc += bf(gout[(size_t)p * np + c]);
    sh[grp][cl] = acc;
    __syncthreads();
    if (grp == 0 && c < np) part[(size_t)blockIdx.y * np + c] = ((sh[0][cl] + sh[1][cl]) + sh[2][cl]) + sh[3][cl];
}

// weight and bias gradients in the flat layout (w[co][ci][ky][kx], then b[co]) from the split partials,
// each sum over the splits in split order
__global__ void grad_reduce_kernel(ConvGeom g, int wsplits, const float* __restrict__ wpart, int bsplits,
                                   const float* __restrict__ bpart, float* __restrict__ gw, float* __restrict__ gb) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int cin = g.ca + g.cb;
    const long long nw = (long long)g.cout * cin * g.taps;
    if (t < nw) {
        const int tap = (int)(t % g.taps), ci = (int)((t / g.taps) % cin), co = (int)(t / ((long long)g.taps * cin));
        const int c = ci < g.ca ? ci : g.Ka + (ci - g.ca);
        const long long N = (long long)g.taps * g.Kc, col = (long long)tap * g.Kc + c;
        float s = 0.0f;
        for (int k = 0; k < wsplits; ++k) s += wpart[((long long)k * g.Np + co) * N + col];
        gw[t] = s;
    } else if (t < nw + g.cout) {
        const int co = (int)(t - nw);
        float s = 0.0f;
        for (int k = 0; k < bsplits; ++k) s += bpart[(size_t)k * g.Np + co];
        gb[co] = s;
    }
}

__global__ void adam_kernel(long long n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float b1, float b2, float c1, float c2, float eps) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gi = g[t];
    const float mi = b1 * m[t] + (1.0f - b1) * gi;
    const float vi = b2 * v[t] + (1.0f - b2) * gi * gi;
    m[t] = mi;
    v[t] = vi;
    p[t] = p[t] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct smm_guess_ctx {
    int H = 0, W = 0, nout = 0, maxb = 0, c1 = 0, c2 = 0, P1 = 0, P2 = 0, Po = 0;
    cudaStream_t stream = nullptr;
    ConvGeom L[6];                   // per layer, B filled in per call
    size_t w_off[6], b_off[6];       // offsets of each layer's weights and biases in the flat vector
    __nv_bfloat16 *wf[6], *wb[6];    // repacked BF16 weights of each layer
    size_t nparam = 0;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // FP32 master, Adam moments, gradients
    long long step = 0;
    // activations and gradients ([b][y][x][channels padded to 16]) for up to maxb samples
    __nv_bfloat16 *x = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *u3 = nullptr, *a4 = nullptr,
                  *a5 = nullptr, *gy = nullptr, *g5 = nullptr, *g4 = nullptr, *g3 = nullptr, *g2 = nullptr,
                  *g1 = nullptr;
    float *y = nullptr, *g1s = nullptr, *gu = nullptr, *wpart = nullptr, *bpart = nullptr, *part = nullptr;
    std::vector<void*> allocs;
    bool alloc_failed = false;
    template <class T>
    T* alloc(size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
            alloc_failed = true;
            return nullptr;
        }
        allocs.push_back(q);
        return (T*)q;
    }
    ~smm_guess_ctx() {
        for (void* q : allocs) cudaFree(q);
    }
};

namespace {

constexpr int kBiasChunk = 1024;  // pixels per bias-gradient partial

ConvGeom geom(const smm_guess_ctx* c, int l, int B) {
    ConvGeom g = c->L[l];
    g.B = B;
    return g;
}

// pixel splits of a weight-gradient pass: about kWgradBlocks CTAs in total, chunks a multiple of the step
void weight_splits(long long K, long long tiles, int* splits, int* kchunk) {
    long long want = std::max(1LL, (kWgradBlocks + tiles - 1) / tiles);
    want = std::min(want, std::max(1LL, (K + kBK - 1) / kBK));
    long long ch = (K + want - 1) / want;
    ch = std::max<long long>(kBK, (ch + kBK - 1) / kBK * kBK);
    *kchunk = (int)ch;
    *splits = (int)std::max(1LL, (K + ch - 1) / ch);
}

// taps of a strided layer that reach an output pixel from the input pixels of parity (py, px)
int class_taps(const ConvGeom& g, int py, int px, int* tapk) {
    int n = 0;
    for (int ky = 0; ky < g.ksz; ++ky)
        for (int kx = 0; kx < g.ksz; ++kx)
            if (((py + g.pad - ky) % g.stride + g.stride) % g.stride == 0 &&
                ((px + g.pad - kx) % g.stride + g.stride) % g.stride == 0)
                tapk[n++] = ky * g.ksz + kx;
    return n;
}

void launch_fwd(smm_guess g, int l, int B, const __nv_bfloat16* ia, const __nv_bfloat16* ib, int relu,
                __nv_bfloat16* out_bf, float* out_nchw) {
    GemmArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = geom(g, l, B);
    a.M = B * a.g.Hout * a.g.Wout;
    a.N = a.g.Np;
    a.K = a.g.taps * a.g.Kc;
    a.in_a = ia;
    a.in_b = ib;
    a.wt = g->wf[l];
    a.bias = g->p + g->b_off[l];
    a.relu = relu;
    a.out_bf = out_bf;
    a.out_nchw = out_nchw;
    a.wt_ld = a.K;
    dim3 grid((a.M + kBM - 1) / kBM, (a.N + kBN - 1) / kBN);
    conv_gemm_kernel<kFwd><<<grid, kGemmThreads, 0, g->stream>>>(a);
}

void launch_bwd_data(smm_guess g, int l, int B, const __nv_bfloat16* gout, GradPart p0, GradPart p1) {
    GemmArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = geom(g, l, B);
    a.M = B * a.g.Hin * a.g.Win;
    a.N = a.g.Kc;
    a.K = a.g.taps * a.g.Np;
    a.gout = gout;
    a.wt = g->wb[l];
    a.wt_ld = a.K;
    a.part[0] = p0;
    a.part[1] = p1;
    if (a.g.stride == 1) {
        dim3 grid((a.M + kBM - 1) / kBM, (a.N + kBN - 1) / kBN);
        conv_gemm_kernel<kBwdData><<<grid, kGemmThreads, 0, g->stream>>>(a);
        return;
    }
    // strided: one launch per parity class of the input pixels, over the taps that reach an output pixel
    a.cls = 1;
    a.M = B * (a.g.Hin / a.g.stride) * (a.g.Win / a.g.stride);
    for (int py = 0; py < a.g.stride; ++py)
        for (int px = 0; px < a.g.stride; ++px) {
            a.py = py;
            a.px = px;
            a.ntap = class_taps(a.g, py, px, a.tapk);
            a.K = a.ntap * a.g.Np;
            dim3 grid((a.M + kBM - 1) / kBM, (a.N + kBN - 1) / kBN);
            conv_gemm_kernel<kBwdData><<<grid, kGemmThreads, 0, g->stream>>>(a);
        }
}

void launch_bwd_weight(smm_guess g, int l, int B, const __nv_bfloat16* ia, const __nv_bfloat16* ib,
                       const __nv_bfloat16* gout) {
    GemmArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = geom(g, l, B);
    a.M = a.g.Np;
    a.N = a.g.taps * a.g.Kc;
    a.K = B * a.g.Hout * a.g.Wout;
    a.in_a = ia;
    a.in_b = ib;
    a.gout = gout;
    a.wpart = g->wpart;
    const long long tiles = (long long)((a.M + kBM - 1) / kBM) * ((a.N + kBN - 1) / kBN);
    int splits = 1;
    weight_splits(a.K, tiles, &splits, &a.kchunk);
    dim3 grid((a.M + kBM - 1) / kBM, (a.N + kBN - 1) / kBN, splits);
    conv_gemm_kernel<kBwdWeight><<<grid, kGemmThreads, 0, g->stream>>>(a);
    const int bsplits = (a.K + kBiasChunk - 1) / kBiasChunk;
    bias_partial_kernel<<<dim3((a.g.Np + 63) / 64, bsplits), 256, 0, g->stream>>>(a.K, a.g.Np, kBiasChunk, gout,
                                                                                    g->bpart);
    const long long nw = (long long)a.g.cout * (a.g.ca + a.g.cb) * a.g.taps;
    grad_reduce_kernel<<<blocks(nw + a.g.cout), 256, 0, g->stream>>>(a.g, splits, g->wpart, bsplits, g->bpart,
                                                                     g->g + g->w_off[l], g->g + g->b_off[l]);
}

void repack_all(smm_guess g) {
    for (int l = 0; l < 6; ++l) {
        const ConvGeom& d = g->L[l];
        const long long tot = (long long)d.Np * d.taps * d.Kc;
        repack_kernel<<<blocks(tot), 256, 0, g->stream>>>(d, g->p + g->w_off[l], g->wf[l], g->wb[l]);
    }
}

smm_status guess_forward(smm_guess g, int B, const float* in) {
    const int H = g->H, W = g->W, H2 = H / 2, W2 = W / 2;
    cudaStream_t s = g->stream;
    pack_input_kernel<<<blocks((long long)B * H * W * 16), 256, 0, s>>>(B, H, W, in, g->x);
    launch_fwd(g, 0, B, g->x, nullptr, 1, g->a1, nullptr);
    launch_fwd(g, 1, B, g->a1, nullptr, 1, g->a2, nullptr);
    launch_fwd(g, 2, B, g->a2, nullptr, 1, g->a3, nullptr);
    upsample_kernel<<<blocks((long long)B * H * W * (g->P2 / 8)), 256, 0, s>>>(B, H2, W2, g->P2, g->a3, g->u3);
    launch_fwd(g, 3, B, g->u3, nullptr, 1, g->a4, nullptr);
    launch_fwd(g, 4, B, g->a4, g->a1, 1, g->a5, nullptr);
    launch_fwd(g, 5, B, g->a5, nullptr, 0, nullptr, g->y);
    if (cudaGetLastError() != cudaSuccess) return fail(SMM_ERR_CUDA, "guess forward launch failed");
    return SMM_OK;
}

// gradients of the mean squared error into g->g (parameters); loss to host
smm_status guess_backward(smm_guess g, int B, const float* target, float* loss) {
    const int H = g->H, W = g->W, H2 = H / 2, W2 = W / 2;
    cudaStream_t s = g->stream;
    const long long ny = (long long)B * g->nout * H * W;
    mse_kernel<<<256, 256, 0, s>>>(B, g->nout, H * W, g->Po, g->y, target, g->gy, g->part);
    const GradPart none{nullptr, nullptr, nullptr, nullptr, 0};
    // y = conv1x1(a5)
    launch_bwd_weight(g, 5, B, g->a5, nullptr, g->gy);
    launch_bwd_data(g, 5, B, g->gy, GradPart{g->a5, nullptr, g->g5, nullptr, g->P1}, none);
    // a5 = relu(conv([a4, a1]))
    launch_bwd_weight(g, 4, B, g->a4, g->a1, g->g5);
    launch_bwd_data(g, 4, B, g->g5, GradPart{g->a4, nullptr, g->g4, nullptr, g->P1},
                    GradPart{g->a1, nullptr, nullptr, g->g1s, g->P1});
    // a4 = relu(conv(u3)), u3 = up2(a3)
    launch_bwd_weight(g, 3, B, g->u3, nullptr, g->g4);
    launch_bwd_data(g, 3, B, g->g4, GradPart{nullptr, nullptr, nullptr, g->gu, g->P2}, none);
    upsample_bwd_kernel<<<blocks((long long)B * H2 * W2 * g->P2), 256, 0, s>>>(B, H2, W2, g->P2, g->gu, g->a3, g->g3);
    // a3 = relu(conv(a2))
    launch_bwd_weight(g, 2, B, g->a2, nullptr, g->g3);
    launch_bwd_data(g, 2, B, g->g3, GradPart{g->a2, nullptr, g->g2, nullptr, g->P2}, none);
    // a2 = relu(conv_s2(a1)); a1's gradient = main path + skip path
    launch_bwd_weight(g, 1, B, g->a1, nullptr, g->g2);
    launch_bwd_data(g, 1, B, g->g2, GradPart{g->a1, g->g1s, g->g1, nullptr, g->P1}, none);
    // a1 = relu(conv(x))
    launch_bwd_weight(g, 0, B, g->x, nullptr, g->g1);
    std::vector<float> part(256);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(part.data(), g->part, 256 * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SMM_ERR_CUDA, "guess backward failed");
    double sum = 0.0;
    for (float v : part) sum += v;
    if (loss) *loss = (float)(sum / (double)ny);
    return SMM_OK;
}

}  // namespace

extern "C" {

smm_status smm_guess_create(int32_t height, int32_t width, int32_t n_out, int32_t c1, int32_t c2, int32_t max_batch,
                            uint64_t seed, void* cuda_stream, smm_guess* out) {
    if (!out || height < 2 || width < 2 || (height & 1) || (width & 1) || n_out < 1 || n_out > 1024 || max_batch < 1 ||
        c1 < 1 || c1 > 1024 || c2 < 1 || c2 > 1024)
        return fail(SMM_ERR_INVALID_ARG,
                    "smm_guess_create: bad sizes (height and width even, 1 <= n_out, c1, c2 <= 1024)");
    const long long pix = (long long)max_batch * height * width;
    if (pix * pad16(c1 > c2 ? c1 : c2) > (1LL << 31) || pix > (1LL << 30))
        return fail(SMM_ERR_INVALID_ARG, "smm_guess_create: max_batch x height x width x width of a layer too large");
    *out = nullptr;
    auto* g = new smm_guess_ctx();
    auto bail = [&](smm_status st, const std::string& msg) {
        delete g;
        return fail(st, msg);
    };
    g->H = height; g->W = width; g->nout = n_out; g->maxb = max_batch; g->c1 = c1; g->c2 = c2;
    g->P1 = pad16(c1); g->P2 = pad16(c2); g->Po = pad16(n_out);
    g->stream = (cudaStream_t)cuda_stream;
    const int H = height, W = width, H2 = H / 2, W2 = W / 2;
    // per layer: input size, output size, kernel, stride, parts (real, padded), cout
    const int spec[6][11] = {{H, W, H, W, 3, 1, kIn, 16, 0, 0, c1},
                             {H, W, H2, W2, 3, 2, c1, g->P1, 0, 0, c2},
                             {H2, W2, H2, W2, 3, 1, c2, g->P2, 0, 0, c2},
                             {H, W, H, W, 3, 1, c2, g->P2, 0, 0, c1},
                             {H, W, H, W, 3, 1, c1, g->P1, c1, g->P1, c1},
                             {H, W, H, W, 1, 1, c1, g->P1, 0, 0, n_out}};
    size_t off = 0;
    for (int l = 0; l < 6; ++l) {
        ConvGeom& d = g->L[l];
        const int* s = spec[l];
        d.B = 0; d.Hin = s[0]; d.Win = s[1]; d.Hout = s[2]; d.Wout = s[3];
        d.ksz = s[4]; d.stride = s[5]; d.pad = s[4] / 2; d.taps = s[4] * s[4];
        d.ca = s[6]; d.Ka = s[7]; d.cb = s[8]; d.Kb = s[9]; d.Kc = d.Ka + d.Kb;
        d.cout = s[10]; d.Np = pad16(d.cout);
        g->w_off[l] = off;
        off += (size_t)d.cout * (d.ca + d.cb) * d.taps;
        g->b_off[l] = off;
        off += d.cout;
    }
    g->nparam = off;
    // He-uniform initialization from a seeded generator, zero biases
    std::vector<float> host(off, 0.0f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 6; ++l) {
        const ConvGeom& d = g->L[l];
        const int fan_in = (d.ca + d.cb) * d.taps;
        const float a = std::sqrt(6.0f / (float)fan_in) * (l == 5 ? 0.5f : 1.0f);
        std::uniform_real_distribution<float> U(-a, a);
        for (size_t i = g->w_off[l]; i < g->b_off[l]; ++i) host[i] = U(rng);
    }
    // split partials of the weight and bias gradients at the largest batch
    size_t wmax = 1, bmax = 1;
    for (int l = 0; l < 6; ++l) {
        const ConvGeom& d = g->L[l];
        const long long K = pix / ((long long)(H / d.Hout) * (W / d.Wout)), N = (long long)d.taps * d.Kc;
        const long long tiles = (long long)((d.Np + kBM - 1) / kBM) * ((N + kBN - 1) / kBN);
        // weight_splits never gives more splits than min(ceil(kWgradBlocks / tiles), ceil(K / kBK)), which is
        // largest at the largest batch
        const long long bound =
            std::max(1LL, std::min((kWgradBlocks + tiles - 1) / tiles, (K + kBK - 1) / kBK));
        wmax = std::max(wmax, (size_t)bound * (size_t)d.Np * (size_t)N);
        bmax = std::max(bmax, (size_t)((K + kBiasChunk - 1) / kBiasChunk) * d.Np);
    }
    const size_t HW = (size_t)H * W, B = max_batch;
    g->p = g->alloc<float>(off); g->m = g->alloc<float>(off); g->v = g->alloc<float>(off); g->g = g->alloc<float>(off);
    for (int l = 0; l < 6; ++l) {
        const ConvGeom& d = g->L[l];
        g->wf[l] = g->alloc<__nv_bfloat16>((size_t)d.Np * d.taps * d.Kc);
        g->wb[l] = g->alloc<__nv_bfloat16>((size_t)d.Np * d.taps * d.Kc);
    }
    g->x = g->alloc<__nv_bfloat16>(B * HW * 16);
    g->a1 = g->alloc<__nv_bfloat16>(B * HW * g->P1);
    g->a2 = g->alloc<__nv_bfloat16>(B * HW / 4 * g->P2);
    g->a3 = g->alloc<__nv_bfloat16>(B * HW / 4 * g->P2);
    g->u3 = g->alloc<__nv_bfloat16>(B * HW * g->P2);
    g->a4 = g->alloc<__nv_bfloat16>(B * HW * g->P1);
    g->a5 = g->alloc<__nv_bfloat16>(B * HW * g->P1);
    g->y = g->alloc<float>(B * HW * n_out);
    g->gy = g->alloc<__nv_bfloat16>(B * HW * g->Po);
    g->g5 = g->alloc<__nv_bfloat16>(B * HW * g->P1);
    g->g4 = g->alloc<__nv_bfloat16>(B * HW * g->P1);
    g->g1s = g->alloc<float>(B * HW * g->P1);
    g->gu = g->alloc<float>(B * HW * g->P2);
    g->g3 = g->alloc<__nv_bfloat16>(B * HW / 4 * g->P2);
    g->g2 = g->alloc<__nv_bfloat16>(B * HW / 4 * g->P2);
    g->g1 = g->alloc<__nv_bfloat16>(B * HW * g->P1);
    g->wpart = g->alloc<float>(wmax);
    g->bpart = g->alloc<float>(bmax);
    g->part = g->alloc<float>(256);
    if (g->alloc_failed) return bail(SMM_ERR_OOM, "smm_guess_create: device allocation failed");
    if (cudaMemcpy(g->p, host.data(), off * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(g->m, 0, off * sizeof(float)) != cudaSuccess || cudaMemset(g->v, 0, off * sizeof(float)) != cudaSuccess ||
        cudaMemset(g->gy, 0, B * HW * g->Po * sizeof(__nv_bfloat16)) != cudaSuccess)
        return bail(SMM_ERR_CUDA, "smm_guess_create: upload failed");
    repack_all(g);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return bail(SMM_ERR_CUDA, "smm_guess_create: init failed");
    *out = g;
    return SMM_OK;
}

smm_status smm_guess_num_params(smm_guess g, int64_t* n) {
    if (!g || !n) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    *n = (int64_t)g->nparam;
    return SMM_OK;
}

smm_status smm_guess_forward(smm_guess g, int32_t batch, const float* in_dev, float* out_dev) {
    if (!g || !in_dev || !out_dev || batch < 1 || batch > g->maxb) return fail(SMM_ERR_INVALID_ARG, "bad argument");
    smm_status st = guess_forward(g, batch, in_dev);
    if (st != SMM_OK) return st;
    if (cudaMemcpyAsync(out_dev, g->y, (size_t)batch * g->nout * g->H * g->W * sizeof(float), cudaMemcpyDeviceToDevice,
                        g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
        return fail(SMM_ERR_CUDA, "guess forward failed");
    return SMM_OK;
}

smm_status smm_guess_gradients(smm_guess g, int32_t batch, const float* in_dev, const float* target_dev,
                               float* grad_host, float* loss_host) {
    if (!g || !in_dev || !target_dev || batch < 1 || batch > g->maxb) return fail(SMM_ERR_INVALID_ARG, "bad argument");
    smm_status st = guess_forward(g, batch, in_dev);
    if (st != SMM_OK) return st;
    st = guess_backward(g, batch, target_dev, loss_host);
    if (st != SMM_OK) return st;
    if (grad_host && cudaMemcpy(grad_host, g->g, g->nparam * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(SMM_ERR_CUDA, "gradient copy failed");
    return SMM_OK;
}

smm_status smm_guess_train_step(smm_guess g, int32_t batch, const float* in_dev, const float* target_dev, float lr,
                                float* loss_host) {
    if (!g || !in_dev || !target_dev || batch < 1 || batch > g->maxb || !(lr > 0))
        return fail(SMM_ERR_INVALID_ARG, "bad argument");
    smm_status st = guess_forward(g, batch, in_dev);
    if (st != SMM_OK) return st;
    st = guess_backward(g, batch, target_dev, loss_host);
    if (st != SMM_OK) return st;
    g->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)g->step), c2 = 1.0f - std::pow(b2, (float)g->step);
    adam_kernel<<<blocks((long long)g->nparam), 256, 0, g->stream>>>((long long)g->nparam, g->p, g->m, g->v, g->g, lr,
                                                                      b1, b2, c1, c2, 1e-8f);
    repack_all(g);
    if (cudaGetLastError() != cudaSuccess) return fail(SMM_ERR_CUDA, "adam launch failed");
    return SMM_OK;
}

smm_status smm_guess_get_params(smm_guess g, float* host) {
    if (!g || !host) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    if (cudaMemcpy(host, g->p, g->nparam * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(SMM_ERR_CUDA, "parameter copy failed");
    return SMM_OK;
}

smm_status smm_guess_set_params(smm_guess g, const float* host) {
    if (!g || !host) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    if (cudaMemcpy(g->p, host, g->nparam * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(SMM_ERR_CUDA, "parameter copy failed");
    repack_all(g);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return fail(SMM_ERR_CUDA, "parameter upload failed");
    return SMM_OK;
}

smm_status smm_guess_destroy(smm_guess g) {
    if (!g) return SMM_OK;
    cudaStreamSynchronize(g->stream);
    delete g;
    return SMM_OK;
}

}  // extern "C"

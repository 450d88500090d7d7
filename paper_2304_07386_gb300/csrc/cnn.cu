// Learned initial guess: a small convolutional encoder-decoder on the element
// grid, trained and run with this file's own kernels (BF16 weights and
// activations, FP32 accumulation, FP32 master weights and Adam state).
//
// Network (all convolutions 3x3, zero padding 1, except the last 1x1):
//   a1 = relu(conv(x, 3 -> C1))                 full resolution
//   a2 = relu(conv_stride2(a1, C1 -> C2))       half resolution
//   a3 = relu(conv(a2, C2 -> C2))               half resolution
//   a4 = relu(conv(up2(a3), C2 -> C1))          full resolution (nearest up-sampling)
//   a5 = relu(conv([a4, a1], 2 C1 -> C1))       skip connection by channel concatenation
//   y  = conv1x1(a5, C1 -> n_out)
// with C1 = 24, C2 = 32.  Loss: mean squared error against the targets.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/smm.h"
#include "kernels.cuh"

namespace {

constexpr int kC1 = 24, kC2 = 32, kIn = 3;

smm_status fail(smm_status s, const std::string& msg) {
    smm::set_last_error(msg.c_str());
    return s;
}

struct ConvDesc {
    int cin1, cin2, cout, k, stride;  // input channels split over two tensors (concatenation)
    size_t w_off, b_off;              // offsets into the parameter vector
};

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// out[b][co][y][x] = bias[co] + sum w[co][ci][ky][kx] in[b][ci][y*s+ky-pad][x*s+kx-pad]
__global__ void conv_fwd_kernel(int B, int Hin, int Win, int Hout, int Wout, ConvDesc d,
                                const __nv_bfloat16* __restrict__ in1, const __nv_bfloat16* __restrict__ in2,
                                const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias, int relu,
                                __nv_bfloat16* __restrict__ out_bf, float* __restrict__ out_f) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)B * d.cout * Hout * Wout;
    if (t >= tot) return;
    const int x = (int)(t % Wout), y = (int)((t / Wout) % Hout), co = (int)((t / ((long long)Wout * Hout)) % d.cout);
    const int b = (int)(t / ((long long)Wout * Hout * d.cout));
    const int pad = d.k / 2, cin = d.cin1 + d.cin2;
    float acc = bias[co];
    for (int ci = 0; ci < cin; ++ci) {
        const __nv_bfloat16* src = ci < d.cin1 ? in1 + ((size_t)b * d.cin1 + ci) * Hin * Win
                                              : in2 + ((size_t)b * d.cin2 + (ci - d.cin1)) * Hin * Win;
        const __nv_bfloat16* wk = w + ((size_t)co * cin + ci) * d.k * d.k;
        for (int ky = 0; ky < d.k; ++ky) {
            const int iy = y * d.stride + ky - pad;
            if (iy < 0 || iy >= Hin) continue;
            for (int kx = 0; kx < d.k; ++kx) {
                const int ix = x * d.stride + kx - pad;
                if (ix < 0 || ix >= Win) continue;
                acc = fmaf(bf(wk[ky * d.k + kx]), bf(src[(size_t)iy * Win + ix]), acc);
            }
        }
    }
    if (relu) acc = fmaxf(acc, 0.0f);
    if (out_bf) out_bf[t] = __float2bfloat16(acc);
    if (out_f) out_f[t] = acc;
}

// gin[b][ci][iy][ix] = sum_{co,ky,kx} w[co][ci][ky][kx] gout[b][co][oy][ox], iy = oy*s+ky-pad;
// ci ranges over the part [c0, c0 + cn) of the concatenated input; gin may be scaled by
// the ReLU mask of that input (act != nullptr)
__global__ void conv_bwd_data_kernel(int B, int Hin, int Win, int Hout, int Wout, ConvDesc d, int c0, int cn,
                                     const __nv_bfloat16* __restrict__ w, const float* __restrict__ gout,
                                     const __nv_bfloat16* __restrict__ act, float* __restrict__ gin) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)B * cn * Hin * Win;
    if (t >= tot) return;
    const int ix = (int)(t % Win), iy = (int)((t / Win) % Hin), cl = (int)((t / ((long long)Win * Hin)) % cn);
    const int b = (int)(t / ((long long)Win * Hin * cn));
    const int ci = c0 + cl, cin = d.cin1 + d.cin2, pad = d.k / 2;
    float acc = 0.0f;
    for (int co = 0; co < d.cout; ++co) {
        const float* go = gout + ((size_t)b * d.cout + co) * Hout * Wout;
        const __nv_bfloat16* wk = w + ((size_t)co * cin + ci) * d.k * d.k;
        for (int ky = 0; ky < d.k; ++ky) {
            const int ny = iy + pad - ky;
            if (ny < 0 || ny % d.stride) continue;
            const int oy = ny / d.stride;
            if (oy >= Hout) continue;
            for (int kx = 0; kx < d.k; ++kx) {
                const int nx = ix + pad - kx;
                if (nx < 0 || nx % d.stride) continue;
                const int ox = nx / d.stride;
                if (ox >= Wout) continue;
                acc = fmaf(bf(wk[ky * d.k + kx]), go[(size_t)oy * Wout + ox], acc);
            }
        }
    }
    if (act && !(bf(act[t]) > 0.0f)) acc = 0.0f;
    gin[t] = acc;
}

// gw[co][ci][ky][kx] = sum_{b,y,x} gout[b][co][y][x] in[b][ci][y*s+ky-pad][x*s+kx-pad]; one block per weight;
// blocks with index >= nweights compute the bias gradients
__global__ void conv_bwd_weight_kernel(int B, int Hin, int Win, int Hout, int Wout, ConvDesc d,
                                       const __nv_bfloat16* __restrict__ in1, const __nv_bfloat16* __restrict__ in2,
                                       const float* __restrict__ gout, float* __restrict__ gw, float* __restrict__ gb) {
    __shared__ float sh[256];
    const int cin = d.cin1 + d.cin2, kk = d.k * d.k;
    const int nw = d.cout * cin * kk;
    const int widx = blockIdx.x;
    const int n = B * Hout * Wout, pad = d.k / 2;
    float acc = 0.0f;
    if (widx < nw) {
        const int kx = widx % d.k, ky = (widx / d.k) % d.k, ci = (widx / kk) % cin, co = widx / (kk * cin);
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int x = t % Wout, y = (t / Wout) % Hout, b = t / (Wout * Hout);
            const int iy = y * d.stride + ky - pad, ix = x * d.stride + kx - pad;
            if (iy < 0 || iy >= Hin || ix < 0 || ix >= Win) continue;
            const __nv_bfloat16* src = ci < d.cin1 ? in1 + ((size_t)b * d.cin1 + ci) * Hin * Win
                                                  : in2 + ((size_t)b * d.cin2 + (ci - d.cin1)) * Hin * Win;
            acc = fmaf(gout[((size_t)b * d.cout + co) * Hout * Wout + (size_t)y * Wout + x], bf(src[(size_t)iy * Win + ix]),
                       acc);
        }
    } else {
        const int co = widx - nw;
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int x = t % Wout, y = (t / Wout) % Hout, b = t / (Wout * Hout);
            acc += gout[((size_t)b * d.cout + co) * Hout * Wout + (size_t)y * Wout + x];
        }
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (widx < nw) gw[widx] = sh[0];
        else gb[widx - nw] = sh[0];
    }
}

__global__ void upsample_kernel(int B, int C, int H, int W, const __nv_bfloat16* __restrict__ in,
                                __nv_bfloat16* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)B * C * 2 * H * 2 * W;
    if (t >= tot) return;
    const int x = (int)(t % (2 * W)), y = (int)((t / (2 * W)) % (2 * H));
    const long long bc = t / (4LL * H * W);
    out[t] = in[bc * H * W + (size_t)(y / 2) * W + x / 2];
}

// g_in[b][c][y][x] = relu'(a) * sum of the four up-sampled gradients
__global__ void upsample_bwd_kernel(int B, int C, int H, int W, const float* __restrict__ gup,
                                    const __nv_bfloat16* __restrict__ act, float* __restrict__ gin) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)B * C * H * W;
    if (t >= tot) return;
    const int x = (int)(t % W), y = (int)((t / W) % H);
    const long long bc = t / ((long long)H * W);
    const float* g = gup + bc * 4LL * H * W;
    float s = g[(size_t)(2 * y) * 2 * W + 2 * x] + g[(size_t)(2 * y) * 2 * W + 2 * x + 1] +
              g[(size_t)(2 * y + 1) * 2 * W + 2 * x] + g[(size_t)(2 * y + 1) * 2 * W + 2 * x + 1];
    if (!(bf(act[t]) > 0.0f)) s = 0.0f;
    gin[t] = s;
}

__global__ void add_f32_kernel(long long n, float* __restrict__ a, const float* __restrict__ b) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) a[t] += b[t];
}

__global__ void to_bf16_kernel(long long n, const float* __restrict__ in, __nv_bfloat16* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = __float2bfloat16(in[t]);
}

// d = 2 (y - target) / count ; partial sums of (y - target)^2 per block
__global__ void mse_kernel(long long n, const float* __restrict__ y, const float* __restrict__ tgt,
                           float* __restrict__ g, float* __restrict__ part) {
    __shared__ float sh[256];
    float acc = 0.0f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float r = y[t] - tgt[t];
        g[t] = 2.0f * r / (float)n;
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

__global__ void adam_kernel(long long n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, __nv_bfloat16* __restrict__ pbf, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gi = g[t];
    const float mi = b1 * m[t] + (1.0f - b1) * gi;
    const float vi = b2 * v[t] + (1.0f - b2) * gi * gi;
    m[t] = mi;
    v[t] = vi;
    const float pi = p[t] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[t] = pi;
    pbf[t] = __float2bfloat16(pi);
}

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct smm_guess_ctx {
    int H = 0, W = 0, nout = 0, maxb = 0;
    cudaStream_t stream = nullptr;
    ConvDesc L[6];
    size_t nparam = 0;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // FP32 master, Adam moments, gradients
    __nv_bfloat16* pb = nullptr;                                       // BF16 copy used by the kernels
    long long step = 0;
    // activations (BF16) and gradients (FP32) for up to maxb samples
    __nv_bfloat16 *x = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *u3 = nullptr, *a4 = nullptr, *a5 = nullptr;
    float *y = nullptr, *gy = nullptr, *g5 = nullptr, *g4a = nullptr, *g1 = nullptr, *gu = nullptr, *g3 = nullptr,
          *g2 = nullptr, *g1b = nullptr, *part = nullptr;
    std::vector<void*> allocs;
    template <class T>
    T* alloc(size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, (n ? n : 1) * sizeof(T)) != cudaSuccess) return nullptr;
        allocs.push_back(q);
        return (T*)q;
    }
    ~smm_guess_ctx() {
        for (void* q : allocs) cudaFree(q);
    }
};

namespace {

smm_status guess_forward(smm_guess g, int B, const float* in) {
    const int H = g->H, W = g->W, H2 = H / 2, W2 = W / 2;
    const long long nin = (long long)B * kIn * H * W;
    cudaStream_t s = g->stream;
    to_bf16_kernel<<<blocks(nin), 256, 0, s>>>(nin, in, g->x);
    const __nv_bfloat16* P = g->pb;
    const float* Pf = g->p;
    auto conv = [&](int l, int Hin, int Win, int Hout, int Wout, const __nv_bfloat16* i1, const __nv_bfloat16* i2,
                    int relu, __nv_bfloat16* ob, float* of) {
        const ConvDesc& d = g->L[l];
        const long long tot = (long long)B * d.cout * Hout * Wout;
        conv_fwd_kernel<<<blocks(tot), 256, 0, s>>>(B, Hin, Win, Hout, Wout, d, i1, i2, P + d.w_off, Pf + d.b_off, relu,
                                                     ob, of);
    };
    conv(0, H, W, H, W, g->x, nullptr, 1, g->a1, nullptr);
    conv(1, H, W, H2, W2, g->a1, nullptr, 1, g->a2, nullptr);
    conv(2, H2, W2, H2, W2, g->a2, nullptr, 1, g->a3, nullptr);
    const long long nup = (long long)B * kC2 * H * W;
    upsample_kernel<<<blocks(nup), 256, 0, s>>>(B, kC2, H2, W2, g->a3, g->u3);
    conv(3, H, W, H, W, g->u3, nullptr, 1, g->a4, nullptr);
    conv(4, H, W, H, W, g->a4, g->a1, 1, g->a5, nullptr);
    conv(5, H, W, H, W, g->a5, nullptr, 0, nullptr, g->y);
    if (cudaGetLastError() != cudaSuccess) return fail(SMM_ERR_CUDA, "guess forward launch failed");
    return SMM_OK;
}

// gradients of the mean squared error into g->g (parameters); loss to host
smm_status guess_backward(smm_guess g, int B, const float* target, float* loss) {
    const int H = g->H, W = g->W, H2 = H / 2, W2 = W / 2;
    cudaStream_t s = g->stream;
    const long long ny = (long long)B * g->nout * H * W;
    mse_kernel<<<256, 256, 0, s>>>(ny, g->y, target, g->gy, g->part);
    const __nv_bfloat16* P = g->pb;
    auto bw = [&](int l, int Hin, int Win, int Hout, int Wout, const __nv_bfloat16* i1, const __nv_bfloat16* i2,
                  const float* gout) {
        const ConvDesc& d = g->L[l];
        const int nw = d.cout * (d.cin1 + d.cin2) * d.k * d.k;
        conv_bwd_weight_kernel<<<nw + d.cout, 256, 0, s>>>(B, Hin, Win, Hout, Wout, d, i1, i2, gout, g->g + d.w_off,
                                                            g->g + d.b_off);
    };
    auto bd = [&](int l, int Hin, int Win, int Hout, int Wout, int c0, int cn, const float* gout,
                  const __nv_bfloat16* act, float* gin) {
        const ConvDesc& d = g->L[l];
        const long long tot = (long long)B * cn * Hin * Win;
        conv_bwd_data_kernel<<<blocks(tot), 256, 0, s>>>(B, Hin, Win, Hout, Wout, d, c0, cn, P + d.w_off, gout, act,
                                                          gin);
    };
    // y = conv1x1(a5)
    bw(5, H, W, H, W, g->a5, nullptr, g->gy);
    bd(5, H, W, H, W, 0, kC1, g->gy, g->a5, g->g5);                 // g5 = dL/d(pre-activation of a5)
    // a5 = relu(conv([a4, a1]))
    bw(4, H, W, H, W, g->a4, g->a1, g->g5);
    bd(4, H, W, H, W, 0, kC1, g->g5, g->a4, g->g4a);                // through a4's ReLU
    bd(4, H, W, H, W, kC1, kC1, g->g5, g->a1, g->g1b);              // skip path into a1 (ReLU of a1)
    // a4 = relu(conv(u3))
    bw(3, H, W, H, W, g->u3, nullptr, g->g4a);
    bd(3, H, W, H, W, 0, kC2, g->g4a, nullptr, g->gu);              // gradient w.r.t. u3
    const long long n3 = (long long)B * kC2 * H2 * W2;
    upsample_bwd_kernel<<<blocks(n3), 256, 0, s>>>(B, kC2, H2, W2, g->gu, g->a3, g->g3);
    // a3 = relu(conv(a2))
    bw(2, H2, W2, H2, W2, g->a2, nullptr, g->g3);
    bd(2, H2, W2, H2, W2, 0, kC2, g->g3, g->a2, g->g2);
    // a2 = relu(conv_s2(a1))
    bw(1, H, W, H2, W2, g->a1, nullptr, g->g2);
    bd(1, H, W, H2, W2, 0, kC1, g->g2, g->a1, g->g1);
    // a1 gradient = main path + skip path; a1 = relu(conv(x))
    {
        const long long n1 = (long long)B * kC1 * H * W;
        add_f32_kernel<<<blocks(n1), 256, 0, s>>>(n1, g->g1, g->g1b);
    }
    bw(0, H, W, H, W, g->x, nullptr, g->g1);
    std::vector<float> part(256);
    if (cudaMemcpyAsync(part.data(), g->part, 256 * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SMM_ERR_CUDA, "guess backward failed");
    double sum = 0.0;
    for (float v : part) sum += v;
    if (loss) *loss = (float)(sum / (double)ny);
    return SMM_OK;
}

}  // namespace

extern "C" {

smm_status smm_guess_create(int32_t height, int32_t width, int32_t n_out, int32_t max_batch, uint64_t seed,
                            void* cuda_stream, smm_guess* out) {
    if (!out || height < 2 || width < 2 || (height & 1) || (width & 1) || n_out < 1 || max_batch < 1)
        return fail(SMM_ERR_INVALID_ARG, "smm_guess_create: bad sizes (height and width must be even)");
    *out = nullptr;
    auto* g = new smm_guess_ctx();
    auto bail = [&](smm_status st, const std::string& m) { delete g; return fail(st, m); };
    g->H = height; g->W = width; g->nout = n_out; g->maxb = max_batch;
    g->stream = (cudaStream_t)cuda_stream;
    const int spec[6][5] = {{kIn, 0, kC1, 3, 1}, {kC1, 0, kC2, 3, 2}, {kC2, 0, kC2, 3, 1},
                            {kC2, 0, kC1, 3, 1}, {kC1, kC1, kC1, 3, 1}, {kC1, 0, n_out, 1, 1}};
    size_t off = 0;
    for (int l = 0; l < 6; ++l) {
        ConvDesc& d = g->L[l];
        d.cin1 = spec[l][0]; d.cin2 = spec[l][1]; d.cout = spec[l][2]; d.k = spec[l][3]; d.stride = spec[l][4];
        d.w_off = off;
        off += (size_t)d.cout * (d.cin1 + d.cin2) * d.k * d.k;
        d.b_off = off;
        off += d.cout;
    }
    g->nparam = off;
    // He-uniform initialization from a seeded generator, zero biases
    std::vector<float> host(off, 0.0f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 6; ++l) {
        const ConvDesc& d = g->L[l];
        const int fan_in = (d.cin1 + d.cin2) * d.k * d.k;
        const float a = std::sqrt(6.0f / (float)fan_in) * (l == 5 ? 0.5f : 1.0f);
        std::uniform_real_distribution<float> U(-a, a);
        for (size_t i = d.w_off; i < d.b_off; ++i) host[i] = U(rng);
    }
    const size_t H = height, W = width, B = max_batch;
    g->p = g->alloc<float>(off); g->m = g->alloc<float>(off); g->v = g->alloc<float>(off); g->g = g->alloc<float>(off);
    g->pb = g->alloc<__nv_bfloat16>(off);
    g->x = g->alloc<__nv_bfloat16>(B * kIn * H * W);
    g->a1 = g->alloc<__nv_bfloat16>(B * kC1 * H * W);
    g->a2 = g->alloc<__nv_bfloat16>(B * kC2 * H * W / 4);
    g->a3 = g->alloc<__nv_bfloat16>(B * kC2 * H * W / 4);
    g->u3 = g->alloc<__nv_bfloat16>(B * kC2 * H * W);
    g->a4 = g->alloc<__nv_bfloat16>(B * kC1 * H * W);
    g->a5 = g->alloc<__nv_bfloat16>(B * kC1 * H * W);
    g->y = g->alloc<float>(B * n_out * H * W);
    g->gy = g->alloc<float>(B * n_out * H * W);
    g->g5 = g->alloc<float>(B * kC1 * H * W);
    g->g4a = g->alloc<float>(B * kC1 * H * W);
    g->g1 = g->alloc<float>(B * kC1 * H * W);
    g->g1b = g->alloc<float>(B * kC1 * H * W);
    g->gu = g->alloc<float>(B * kC2 * H * W);
    g->g3 = g->alloc<float>(B * kC2 * H * W / 4);
    g->g2 = g->alloc<float>(B * kC2 * H * W / 4);
    g->part = g->alloc<float>(256);
    for (void* q : g->allocs)
        if (!q) return bail(SMM_ERR_OOM, "smm_guess_create: device allocation failed");
    if (g->allocs.size() < 22) return bail(SMM_ERR_OOM, "smm_guess_create: device allocation failed");
    if (cudaMemcpy(g->p, host.data(), off * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(g->m, 0, off * sizeof(float)) != cudaSuccess || cudaMemset(g->v, 0, off * sizeof(float)) != cudaSuccess)
        return bail(SMM_ERR_CUDA, "smm_guess_create: upload failed");
    to_bf16_kernel<<<blocks((long long)off), 256, 0, g->stream>>>((long long)off, g->p, g->pb);
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
    adam_kernel<<<blocks((long long)g->nparam), 256, 0, g->stream>>>((long long)g->nparam, g->p, g->m, g->v, g->g, g->pb,
                                                                      lr, b1, b2, c1, c2, 1e-8f);
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
    to_bf16_kernel<<<blocks((long long)g->nparam), 256, 0, g->stream>>>((long long)g->nparam, g->p, g->pb);
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

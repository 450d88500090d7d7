// Device helpers shared by the PCG and multigrid kernels: rows of the IP-SMM
// moment operator with column-major n x n diagonal blocks and face-factored
// neighbour blocks (see FaceOp).  Thread blocks cover whole elements: EPB =
// 256 / n elements of n rows each.
#pragma once

#include "dfloat.cuh"
#include "kernels.cuh"

namespace smm {

template <int N>
struct FaceDims {
    static constexpr int P1 = N == 4 ? 2 : N == 9 ? 3 : N == 16 ? 4 : 5;  // p + 1
    static constexpr int G = 2 * P1;                                      // face data per face
    static constexpr int NG = 4 * G;                                      // face data per element
    static constexpr int EPB = 256 / N;                                   // elements per block
};

// L2 eviction priority of loads (per-load cache policies, nothing global):
// the level-0 FP32 blocks, which every V-cycle step reads again, are loaded
// with evict_last; the FP32-pair operator of the CG product, streamed once per
// iteration, with evict_first, so that it does not push the former out of L2
__device__ __forceinline__ unsigned long long l2_keep() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_stream() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float ld_hint(const float* a, unsigned long long pol) {
    float v;
    asm("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 ld_hint(const float2* a, unsigned long long pol) {
    float2 v;
    asm("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_hint(const double* a, unsigned long long) { return *a; }

// element-local node at face position a, line position t (t = 0 on face f)
template <int P1>
__device__ __forceinline__ int line_node(int f, int a, int t) {
    constexpr int p = P1 - 1;
    switch (f) {
        case 0: return t * P1 + a;
        case 1: return a * P1 + p - t;
        case 2: return (p - t) * P1 + a;
        default: return a * P1 + t;
    }
}

// the line of nodes of element-local face f at face position a: node(t) =
// base + t * stride for line positions t = 0..p (the same nodes as line_node)
template <int P1>
__device__ __forceinline__ void line_of(int f, int a, int& base, int& stride) {
    constexpr int p = P1 - 1;
    base = f == 0 ? a : (f == 1 ? a * P1 + p : (f == 2 ? p * P1 + a : a * P1));
    stride = f == 0 ? P1 : (f == 1 ? -1 : (f == 2 ? -P1 : 1));
}

// shared scratch of one thread block: neighbour face data and coupled face
// data of its S element slots (the EPB elements of a block, or more when a
// thread handles rows of several elements)
template <int N, typename AT, int S = FaceDims<N>::EPB>
struct FaceScratch {
    AT g[S * FaceDims<N>::NG];
    AT w[S * FaceDims<N>::NG];
};

// (A x)_i for row i of element e, in three phases separated by block
// barriers: (1) the neighbours' face data g = E_f2 x_e2 (trace values and
// normal derivatives) into shared scratch, (2) w = C_{e,f} g per face,
// (3) the lift (E_f^T w)_i.  The diagonal block row is added before the lift.
// The phases are separate functions so that a kernel can stage the matrix
// data (the diagonal block and the face couplings) while phase 1 runs.

// phase 1 for the thread of row i of element e (element slot le of the
// block's scratch; le < 0: threadIdx.x / N): face data v = i, i + N, ...
template <int N, typename T, typename AT, typename VT, int S>
__device__ __forceinline__ void face_gather(const FaceOp<T>& op, const VT* __restrict__ x, int e, int i,
                                            FaceScratch<N, AT, S>& sc, int le = -1) {
    using D = FaceDims<N>;
    constexpr int P1 = D::P1, G = D::G, NG = D::NG;
    if (le < 0) le = threadIdx.x / N;
#pragma unroll
    for (int v0 = 0; v0 < NG; v0 += N) {
        const int v = v0 + i;
        if (v < NG) {
            const int f = v / G, r = v - f * G;
            const int e2 = op.nbr[e * 4 + f];
            AT g = 0;
            if (e2 >= 0) {
                const int f2 = op.nface[e * 4 + f];
                int base, stride;
                line_of<P1>(f2, r < P1 ? r : r - P1, base, stride);
                const VT* x2 = x + (size_t)e2 * N + base;
                if (r < P1) {
                    g = (AT)x2[0];
                } else {
#pragma unroll
                    for (int t = 0; t < P1; ++t) g += (AT)op.wd[t] * (AT)x2[t * stride];
                }
            }
            sc.g[le * NG + v] = g;
        }
    }
}

// phase 2: w = C g with Ce the element's four G x G face blocks (column-major)
template <int N, typename CTy, typename AT, int S>
__device__ __forceinline__ void face_couple(const CTy* __restrict__ Ce, const int32_t* __restrict__ nbr, int e, int i,
                                            FaceScratch<N, AT, S>& sc, int le = -1) {
    using D = FaceDims<N>;
    constexpr int G = D::G, NG = D::NG;
    if (le < 0) le = threadIdx.x / N;
#pragma unroll
    for (int v0 = 0; v0 < NG; v0 += N) {
        const int v = v0 + i;
        if (v < NG) {
            const int f = v / G, r = v - f * G;
            AT w = 0;
            if (nbr[e * 4 + f] >= 0) {
                const CTy* C = Ce + (size_t)f * G * G + r;
                const AT* g = sc.g + le * NG + f * G;
                const unsigned long long pol = l2_keep();
#pragma unroll
                for (int c = 0; c < G; ++c) w += (AT)ld_hint(C + c * G, pol) * g[c];
            }
            sc.w[le * NG + v] = w;
        }
    }
}

// phase 3: y + (E_f^T w)_i
template <int N, typename T, typename AT, int S>
__device__ __forceinline__ AT face_lift(const FaceOp<T>& op, int i, AT y, const FaceScratch<N, AT, S>& sc,
                                        int le = -1) {
    using D = FaceDims<N>;
    constexpr int P1 = D::P1, G = D::G, NG = D::NG;
    constexpr int p = P1 - 1;
    if (le < 0) le = threadIdx.x / N;
    const int ix = i % P1, iy = i / P1;
    const AT* w = sc.w + le * NG;
    // (face, face position, line position) of this node for each face
    const int fa[4] = {ix, iy, ix, iy};
    const int ft[4] = {iy, p - ix, p - iy, ix};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        AT c = 0;
#pragma unroll
        for (int t = 0; t < P1; ++t)
            if (t == ft[f]) c = (AT)op.wd[t];
        y += c * w[f * G + P1 + fa[f]];
        if (ft[f] == 0) y += w[f * G + fa[f]];
    }
    return y;
}

// (A x)_i (act: this thread owns a row); every thread of the block must call
// it (two block barriers).  With DIAG false the diagonal block is left out:
// the row of the off-diagonal part alone.
template <int N, typename T, typename AT, typename VT, bool DIAG = true>
__device__ __forceinline__ AT faceop_row(const FaceOp<T>& op, const VT* __restrict__ x, int e, int i, bool act,
                                         FaceScratch<N, AT>& sc) {
    constexpr int G = FaceDims<N>::G;
    AT y = 0;
    if (act) {
        if constexpr (DIAG) {
            const T* Ad = op.AdT + (size_t)e * N * N + i;
            const VT* xe = x + (size_t)e * N;
            const unsigned long long pol = l2_keep();
#pragma unroll
            for (int j = 0; j < N; ++j) y += (AT)ld_hint(Ad + j * N, pol) * (AT)xe[j];
        }
        face_gather<N>(op, x, e, i, sc);
    }
    __syncthreads();
    if (act) face_couple<N>(op.CT + (size_t)e * 4 * G * G, op.nbr, e, i, sc);
    __syncthreads();
    if (act) y = face_lift<N>(op, i, y, sc);
    return y;
}

template <int N, int S = FaceDims<N>::EPB>
struct FaceScratchDF {
    float2 g[S * FaceDims<N>::NG];
    float2 w[S * FaceDims<N>::NG];
};

// the three phases with the operator and x as FP32 pairs, pair arithmetic
// throughout (see dfloat.cuh)
template <int N, int S>
__device__ __forceinline__ void face_gather_df(const FaceOpDF& op, const float2* __restrict__ x, int e, int i,
                                               FaceScratchDF<N, S>& sc, int le = -1) {
    using D = FaceDims<N>;
    constexpr int P1 = D::P1, G = D::G, NG = D::NG;
    if (le < 0) le = threadIdx.x / N;
#pragma unroll
    for (int v0 = 0; v0 < NG; v0 += N) {
        const int v = v0 + i;
        if (v < NG) {
            const int f = v / G, r = v - f * G;
            const int e2 = op.nbr[e * 4 + f];
            float2 g = make_float2(0.0f, 0.0f);
            if (e2 >= 0) {
                const int f2 = op.nface[e * 4 + f];
                int base, stride;
                line_of<P1>(f2, r < P1 ? r : r - P1, base, stride);
                const float2* x2 = x + (size_t)e2 * N + base;
                if (r < P1) {
                    g = x2[0];
                } else {
                    float gs = 0.0f, gc = 0.0f;
#pragma unroll
                    for (int t = 0; t < P1; ++t) {
                        const float2 xv = x2[t * stride];
                        df_acc(gs, gc, op.wd[t].x, op.wd[t].y, xv.x, xv.y);
                    }
                    g = df_norm(gs, gc);
                }
            }
            sc.g[le * NG + v] = g;
        }
    }
}

template <int N, int S>
__device__ __forceinline__ void face_couple_df(const float2* __restrict__ Ce, const int32_t* __restrict__ nbr, int e,
                                               int i, FaceScratchDF<N, S>& sc, int le = -1) {
    using D = FaceDims<N>;
    constexpr int G = D::G, NG = D::NG;
    if (le < 0) le = threadIdx.x / N;
#pragma unroll
    for (int v0 = 0; v0 < NG; v0 += N) {
        const int v = v0 + i;
        if (v < NG) {
            const int f = v / G, r = v - f * G;
            float ws = 0.0f, wc = 0.0f;
            if (nbr[e * 4 + f] >= 0) {
                const float2* C = Ce + (size_t)f * G * G + r;
                const float2* g = sc.g + le * NG + f * G;
                const unsigned long long pol = l2_stream();
#pragma unroll
                for (int c = 0; c < G; ++c) {
                    const float2 cv = ld_hint(C + c * G, pol), gv = g[c];
                    df_acc(ws, wc, cv.x, cv.y, gv.x, gv.y);
                }
            }
            sc.w[le * NG + v] = df_norm(ws, wc);
        }
    }
}

// diagonal block row (Ad: row i of the element's column-major block) into the pair sum (ys, yc)
template <int N>
__device__ __forceinline__ void diag_row_df(const float2* __restrict__ Ad, const float2* __restrict__ xe, float& ys,
                                            float& yc) {
    const unsigned long long pol = l2_stream();
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const float2 a = ld_hint(Ad + j * N, pol), v = xe[j];
        df_acc(ys, yc, a.x, a.y, v.x, v.y);
    }
}

// phase 3 added to the pair sum (ys, yc); the row value in FP64
template <int N, int S>
__device__ __forceinline__ double face_lift_df(const FaceOpDF& op, int i, float ys, float yc,
                                               const FaceScratchDF<N, S>& sc, int le = -1) {
    using D = FaceDims<N>;
    constexpr int P1 = D::P1, G = D::G, NG = D::NG;
    constexpr int p = P1 - 1;
    if (le < 0) le = threadIdx.x / N;
    const int ix = i % P1, iy = i / P1;
    const float2* w = sc.w + le * NG;
    const int fa[4] = {ix, iy, ix, iy};
    const int ft[4] = {iy, p - ix, p - iy, ix};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        float2 cf = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int t = 0; t < P1; ++t)
            if (t == ft[f]) cf = op.wd[t];
        const float2 wv = w[f * G + P1 + fa[f]];
        df_acc(ys, yc, cf.x, cf.y, wv.x, wv.y);
        if (ft[f] == 0) {
            const float2 wt = w[f * G + fa[f]];
            df_add(ys, yc, wt.x, wt.y);
        }
    }
    return df_to_double(ys, yc);
}

// (A v)_i with dense column-major neighbour blocks (runtime n)
__device__ __forceinline__ double dense_block_row(const double* __restrict__ AdT, const double* __restrict__ AoT,
                                                  const int32_t* __restrict__ nbr, int n, const double* __restrict__ v,
                                                  int e, int i) {
    const double* Ad = AdT + (size_t)e * n * n + i;
    const double* ve = v + (size_t)e * n;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += Ad[(size_t)j * n] * ve[j];
    for (int f = 0; f < 4; ++f) {
        const int e2 = nbr[e * 4 + f];
        if (e2 < 0) continue;
        const double* Ao = AoT + ((size_t)e * 4 + f) * n * n + i;
        const double* v2 = v + (size_t)e2 * n;
        for (int j = 0; j < n; ++j) acc += Ao[(size_t)j * n] * v2[j];
    }
    return acc;
}

__device__ __forceinline__ bool cg_finished(const int* ctl) { return ctl && *(const volatile int*)ctl; }

// ---- deterministic reductions of the CG kernels ----

// Sum over the lanes of the calling warp, valid in lane 0.  Blocks of
// (256 / n) n threads (n = 9, 25) end in a partial warp: its missing lanes
// take no part (the mask names the lanes that exist) and count as zero (a
// value shuffled from a missing lane is undefined, so it is not added).  For
// a full warp this is the plain butterfly.
__device__ __forceinline__ double warp_sum(double v) {
    const int lane = threadIdx.x & 31;
    const int nl = min(32, (int)blockDim.x - (int)(threadIdx.x & ~31u));
    const unsigned mask = nl == 32 ? 0xffffffffu : (1u << nl) - 1u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(mask, v, o);
        if ((lane ^ o) < nl) v += u;
    }
    return v;
}

// Block sum of v into out (thread 0 writes); deterministic order.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    v = warp_sum(v);
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) s += sh[i];
    return s;  // valid in thread 0
}

// two block sums in one pass (one pair of barriers); each is summed in the
// same order as block_sum (warp sums, then the warps in order); valid in
// thread 0; blocks of at most 512 threads, sh at least 32 words
__device__ __forceinline__ void block_sum2(double a, double b, double* sh, double& sa, double& sb) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    a = warp_sum(a);
    b = warp_sum(b);
    __syncthreads();
    if (l == 0) {
        sh[w] = a;
        sh[16 + w] = b;
    }
    __syncthreads();
    sa = 0.0;
    sb = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) {
            sa += sh[i];
            sb += sh[16 + i];
        }
}

// sum over partials written by other blocks of the running kernel (read
// through L2, four loads in flight per thread); deterministic order
__device__ __forceinline__ double sum_partials_cg(const double* part, int nblk, double* sh) {
    const int bd = blockDim.x;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int i = threadIdx.x;
    for (; i + 3 * bd < nblk; i += 4 * bd) {
        const double a0 = __ldcg(part + i), a1 = __ldcg(part + i + bd), a2 = __ldcg(part + i + 2 * bd),
                     a3 = __ldcg(part + i + 3 * bd);
        v0 += a0;
        v1 += a1;
        v2 += a2;
        v3 += a3;
    }
    for (; i < nblk; i += bd) v0 += __ldcg(part + i);
    double s = block_sum((v0 + v1) + (v2 + v3), sh);
    if (threadIdx.x == 0) sh[32] = s;
    __syncthreads();
    s = sh[32];
    __syncthreads();
    return s;
}

// the three partial arrays part[0..count), part[stride..stride + count),
// part[2 stride..2 stride + count) summed in one pass (six independent loads
// in flight per thread); stride < 0: stride = count
__device__ __forceinline__ void sum3_partials_cg(const double* part, int count, double* sh, double& s0, double& s1,
                                                 double& s2, int stride = -1) {
    const int nblk = count;
    const int st = stride < 0 ? count : stride;
    const int bd = blockDim.x;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, u0 = 0.0, u1 = 0.0, u2 = 0.0;
    int i = threadIdx.x;
    for (; i + bd < nblk; i += 2 * bd) {
        const double a0 = __ldcg(part + i), a1 = __ldcg(part + st + i), a2 = __ldcg(part + 2 * st + i);
        const double b0 = __ldcg(part + i + bd), b1 = __ldcg(part + st + i + bd), b2 = __ldcg(part + 2 * st + i + bd);
        v0 += a0;
        v1 += a1;
        v2 += a2;
        u0 += b0;
        u1 += b1;
        u2 += b2;
    }
    for (; i < nblk; i += bd) {
        v0 += __ldcg(part + i);
        v1 += __ldcg(part + st + i);
        v2 += __ldcg(part + 2 * st + i);
    }
    v0 += u0;
    v1 += u1;
    v2 += u2;
    s0 = block_sum(v0, sh);
    s1 = block_sum(v1, sh);
    s2 = block_sum(v2, sh);
    if (threadIdx.x == 0) {
        sh[32] = s0;
        sh[33] = s1;
        sh[34] = s2;
    }
    __syncthreads();
    s0 = sh[32];
    s1 = sh[33];
    s2 = sh[34];
    __syncthreads();
}

// True in the last block of the grid to get here (after its partials are
// written): that block then reduces all partials.  No block waits.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        am_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

}  // namespace smm

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

// shared scratch of one thread block: neighbour face data and coupled face data
template <int N, typename AT>
struct FaceScratch {
    AT g[FaceDims<N>::EPB * FaceDims<N>::NG];
    AT w[FaceDims<N>::EPB * FaceDims<N>::NG];
};

// (A x)_i for row i of element e (act: this thread owns a row).  Every thread
// of the block must call it (two block barriers).  Steps: diagonal block row;
// the neighbours' face data g = E_f2 x_e2 (trace values and normal
// derivatives); w = C_{e,f} g per face; lift (E_f^T w)_i.
template <int N, typename T, typename AT, typename VT>
__device__ __forceinline__ AT faceop_row(const FaceOp<T>& op, const VT* __restrict__ x, int e, int i, bool act,
                                         FaceScratch<N, AT>& sc) {
    using D = FaceDims<N>;
    constexpr int P1 = D::P1, G = D::G, NG = D::NG;
    const int le = threadIdx.x / N;
    AT y = 0;
    if (act) {
        const T* Ad = op.AdT + (size_t)e * N * N + i;
        const VT* xe = x + (size_t)e * N;
#pragma unroll
        for (int j = 0; j < N; ++j) y += (AT)Ad[j * N] * (AT)xe[j];
#pragma unroll
        for (int v0 = 0; v0 < NG; v0 += N) {
            const int v = v0 + i;
            if (v < NG) {
                const int f = v / G, r = v - f * G;
                const int e2 = op.nbr[e * 4 + f];
                AT g = 0;
                if (e2 >= 0) {
                    const int f2 = op.nface[e * 4 + f];
                    const VT* x2 = x + (size_t)e2 * N;
                    if (r < P1) {
                        g = (AT)x2[line_node<P1>(f2, r, 0)];
                    } else {
                        const int a = r - P1;
#pragma unroll
                        for (int t = 0; t < P1; ++t) g += (AT)op.wd[t] * (AT)x2[line_node<P1>(f2, a, t)];
                    }
                }
                sc.g[le * NG + v] = g;
            }
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int v0 = 0; v0 < NG; v0 += N) {
            const int v = v0 + i;
            if (v < NG) {
                const int f = v / G, r = v - f * G;
                AT w = 0;
                if (op.nbr[e * 4 + f] >= 0) {
                    const T* C = op.CT + ((size_t)(e * 4 + f) * G) * G + r;
                    const AT* g = sc.g + le * NG + f * G;
#pragma unroll
                    for (int c = 0; c < G; ++c) w += (AT)C[c * G] * g[c];
                }
                sc.w[le * NG + v] = w;
            }
        }
    }
    __syncthreads();
    if (act) {
        constexpr int p = P1 - 1;
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
    }
    return y;
}

template <int N>
struct FaceScratchDF {
    float2 g[FaceDims<N>::EPB * FaceDims<N>::NG];
    float2 w[FaceDims<N>::EPB * FaceDims<N>::NG];
};

// faceop_row with the operator and x as FP32 pairs, pair arithmetic
// throughout (see dfloat.cuh); the row value is returned in FP64
template <int N>
__device__ __forceinline__ double faceop_row_df(const FaceOpDF& op, const float2* __restrict__ x, int e, int i,
                                                bool act, FaceScratchDF<N>& sc) {
    using D = FaceDims<N>;
    constexpr int P1 = D::P1, G = D::G, NG = D::NG;
    const int le = threadIdx.x / N;
    float ys = 0.0f, yc = 0.0f;
    if (act) {
        const float2* Ad = op.AdT + (size_t)e * N * N + i;
        const float2* xe = x + (size_t)e * N;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float2 a = Ad[j * N], v = xe[j];
            df_acc(ys, yc, a.x, a.y, v.x, v.y);
        }
#pragma unroll
        for (int v0 = 0; v0 < NG; v0 += N) {
            const int v = v0 + i;
            if (v < NG) {
                const int f = v / G, r = v - f * G;
                const int e2 = op.nbr[e * 4 + f];
                float2 g = make_float2(0.0f, 0.0f);
                if (e2 >= 0) {
                    const int f2 = op.nface[e * 4 + f];
                    const float2* x2 = x + (size_t)e2 * N;
                    if (r < P1) {
                        g = x2[line_node<P1>(f2, r, 0)];
                    } else {
                        const int a = r - P1;
                        float gs = 0.0f, gc = 0.0f;
#pragma unroll
                        for (int t = 0; t < P1; ++t) {
                            const float2 xv = x2[line_node<P1>(f2, a, t)];
                            df_acc(gs, gc, op.wd[t].x, op.wd[t].y, xv.x, xv.y);
                        }
                        g = df_norm(gs, gc);
                    }
                }
                sc.g[le * NG + v] = g;
            }
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int v0 = 0; v0 < NG; v0 += N) {
            const int v = v0 + i;
            if (v < NG) {
                const int f = v / G, r = v - f * G;
                float ws = 0.0f, wc = 0.0f;
                if (op.nbr[e * 4 + f] >= 0) {
                    const float2* C = op.CT + ((size_t)(e * 4 + f) * G) * G + r;
                    const float2* g = sc.g + le * NG + f * G;
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        const float2 cv = C[c * G], gv = g[c];
                        df_acc(ws, wc, cv.x, cv.y, gv.x, gv.y);
                    }
                }
                sc.w[le * NG + v] = df_norm(ws, wc);
            }
        }
    }
    __syncthreads();
    if (act) {
        constexpr int p = P1 - 1;
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

}  // namespace smm

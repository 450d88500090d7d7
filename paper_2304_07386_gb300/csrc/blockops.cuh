// Device helpers shared by the PCG and multigrid kernels: element-block
// operator rows with column-major (transposed) n x n blocks.
#pragma once

#include "kernels.cuh"

namespace smm {

// (A v)_i for row i of element e: diagonal block plus the four face-neighbour blocks
// (blocks of type BT, FP64 accumulation)
template <typename BT>
__device__ __forceinline__ double block_row(const BT* __restrict__ AdT, const BT* __restrict__ AoT,
                                            const int32_t* __restrict__ nbr, int n, const double* __restrict__ v,
                                            int e, int i) {
    const BT* Ad = AdT + (size_t)e * n * n + i;
    const double* ve = v + (size_t)e * n;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += (double)Ad[(size_t)j * n] * ve[j];
    for (int f = 0; f < 4; ++f) {
        const int e2 = nbr[e * 4 + f];
        if (e2 < 0) continue;
        const BT* Ao = AoT + ((size_t)e * 4 + f) * n * n + i;
        const double* v2 = v + (size_t)e2 * n;
        for (int j = 0; j < n; ++j) acc += (double)Ao[(size_t)j * n] * v2[j];
    }
    return acc;
}

// FP32 variant for the multigrid smoother: FP32 blocks, vector and accumulation
__device__ __forceinline__ float block_row_f(const float* __restrict__ AdT, const float* __restrict__ AoT,
                                             const int32_t* __restrict__ nbr, int n, const float* __restrict__ v,
                                             int e, int i) {
    const float* Ad = AdT + (size_t)e * n * n + i;
    const float* ve = v + (size_t)e * n;
    float acc = 0.0f;
    for (int j = 0; j < n; ++j) acc = fmaf(Ad[(size_t)j * n], ve[j], acc);
    for (int f = 0; f < 4; ++f) {
        const int e2 = nbr[e * 4 + f];
        if (e2 < 0) continue;
        const float* Ao = AoT + ((size_t)e * 4 + f) * n * n + i;
        const float* v2 = v + (size_t)e2 * n;
        for (int j = 0; j < n; ++j) acc = fmaf(Ao[(size_t)j * n], v2[j], acc);
    }
    return acc;
}

// compile-time block size variants (n = (p+1)^2), fully unrolled
template <int N, typename BT, typename VT, typename AT>
__device__ __forceinline__ AT block_row_n(const BT* __restrict__ AdT, const BT* __restrict__ AoT,
                                          const int32_t* __restrict__ nbr, const VT* __restrict__ v, int e, int i) {
    const BT* Ad = AdT + (size_t)e * N * N + i;
    const VT* ve = v + (size_t)e * N;
    AT acc = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) acc += (AT)Ad[j * N] * (AT)ve[j];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int e2 = nbr[e * 4 + f];
        if (e2 < 0) continue;
        const BT* Ao = AoT + ((size_t)e * 4 + f) * N * N + i;
        const VT* v2 = v + (size_t)e2 * N;
#pragma unroll
        for (int j = 0; j < N; ++j) acc += (AT)Ao[j * N] * (AT)v2[j];
    }
    return acc;
}

__device__ __forceinline__ bool cg_finished(const int* ctl) { return ctl && *(const volatile int*)ctl; }

}  // namespace smm

// Device helpers shared by the PCG and multigrid kernels: element-block
// operator rows with column-major (transposed) n x n blocks.
#pragma once

#include "kernels.cuh"

namespace smm {

// (A v)_i for row i of element e: diagonal block plus the four face-neighbour blocks
__device__ __forceinline__ double block_row(const double* __restrict__ AdT, const double* __restrict__ AoT,
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

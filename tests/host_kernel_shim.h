// Test-only host shim that lets a CUDA kernel body written in plain C++ run on
// the CPU: one std::thread per CUDA thread of a block (blocks run one after
// another), a std::barrier for __syncthreads, the block's dynamic shared memory
// as an exact-size heap buffer, and the round-to-nearest intrinsics as IEEE
// single-precision operations (compile with -ffp-contract=off so that no
// multiply-add is fused that the kernel did not fuse).
#pragma once

#include <algorithm>
#include <barrier>
#include <cmath>
#include <functional>
#include <thread>
#include <vector>

struct float2 {
    float x, y;
};
inline float2 make_float2(float a, float b) { return float2{a, b}; }

struct emu_dim3 {
    int x = 0, y = 0, z = 0;
};
inline thread_local emu_dim3 threadIdx;
inline emu_dim3 blockIdx, blockDim, gridDim;
inline void* emu_dynamic_smem = nullptr;
inline std::barrier<>* emu_block_barrier = nullptr;

#define __global__
#define __device__
#define __forceinline__ inline
#define __restrict__
#define __syncthreads() emu_block_barrier->arrive_and_wait()
using std::max;
using std::min;

inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
inline float __double2float_rn(double v) { return (float)v; }

// Run body() as every thread of grid x threads, with smem bytes of dynamic
// shared memory per block.
inline void emu_launch(int grid, int threads, size_t smem, const std::function<void()>& body) {
    gridDim.x = grid;
    blockDim.x = threads;
    for (int b = 0; b < grid; ++b) {
        blockIdx.x = b;
        std::vector<char> sm(std::max<size_t>(smem, 1));
        emu_dynamic_smem = sm.data();
        std::barrier<> bar(threads);
        emu_block_barrier = &bar;
        std::vector<std::thread> th;
        th.reserve(threads);
        for (int t = 0; t < threads; ++t) th.emplace_back([t, &body] { threadIdx.x = t; body(); });
        for (auto& x : th) x.join();
    }
}

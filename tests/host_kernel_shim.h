// Test-only host shim that lets a CUDA kernel body written in plain C++ run on
// the CPU: one std::thread per CUDA thread of a block (blocks run one after
// another), a std::barrier for __syncthreads, the block's dynamic shared memory
// as an exact-size heap buffer, the round-to-nearest intrinsics as IEEE
// single-precision operations (compile with -ffp-contract=off so that no
// multiply-add is fused that the kernel did not fuse), and __shfl_xor_sync as
// an exchange through per-thread slots with a barrier per warp (every lane of
// a warp that reaches a shuffle must take part, as the full mask requires).
#pragma once

#include <algorithm>
#include <barrier>
#include <cmath>
#include <functional>
#include <memory>
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
#define __launch_bounds__(...)
#define __syncthreads() emu_block_barrier->arrive_and_wait()
using std::max;
using std::min;

inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
inline float __double2float_rn(double v) { return (float)v; }

template <class T>
inline T __ldcg(const T* p) { return *p; }

inline std::vector<double>* emu_warp_slots = nullptr;
inline std::vector<std::unique_ptr<std::barrier<>>>* emu_warp_barriers = nullptr;

inline double __shfl_xor_sync(unsigned, double v, int lane_mask) {
    const int t = threadIdx.x, w = t >> 5;
    (*emu_warp_slots)[t] = v;
    (*emu_warp_barriers)[w]->arrive_and_wait();
    const double r = (*emu_warp_slots)[t ^ lane_mask];
    (*emu_warp_barriers)[w]->arrive_and_wait();
    return r;
}

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
        std::vector<double> slots(threads);
        std::vector<std::unique_ptr<std::barrier<>>> warp_bars;
        for (int w = 0; w * 32 < threads; ++w)
            warp_bars.push_back(std::make_unique<std::barrier<>>(std::min(32, threads - 32 * w)));
        emu_warp_slots = &slots;
        emu_warp_barriers = &warp_bars;
        std::vector<std::thread> th;
        th.reserve(threads);
        for (int t = 0; t < threads; ++t) th.emplace_back([t, &body] { threadIdx.x = t; body(); });
        for (auto& x : th) x.join();
    }
}

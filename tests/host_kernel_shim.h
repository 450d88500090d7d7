// Test-only host shim that lets a CUDA kernel body written in plain C++ run on
// the CPU: one std::thread per CUDA thread of a block (blocks run one after
// another), a std::barrier for __syncthreads, the block's dynamic shared memory
// as an exact-size heap buffer, the round-to-nearest intrinsics as IEEE
// single-precision operations (compile with -ffp-contract=off so that no
// multiply-add is fused that the kernel did not fuse), the warp shuffles and
// votes as an exchange through per-thread slots with a barrier per warp (every
// lane of a warp that reaches one must take part, as the full mask requires),
// and the device atomics and fences as C++ atomics on the same memory.
#pragma once

#include <algorithm>
#include <atomic>
#include <barrier>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>
#include <thread>
#include <vector>

struct float2 {
    float x, y;
};
inline float2 make_float2(float a, float b) { return float2{a, b}; }
struct int2 {
    int x, y;
};
inline int2 make_int2(int a, int b) { return int2{a, b}; }
struct char4 {
    signed char x, y, z, w;
};

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
#define __noinline__
#define __restrict__
#define __launch_bounds__(...)
// a block's static shared variables: one instance, which the block's threads
// share (blocks run one after another)
#define __shared__ static
#define __syncthreads() emu_block_barrier->arrive_and_wait()
using std::isfinite;
using std::max;
using std::min;

inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
inline float __double2float_rn(double v) { return (float)v; }

template <class T>
inline T __ldcg(const T* p) { return *p; }

inline std::vector<unsigned long long>* emu_warp_slots = nullptr;
inline std::vector<std::unique_ptr<std::barrier<>>>* emu_warp_barriers = nullptr;

inline void __syncwarp(unsigned = 0xffffffffu) { (*emu_warp_barriers)[threadIdx.x >> 5]->arrive_and_wait(); }

// every lane publishes v, then reads lane src of its warp
template <class T>
inline T emu_warp_exchange(T v, int src) {
    static_assert(sizeof(T) <= sizeof(unsigned long long), "shuffled values are at most 8 bytes");
    const int t = threadIdx.x, w = t >> 5;
    unsigned long long bits = 0;
    std::memcpy(&bits, &v, sizeof(T));
    (*emu_warp_slots)[t] = bits;
    __syncwarp();
    const unsigned long long got = (*emu_warp_slots)[(w << 5) + src];
    __syncwarp();
    T r;
    std::memcpy(&r, &got, sizeof(T));
    return r;
}

template <class T>
inline T __shfl_sync(unsigned, T v, int src_lane) { return emu_warp_exchange(v, src_lane & 31); }
template <class T>
inline T __shfl_xor_sync(unsigned, T v, int lane_mask) { return emu_warp_exchange(v, (threadIdx.x & 31) ^ lane_mask); }
template <class T>
inline T __shfl_down_sync(unsigned, T v, unsigned delta) {
    const int lane = threadIdx.x & 31, src = lane + (int)delta;
    return emu_warp_exchange(v, src < 32 ? src : lane);
}

// number of lanes of the warp whose predicate holds
inline int emu_warp_count(int pred) {
    const int t = threadIdx.x, w = t >> 5;
    (*emu_warp_slots)[t] = pred ? 1 : 0;
    __syncwarp();
    int c = 0;
    for (int l = 0; l < 32; ++l) c += (int)(*emu_warp_slots)[(w << 5) + l];
    __syncwarp();
    return c;
}
inline int __all_sync(unsigned, int pred) { return emu_warp_count(pred) == 32; }
inline int __any_sync(unsigned, int pred) { return emu_warp_count(pred) > 0; }

inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline void __nanosleep(unsigned) { std::this_thread::yield(); }
inline unsigned atomicAdd(unsigned* p, unsigned v) { return std::atomic_ref<unsigned>(*p).fetch_add(v); }
inline int atomicCAS(int* p, int compare, int val) {
    std::atomic_ref<int>(*p).compare_exchange_strong(compare, val);
    return compare;
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
        // a slot for every lane of every warp, the missing lanes of a partial
        // last warp included: a value read from one of those is undefined on
        // the device, and here it is a NaN as a double and as a float
        std::vector<unsigned long long> slots((threads + 31) / 32 * 32, 0x7ff800007fc00000ull);
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

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
// barriers of the lane groups a mask can name: for each warp, group sizes 4, 8,
// 16 and 32 (index log2(size) - 2), 32 / size aligned groups of each size,
// each sized to the threads that exist (a partial last warp has fewer)
inline std::vector<std::unique_ptr<std::barrier<>>>* emu_group_barriers = nullptr;

inline int emu_log2(unsigned v) { int k = 0; while ((1u << k) < v) ++k; return k; }

// the barrier of the aligned lane group that `mask` names (a whole warp for
// the full mask); groups are contiguous, aligned, of 4 to 32 lanes
inline std::barrier<>& emu_group_barrier(unsigned mask) {
    const int w = threadIdx.x >> 5;
    const int size = mask == 0xffffffffu ? 32 : __builtin_popcount(mask);
    const int base = mask == 0xffffffffu ? 0 : __builtin_ctz(mask);
    const int lg = emu_log2((unsigned)size);
    // per warp: 8 groups of 4, 4 of 8, 2 of 16, 1 of 32 = 15 barriers
    static const int offset[4] = {0, 8, 12, 14};
    return *(*emu_group_barriers)[(size_t)w * 15 + offset[lg - 2] + base / size];
}

inline void __syncwarp(unsigned mask = 0xffffffffu) { emu_group_barrier(mask).arrive_and_wait(); }

// every lane of the group publishes v, then reads lane src of its warp
template <class T>
inline T emu_warp_exchange(T v, int src, unsigned mask) {
    static_assert(sizeof(T) <= sizeof(unsigned long long), "shuffled values are at most 8 bytes");
    const int t = threadIdx.x, w = t >> 5;
    unsigned long long bits = 0;
    std::memcpy(&bits, &v, sizeof(T));
    (*emu_warp_slots)[t] = bits;
    __syncwarp(mask);
    const unsigned long long got = (*emu_warp_slots)[(w << 5) + src];
    __syncwarp(mask);
    T r;
    std::memcpy(&r, &got, sizeof(T));
    return r;
}

// CUDA's width argument: the warp is cut into segments of `width` lanes
template <class T>
inline T __shfl_sync(unsigned mask, T v, int src_lane, int width = 32) {
    const int lane = threadIdx.x & 31;
    return emu_warp_exchange(v, (lane & ~(width - 1)) + (src_lane & (width - 1)), mask);
}
template <class T>
inline T __shfl_xor_sync(unsigned mask, T v, int lane_mask, int width = 32) {
    const int lane = threadIdx.x & 31, src = lane ^ lane_mask;
    return emu_warp_exchange(v, (src & ~(width - 1)) > (lane & ~(width - 1)) ? lane : src, mask);
}
template <class T>
inline T __shfl_down_sync(unsigned mask, T v, unsigned delta, int width = 32) {
    const int lane = threadIdx.x & 31, src = (lane & (width - 1)) + (int)delta;
    return emu_warp_exchange(v, src < width ? lane + (int)delta : lane, mask);
}

// number of lanes of the group whose predicate holds, and the group's size
inline int emu_warp_count(int pred, unsigned mask, int* members) {
    const int t = threadIdx.x, w = t >> 5;
    (*emu_warp_slots)[t] = pred ? 1 : 0;
    __syncwarp(mask);
    int c = 0, m = 0;
    for (int l = 0; l < 32; ++l)
        if ((mask >> l) & 1u) {
            const int tl = (w << 5) + l;
            if (tl < (int)blockDim.x) {
                c += (int)(*emu_warp_slots)[tl];
                ++m;
            }
        }
    __syncwarp(mask);
    *members = m;
    return c;
}
inline int __all_sync(unsigned mask, int pred) {
    int m = 0;
    return emu_warp_count(pred, mask, &m) == m;
}
inline int __any_sync(unsigned mask, int pred) {
    int m = 0;
    return emu_warp_count(pred, mask, &m) > 0;
}

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
        std::vector<std::unique_ptr<std::barrier<>>> group_bars;
        for (int w = 0; w * 32 < threads; ++w)
            for (int size : {4, 8, 16, 32})
                for (int g = 0; g < 32 / size; ++g) {
                    const int first = 32 * w + g * size;
                    const int members = std::max(1, std::min(size, threads - first));
                    group_bars.push_back(std::make_unique<std::barrier<>>(members));
                }
        emu_warp_slots = &slots;
        emu_group_barriers = &group_bars;
        std::vector<std::thread> th;
        th.reserve(threads);
        for (int t = 0; t < threads; ++t) th.emplace_back([t, &body] { threadIdx.x = t; body(); });
        for (auto& x : th) x.join();
    }
}

// Multigrid V-cycle preconditioner for the IP-SMM moment operator.
//
// Level 0: DG-p element blocks, nu0 smoothing steps before and after the
// coarse correction -- the degree-nu0 Chebyshev polynomial in Pinv A (Pinv
// the element-block inverses) or damped element-block Jacobi -- in FP32 (the
// preconditioner only has to approximate the inverse; FP64 arithmetic on these
// blocks is bound by the GPU's FP64 rate, FP32 by HBM).  The CG around it is
// flexible, so the rounding of the FP32 cycle does not break its recurrences.
// Level 1: continuous bilinear functions on the mesh vertices (restriction
// gathers the four corner weights of every element node, prolongation
// interpolates them back).  Levels 2..: smoothed-aggregation operators with
// one damped Jacobi step before and after; the coarsest level is a dense
// inverse.  Levels >= 1 are stored (k-major ELL) and applied in FP32 and run
// as one cluster launch.  The same smoothing polynomial before and after keeps
// the cycle symmetric.  Every kernel returns at once when the CG control word
// says the solve has finished.
#include <algorithm>

#include <cooperative_groups.h>

#include "blockops.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace smm {

namespace {

// ---- level-0 kernels: one block per EPB = 256 / N elements (thread = row)

// asynchronous L2 prefetch of a 16-byte-aligned span (size a multiple of 16);
// nothing waits for it
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// rows per thread of the level-0 smoothing steps (see bj_smooth_kernel)
constexpr int kSmoothRows = 2;

// true when the CG has finished
__device__ __forceinline__ bool mg_skip(const int* ctl) { return ((const volatile int*)ctl)[0] != 0; }

// One level-0 smoothing step in FP32:
//   xout = xin + c2 Pinv (b - A xin) + c1 (xin - xprev)
// (damped block Jacobi: c1 = 0, c2 = omega; a Chebyshev step: the three-term
// recurrence's coefficients).  xin == nullptr means xin = 0, xprev == nullptr
// means xprev = 0; xout may be xprev (each row reads only its own xprev).  b is
// the FP64 right-hand side, xout is FP32 (inner steps) or FP64 (last step).
// Pinv is the inverse of the diagonal block A_d (formed in FP64), so
// Pinv (b - A xin) = Pinv (b - A_off xin) - xin: the step reads the face
// couplings and Pinv but not A_d, and uses z - xin with z = Pinv (b - A_off xin).
// Thread (slot le, row i) of a block handles row i of the R elements
// e0 + k EPB, k < R (e0 = blockIdx.x EPB R + le): with R = 2 the 16,384 x 25
// rows of the bench workload fit the GPU's resident threads at once instead
// of 1.35 waves, and each thread has R independent rows in flight.
template <typename OT, int N, int R>
__global__ void __launch_bounds__(256) bj_smooth_kernel(int ne, FaceOp<float> A, const float* __restrict__ PinvT,
                                                        float c1, float c2, const double* __restrict__ b,
                                                        const float* __restrict__ xin, const float* xprev,
                                                        OT* xout, const int* ctl) {
    if (mg_skip(ctl)) return;
    constexpr int EPB = FaceDims<N>::EPB, G = FaceDims<N>::G;
    __shared__ float res[R][256];
    __shared__ FaceScratch<N, float, EPB * R> sc;
    const int le = threadIdx.x / N, i = threadIdx.x % N;
    const int e0 = blockIdx.x * EPB * R + le;
    float r[R], x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        r[k] = 0.0f;
        x[k] = 0.0f;
    }
    if (xin) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int e = e0 + k * EPB;
            if (e < ne) face_gather<N>(A, xin, e, i, sc, le + k * EPB);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int e = e0 + k * EPB;
            if (e < ne) face_couple<N>(A.CT + (size_t)e * 4 * G * G, A.nbr, e, i, sc, le + k * EPB);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int e = e0 + k * EPB;
            if (e < ne) {
                const float ax = face_lift<N>(A, i, 0.0f, sc, le + k * EPB);
                x[k] = xin[(size_t)e * N + i];
                r[k] = (float)b[(size_t)e * N + i] - ax;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int e = e0 + k * EPB;
            if (e < ne) r[k] = (float)b[(size_t)e * N + i];
        }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) res[k][threadIdx.x] = r[k];
    __syncthreads();
    const unsigned long long pol = l2_keep();
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        if (e < ne) {
            const float* P = PinvT + (size_t)e * N * N + i;
            const float* re = res[k] + le * N;
            float z = 0.0f;
#pragma unroll
            for (int j = 0; j < N; ++j) z = fmaf(ld_hint(P + j * N, pol), re[j], z);
            const size_t o = (size_t)e * N + i;
            const float xp = xprev ? xprev[o] : 0.0f;
            xout[o] = (OT)(x[k] + c2 * (z - x[k]) + c1 * (x[k] - xp));
        }
    }
}

// Level-0 residual res = b - A x (FP32) restricted to the element corners:
// cres[e][c] = sum_i w4[i][c] res[e][i] (the vertex level sums these over the
// elements at each vertex).  Only these sums are needed, so the diagonal
// blocks enter through W = w4^T A_d (WdT [e][j][c], 4 n words per element):
// cres[e][c] = sum_i w4[i][c] (b - A_off x)_i - sum_j W[c][j] x_j.  The
// coarse cycle runs next and chains dependent loads through its levels' data,
// which the operator product has pushed out of L2: thread 0 of the first
// blocks prefetches those chunks (pf) into L2.  R rows per thread as in
// bj_smooth_kernel.
template <int N, int R>
__global__ void __launch_bounds__(256) bj_residual_kernel(int ne, FaceOp<float> A, const float* __restrict__ WdT,
                                                          const double* __restrict__ b, const float* __restrict__ x,
                                                          const float* __restrict__ w4, float* __restrict__ cres,
                                                          const L2Chunk* __restrict__ pf, int npf, const int* ctl) {
    if (mg_skip(ctl)) return;
    if (threadIdx.x == 0)
        for (int c = blockIdx.x; c < npf; c += gridDim.x) prefetch_l2(pf[c].p, pf[c].bytes);
    constexpr int EPB = FaceDims<N>::EPB, G = FaceDims<N>::G;
    __shared__ FaceScratch<N, float, EPB * R> sc;
    __shared__ float rs[R][256];
    const int le = threadIdx.x / N, i = threadIdx.x % N;
    const int e0 = blockIdx.x * EPB * R + le;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        if (e < ne) face_gather<N>(A, x, e, i, sc, le + k * EPB);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        if (e < ne) face_couple<N>(A.CT + (size_t)e * 4 * G * G, A.nbr, e, i, sc, le + k * EPB);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        float rv = 0.0f;
        if (e < ne) rv = (float)b[(size_t)e * N + i] - face_lift<N>(A, i, 0.0f, sc, le + k * EPB);
        rs[k][threadIdx.x] = rv;
    }
    __syncthreads();
    if (i < 4) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int e = e0 + k * EPB;
            if (e < ne) {
                const float* re = rs[k] + le * N;
                const float* W = WdT + (size_t)e * N * 4 + i;
                const float* xe = x + (size_t)e * N;
                float s = 0.0f;
#pragma unroll
                for (int j = 0; j < N; ++j) s = fmaf(w4[j * 4 + i], re[j], s);
#pragma unroll
                for (int j = 0; j < N; ++j) s = fmaf(-W[j * 4], xe[j], s);
                cres[(size_t)e * 4 + i] = s;
            }
        }
    }
}

// First pre-smoothing step (from zero) of a flexible-CG iteration with the
// CG update folded in: x += alpha p, r_old = r, r -= alpha q (alpha = rz / p.q
// from the operator product's last block), partial r.r -> part[nblk + block];
// xout = c2 Pinv r in FP32.  R rows per thread as in bj_smooth_kernel.
template <int N, int R>
__global__ void __launch_bounds__(256) bj_first_update_kernel(CGArgs a, const float* __restrict__ PinvT, float c2,
                                                              float* __restrict__ xout) {
    if (mg_skip(a.ctl)) return;
    constexpr int EPB = FaceDims<N>::EPB;
    __shared__ float res[R][256];
    __shared__ double sh[40];
    const int le = threadIdx.x / N, i = threadIdx.x % N;
    const int e0 = blockIdx.x * EPB * R + le;
    const double alpha = a.scal[5];
    double rr = 0.0;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        float r = 0.0f;
        if (e < a.ne) {
            const size_t o = (size_t)e * N + i;
            a.x[o] += alpha * a.p[o];
            const double ro = a.r[o];
            a.rold[o] = ro;
            const double rn = ro - alpha * a.q[o];
            a.r[o] = rn;
            rr += rn * rn;
            r = (float)rn;
        }
        res[k][threadIdx.x] = r;
    }
    __syncthreads();
    const unsigned long long pol = l2_keep();
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        if (e < a.ne) {
            const float* P = PinvT + (size_t)e * N * N + i;
            const float* re = res[k] + le * N;
            float z = 0.0f;
#pragma unroll
            for (int j = 0; j < N; ++j) z = fmaf(ld_hint(P + j * N, pol), re[j], z);
            xout[(size_t)e * N + i] = c2 * z;
        }
    }
    const double s = block_sum(rr, sh);
    if (threadIdx.x == 0) a.part[a.nblk + blockIdx.x] = s;
}

// Last post-smoothing step of a flexible-CG iteration, z = x + c2 (Pinv
// (r - A_off x) - x) + c1 (x - xprev) written in FP64 (xprev == nullptr:
// zero), with the CG dot products folded in: partials r.z -> part[2 nblk +
// block] and (r - r_old).z -> part[3 nblk + block].  The last block reduces
// them with the first step's r.r partials (gridDim.x of each): beta =
// (r - r_old).z / rz_old, rz, rr, the iteration count and the convergence
// test.  R rows per thread as in bj_smooth_kernel; the first step has the same
// grid, so the partial counts agree.
template <int N, int R>
__global__ void __launch_bounds__(256) bj_last_dots_kernel(CGArgs a, FaceOp<float> A, const float* __restrict__ PinvT,
                                                           float c1, float c2, const float* __restrict__ xin,
                                                           const float* __restrict__ xprev) {
    if (mg_skip(a.ctl)) return;
    constexpr int EPB = FaceDims<N>::EPB, G = FaceDims<N>::G;
    __shared__ float res[R][256];
    __shared__ FaceScratch<N, float, EPB * R> sc;
    __shared__ double sh[40];
    const int le = threadIdx.x / N, i = threadIdx.x % N;
    const int e0 = blockIdx.x * EPB * R + le;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        if (e < a.ne) face_gather<N>(A, xin, e, i, sc, le + k * EPB);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        if (e < a.ne) face_couple<N>(A.CT + (size_t)e * 4 * G * G, A.nbr, e, i, sc, le + k * EPB);
    }
    __syncthreads();
    float x[R];
    double rd[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        float r = 0.0f;
        x[k] = 0.0f;
        rd[k] = 0.0;
        if (e < a.ne) {
            const float ax = face_lift<N>(A, i, 0.0f, sc, le + k * EPB);
            x[k] = xin[(size_t)e * N + i];
            rd[k] = a.r[(size_t)e * N + i];
            r = (float)rd[k] - ax;
        }
        res[k][threadIdx.x] = r;
    }
    __syncthreads();
    double rz = 0.0, dz = 0.0;
    const unsigned long long pol = l2_keep();
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        if (e < a.ne) {
            const float* P = PinvT + (size_t)e * N * N + i;
            const float* re = res[k] + le * N;
            float z = 0.0f;
#pragma unroll
            for (int j = 0; j < N; ++j) z = fmaf(ld_hint(P + j * N, pol), re[j], z);
            const size_t o = (size_t)e * N + i;
            const float xp = xprev ? xprev[o] : 0.0f;
            const double zd = (double)(x[k] + c2 * (z - x[k]) + c1 * (x[k] - xp));
            a.z[o] = zd;
            rz += rd[k] * zd;
            dz += (rd[k] - a.rold[o]) * zd;
        }
    }
    double s1, s2;
    block_sum2(rz, dz, sh, s1, s2);
    if (threadIdx.x == 0) {
        a.part[2 * a.nblk + blockIdx.x] = s1;
        a.part[3 * a.nblk + blockIdx.x] = s2;
    }
    if (last_block((unsigned*)(a.ctl + 6))) {
        double rr, rz_new, dz_all;
        sum3_partials_cg(a.part + a.nblk, gridDim.x, sh, rr, rz_new, dz_all, a.nblk);
        if (threadIdx.x == 0) {
            a.scal[6] = dz_all / a.scal[0];
            a.scal[0] = rz_new;
            a.scal[2] = rr;
            const int it = a.ctl[1] + 1;
            a.ctl[1] = it;
            const bool bad = !(isfinite(rz_new) && isfinite(rr) && isfinite(dz_all));
            if (bad) a.ctl[3] = 1;
            if (rr <= a.scal[4] || it >= a.ctl[2] || bad) a.ctl[0] = 1;
            a.ctl[6] = 0;
        }
    }
}

// x[e][i] += sum_c w4[i][c] xv[vid[e][c]]
__global__ void prolong_q1_kernel(int ne, int n, const int* __restrict__ vid, const float* __restrict__ w4,
                                  const float* __restrict__ xv, float* __restrict__ x, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * n) return;
    const int e = t / n, i = t - e * n;
    const int* ve = vid + e * 4;
    const float* w = w4 + i * 4;
    x[t] += w[0] * xv[ve[0]] + w[1] * xv[ve[1]] + w[2] * xv[ve[2]] + w[3] * xv[ve[3]];
}

// The coarse part of the cycle -- the vertex-level right-hand side from the
// element-corner residuals, the CSR levels down and up and the dense
// coarsest solve -- in one launch of one thread-block cluster.  Each stage is
// a grid-stride loop over the cluster's threads; stages are separated by the
// cluster's hardware barrier (no flag waits).  Vectors written inside the
// kernel are read through L2 (ld.global.cg).  The result is lv[1].t (or the
// coarsest x when the vertex level is the coarsest).
constexpr int kCoarseThreads = 512;   // 128 registers per thread: a row's loads stay in flight

struct CoarseArgs {
    int nvert, nlev;
    int first;                                  // 1: the whole coarse cycle; 2: the vertex level runs as
                                                // grid kernels around the launch, which starts with b_2 = R r_1
    int cap;                                    // floats of dynamic shared memory (staged vectors)
    const float* cres;                          // [ne][4] corner sums of the level-0 residual
    int vw; const int* vinc;                    // vertex incidences, k-major ELL with -1 padding
    MGLevelDev lv[12];
    const float* cinv;
};

// vectors of up to this many floats are staged in each CTA's shared memory
// for a stage's gathers (192 KB of the 227 KB a CTA may hold)
constexpr int kCoarseSmemFloats = 49152;

// row i of a k-major ELL matrix (width w <= W, R rows) times x: the column and
// value loads are issued first (coalesced: a warp's loads for one k cover
// consecutive rows), then the gathers of x, from shared memory (SH) or
// through L2
template <int W, bool SH>
__device__ __forceinline__ float ell_row_w(int w, int R, const int* __restrict__ ci, const float* __restrict__ v,
                                           const float* x, int i) {
    int c[W];
    float wv[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const bool on = k < w;
        c[k] = on ? ci[(size_t)k * R + i] : 0;
        wv[k] = on ? v[(size_t)k * R + i] : 0.0f;
    }
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
    for (int k = 0; k < W; k += 2) {
        const float x0 = k < w ? (SH ? x[c[k]] : __ldcg(x + c[k])) : 0.0f;
        const float x1 = k + 1 < w ? (SH ? x[c[k + 1]] : __ldcg(x + c[k + 1])) : 0.0f;
        a0 = fmaf(wv[k], x0, a0);
        a1 = fmaf(wv[k + 1], x1, a1);
    }
    return a0 + a1;
}

// row i of a k-major ELL matrix of any width: one pass for w <= 24, passes of
// 24 entries beyond
template <bool SH>
__device__ __forceinline__ float ell_row(int w, int R, const int* __restrict__ ci, const float* __restrict__ v,
                                      const float* x, int i) {
    if (w <= 8) return ell_row_w<8, SH>(w, R, ci, v, x, i);
    if (w <= 16) return ell_row_w<16, SH>(w, R, ci, v, x, i);
    float s = 0.0f;
    for (int k0 = 0; k0 < w; k0 += 24)
        s += ell_row_w<24, SH>(min(24, w - k0), R, ci + (size_t)k0 * R, v + (size_t)k0 * R, x, i);
    return s;
}

// Copy x[0..n) into this CTA's shared memory xs when it fits (every thread of
// the CTA takes part); true if staged.  x (16-byte aligned, a device
// allocation) was written by other CTAs before the last cluster barrier, so it
// is read through L2, as 16-byte loads with four in flight per thread.
__device__ __forceinline__ bool stage_x(const float* x, int n, float* xs, int cap) {
    if (n > cap) return false;
    const int n4 = n >> 2;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4* xs4 = reinterpret_cast<float4*>(xs);
    for (int k0 = threadIdx.x; k0 < n4; k0 += 4 * blockDim.x) {
        float4 t[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + q * blockDim.x;
            if (k < n4) t[q] = __ldcg(x4 + k);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + q * blockDim.x;
            if (k < n4) xs4[k] = t[q];
        }
    }
    for (int k = 4 * n4 + threadIdx.x; k < n; k += blockDim.x) xs[k] = __ldcg(x + k);
    __syncthreads();
    return true;
}

// row with x in global memory (vectors larger than the shared-memory budget);
// out of line, so that it does not add to the registers of the staged path
__device__ __noinline__ float ell_row_global(int w, int R, const int* ci, const float* v, const float* x, int i) {
    return ell_row<false>(w, R, ci, v, x, i);
}

// (M x)_i with x staged in xs (sh) or read from global memory
__device__ __forceinline__ float ell_apply(bool sh, int w, int R, const int* ci, const float* v, const float* x,
                                           const float* xs, int i) {
    return sh ? ell_row<true>(w, R, ci, v, xs, i) : ell_row_global(w, R, ci, v, x, i);
}

// launched as one cluster of gridDim.x CTAs (8, or 16 where the GPU allows it)
__global__ void __launch_bounds__(kCoarseThreads) coarse_cycle_kernel(CoarseArgs a, const int* ctl) {
    if (cg_finished(ctl)) return;  // uniform over the cluster: no barrier is left waiting
    extern __shared__ __align__(16) float xs[];   // a.cap floats
    cg::cluster_group cl = cg::this_cluster();
    const int T = gridDim.x * kCoarseThreads;
    // warps numbered across the CTAs first (warp slot w of CTA c is warp w * gridDim.x + c), so
    // that a stage with few rows still spreads over every SM of the cluster while each warp
    // covers 32 consecutive rows (coalesced ELL loads)
    const int tid = (((int)threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x) * 32 + ((int)threadIdx.x & 31);
    // vertex-level right-hand side: sum of the corner sums of the elements at each vertex
    if (a.first == 1) {
        float* b1 = a.lv[1].b;
        for (int v = tid; v < a.nvert; v += T) {
            float s = 0.0f;
            for (int k0 = 0; k0 < a.vw; k0 += 8) {
                int c[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) c[k] = k0 + k < a.vw ? a.vinc[(size_t)(k0 + k) * a.nvert + v] : -1;
#pragma unroll
                for (int k = 0; k < 8; ++k) s += c[k] >= 0 ? __ldcg(a.cres + c[k]) : 0.0f;
            }
            b1[v] = s;
        }
        cl.sync();
    }
    // Each stage below reads one vector written in the stage before (by any
    // CTA): it is first copied into every CTA's shared memory (when it fits)
    // so that the row gathers are shared-memory loads.
    // down: x = omega dinv b ; r = b - A x ; b_{l+1} = R r.  The residual is
    // formed as b - As b with As = A diag(omega dinv) (stored), so x and r come
    // out of one pass over b.
    for (int l = 1; l < a.nlev; ++l) {
        const MGLevelDev& L = a.lv[l];
        if (l >= a.first) {
            const bool sb = stage_x(L.b, L.n, xs, a.cap);
            for (int i = tid; i < L.n; i += T) {
                const float bi = sb ? xs[i] : __ldcg(L.b + i);
                const float si = ell_apply(sb, L.aw, L.n, L.Aci, L.Asv, L.b, xs, i);
                L.r[i] = bi - si;
                L.x[i] = L.omega * L.dinv[i] * bi;
            }
            cl.sync();
        }
        const MGLevelDev& Lc = a.lv[l + 1];
        const bool sr = stage_x(L.r, L.n, xs, a.cap);
        for (int i = tid; i < Lc.n; i += T) Lc.b[i] = ell_apply(sr, L.rw, Lc.n, L.Rci, L.Rv, L.r, xs, i);
        cl.sync();
    }
    // coarsest: x = Cinv b, one warp per row
    {
        const MGLevelDev& C = a.lv[a.nlev];
        const bool sc = stage_x(C.b, C.n, xs, a.cap);
        const float* bsrc = sc ? (const float*)xs : C.b;
        const int lane = threadIdx.x & 31, w = tid >> 5, nw = T >> 5;
        for (int row = w; row < C.n; row += nw) {
            const float* cr = a.cinv + (size_t)row * C.n;
            float s = 0.0f;
            for (int j0 = 0; j0 < C.n; j0 += 256) {
                float cv[8], bv[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = j0 + q * 32 + lane;
                    cv[q] = j < C.n ? cr[j] : 0.0f;
                    bv[q] = j < C.n ? (sc ? bsrc[j] : __ldcg(bsrc + j)) : 0.0f;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) s = fmaf(cv[q], bv[q], s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) C.x[row] = s;
        }
    }
    cl.sync();
    // up: x += P x_{l+1} ; t = x + omega dinv (b - A x)
    const float* coarse_out = a.lv[a.nlev].x;
    for (int l = a.nlev - 1; l >= a.first; --l) {
        const MGLevelDev& L = a.lv[l];
        const bool sp = stage_x(coarse_out, a.lv[l + 1].n, xs, a.cap);
        for (int i = tid; i < L.n; i += T) {
            const float xi = __ldcg(L.x + i);
            L.x[i] = xi + ell_apply(sp, L.pw, L.n, L.Pci, L.Pv, coarse_out, xs, i);
        }
        cl.sync();
        const bool sx = stage_x(L.x, L.n, xs, a.cap);
        for (int i = tid; i < L.n; i += T) {
            const float xi = sx ? xs[i] : __ldcg(L.x + i), bi = __ldcg(L.b + i), di = L.dinv[i];
            const float si = ell_apply(sx, L.aw, L.n, L.Aci, L.Av, L.x, xs, i);
            L.t[i] = xi + L.omega * di * (bi - si);
        }
        cl.sync();
        coarse_out = L.t;
    }
}

// The vertex level's stages on the whole GPU (a thread per vertex), for vertex
// levels too large for the cluster's shared memory; the same arithmetic as the
// cluster's stages.  b_1 = the corner sums of the elements at each vertex:
__global__ void vertex_rhs_kernel(int nvert, int vw, const int* __restrict__ vinc, const float* __restrict__ cres,
                                  float* __restrict__ b1, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvert) return;
    float s = 0.0f;
    for (int k0 = 0; k0 < vw; k0 += 8) {
        int c[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) c[k] = k0 + k < vw ? vinc[(size_t)(k0 + k) * nvert + v] : -1;
#pragma unroll
        for (int k = 0; k < 8; ++k) s += c[k] >= 0 ? __ldcg(cres + c[k]) : 0.0f;
    }
    b1[v] = s;
}

// x_1 = omega dinv b_1 ; r_1 = b_1 - A_1 x_1 (as b_1 - As_1 b_1)
__global__ void vertex_down_kernel(MGLevelDev L, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const float bi = __ldcg(L.b + i);
    const float si = ell_row<false>(L.aw, L.n, L.Aci, L.Asv, L.b, i);
    L.r[i] = bi - si;
    L.x[i] = L.omega * L.dinv[i] * bi;
}

// x_1 += P_1 x_2 (the coarse correction from level 2)
__global__ void vertex_up_kernel(MGLevelDev L, const float* __restrict__ x2, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    L.x[i] = __ldcg(L.x + i) + ell_row<false>(L.pw, L.n, L.Pci, L.Pv, x2, i);
}

// t_1 = x_1 + omega dinv (b_1 - A_1 x_1)
__global__ void vertex_post_kernel(MGLevelDev L, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const float xi = __ldcg(L.x + i), bi = __ldcg(L.b + i), di = L.dinv[i];
    const float si = ell_row<false>(L.aw, L.n, L.Aci, L.Av, L.x, i);
    L.t[i] = xi + L.omega * di * (bi - si);
}

}  // namespace

template <int N>
int mg_apply_n(const MGPlan& m, const double* r, double* z, const int* ctl, cudaStream_t s);

int mg_coarse_cluster_size() {
    // 16 CTAs (a non-portable cluster size) where the device can co-schedule
    // them, else the portable 8
    static int chosen = 0;
    if (chosen) return chosen;
    int ctas = 8;
    cudaFuncSetAttribute(coarse_cycle_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kCoarseSmemFloats * (int)sizeof(float));
    if (cudaFuncSetAttribute(coarse_cycle_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        cfg.gridDim = dim3(16, 1, 1);
        cfg.blockDim = dim3(kCoarseThreads, 1, 1);
        cfg.dynamicSmemBytes = kCoarseSmemFloats * sizeof(float);
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, coarse_cycle_kernel, &cfg) == cudaSuccess && nclusters >= 1)
            ctas = 16;
    }
    cudaGetLastError();
    chosen = ctas;
    return chosen;
}

// The vertex level goes to grid kernels when it has more rows than this (its
// vectors then no longer fit the cluster's shared memory, and one cluster's 16
// SMs take its passes alone) and a level below it exists.
constexpr int kSplitVertexRows = 32768;

bool mg_split_vertex_level(const MGPlan& m) { return m.nlev >= 2 && m.nvert > kSplitVertexRows; }

// The coarse part of the V-cycle: one cluster launch, or, for a large vertex
// level, the vertex level's stages as grid kernels around a cluster launch
// that covers the levels below it.  Returns the vertex-level correction that
// prolong_q1_kernel reads; *launches gets the kernels launched.
const float* launch_coarse_cycle(const MGPlan& m, const float* cres, const int* ctl, cudaStream_t s, int* launches) {
    const bool split = mg_split_vertex_level(m);
    const MGLevelDev& L1 = m.lv[1];
    const int g1 = (m.nvert + 255) / 256;
    if (split) {
        vertex_rhs_kernel<<<g1, 256, 0, s>>>(m.nvert, m.vw, m.vinc, cres, L1.b, ctl);
        vertex_down_kernel<<<g1, 256, 0, s>>>(L1, ctl);
    }
    CoarseArgs ca{};
    ca.nvert = m.nvert; ca.nlev = m.nlev; ca.cres = cres; ca.vw = m.vw; ca.vinc = m.vinc;
    ca.first = split ? 2 : 1;
    for (int l = 0; l <= m.nlev; ++l) ca.lv[l] = m.lv[l];
    ca.cinv = m.cinv;
    // shared memory for the largest vector a stage stages, up to kCoarseSmemFloats
    int vmax = 0;
    for (int l = ca.first; l <= m.nlev; ++l) vmax = std::max(vmax, m.lv[l].n);
    ca.cap = std::min(vmax, kCoarseSmemFloats);
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(m.coarse_ctas, 1, 1);
    cfg.blockDim = dim3(kCoarseThreads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)ca.cap * sizeof(float);
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = m.coarse_ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, coarse_cycle_kernel, ca, ctl);
    if (!split) {
        *launches = 1;
        return m.nlev > 1 ? m.lv[1].t : m.lv[1].x;
    }
    vertex_up_kernel<<<g1, 256, 0, s>>>(L1, m.nlev > 2 ? m.lv[2].t : m.lv[2].x, ctl);
    vertex_post_kernel<<<g1, 256, 0, s>>>(L1, ctl);
    *launches = 5;
    return L1.t;
}

int mg_apply(const MGPlan& m, const double* r, double* z, const int* ctl, cudaStream_t s) {
    switch (m.n) {
        case 4: return mg_apply_n<4>(m, r, z, ctl, s);
        case 9: return mg_apply_n<9>(m, r, z, ctl, s);
        case 16: return mg_apply_n<16>(m, r, z, ctl, s);
        case 25: return mg_apply_n<25>(m, r, z, ctl, s);
        default: return 0;
    }
}

// Coefficients (c1[k], c2[k]) of the level-0 smoothing steps k = 0..nu0-1,
// x_{k+1} = x_k + c2 Pinv (b - A x_k) + c1 (x_k - x_{k-1}).  Damped block
// Jacobi: c1 = 0, c2 = omega0.  Chebyshev of degree nu0 for Pinv A on
// [lmax / 60, lmax], lmax = (4/3) / omega0 (the power-iteration estimate times
// 1.05), by the three-term recurrence of Chebyshev acceleration: with
// theta, delta the interval's centre and half-width, sigma = theta / delta,
// rho_0 = 1 / sigma, rho_k = 1 / (2 sigma - rho_{k-1}): c2 = 1 / theta, c1 = 0
// for k = 0 and c2 = 2 rho_k / delta, c1 = rho_k rho_{k-1} after.
static void smoother_coeffs(const MGPlan& m, float* c1, float* c2) {
    if (!m.chebyshev) {
        for (int k = 0; k < m.nu0; ++k) {
            c1[k] = 0.0f;
            c2[k] = (float)m.omega0;
        }
        return;
    }
    const double hi = (4.0 / 3.0) / m.omega0, lo = hi / 60.0;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    c1[0] = 0.0f;
    c2[0] = (float)(1.0 / theta);
    for (int k = 1; k < m.nu0; ++k) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        c1[k] = (float)(rn * rho);
        c2[k] = (float)(2.0 * rn / delta);
        rho = rn;
    }
}

// The smoothing steps after the first keep the current and the previous
// iterate in the two FP32 buffers; a step writes over the previous iterate
// (or into the other buffer while the previous iterate is zero).
struct SmoothState {
    float* cur;
    float* prev;   // nullptr: zero
    float* other;  // the buffer that is not cur
    float* next() const { return prev ? prev : other; }
    void advance(float* out) {
        other = cur == out ? other : cur;
        prev = cur;
        cur = out;
    }
};

template <int N>
int mg_apply_n(const MGPlan& m, const double* r, double* z, const int* ctl, cudaStream_t s) {
    int launches = 0;
    const int tpb = cg_threads_per_block(N);
    const int nblkR = (m.ne + FaceDims<N>::EPB * kSmoothRows - 1) / (FaceDims<N>::EPB * kSmoothRows);
    float c1[4], c2[4];
    smoother_coeffs(m, c1, c2);
    // level 0 pre-smoothing from zero (FP32)
    SmoothState st{m.x0, nullptr, m.x0b};
    bj_smooth_kernel<float, N, kSmoothRows><<<nblkR, tpb, 0, s>>>(m.ne, m.A, m.PinvT, c1[0], c2[0], r, nullptr, nullptr, st.cur,
                                                     ctl);
    ++launches;
    for (int k = 1; k < m.nu0; ++k) {
        float* out = st.next();
        bj_smooth_kernel<float, N, kSmoothRows><<<nblkR, tpb, 0, s>>>(m.ne, m.A, m.PinvT, c1[k], c2[k], r, st.cur, st.prev, out,
                                                         ctl);
        st.advance(out);
        ++launches;
    }
    bj_residual_kernel<N, kSmoothRows><<<nblkR, tpb, 0, s>>>(m.ne, m.A, m.WdT, r, st.cur, m.w4, m.res0,
                                                           m.coarse_pf, m.coarse_npf, ctl);
    // vertex and aggregation levels and the coarsest solve
    int lc = 0;
    const float* coarse_out = launch_coarse_cycle(m, m.res0, ctl, s, &lc);
    const int rows0 = m.ne * N;
    prolong_q1_kernel<<<(rows0 + 255) / 256, 256, 0, s>>>(m.ne, N, m.vid, m.w4, coarse_out, st.cur, ctl);
    launches += 2 + lc;
    // post-smoothing: the recurrence restarts from the corrected iterate
    st.prev = nullptr;
    for (int k = 0; k < m.nu0; ++k) {
        if (k == m.nu0 - 1) {
            bj_smooth_kernel<double, N, kSmoothRows><<<nblkR, tpb, 0, s>>>(m.ne, m.A, m.PinvT, c1[k], c2[k], r, st.cur, st.prev, z,
                                                              ctl);
        } else {
            float* out = st.next();
            bj_smooth_kernel<float, N, kSmoothRows><<<nblkR, tpb, 0, s>>>(m.ne, m.A, m.PinvT, c1[k], c2[k], r, st.cur, st.prev,
                                                             out, ctl);
            st.advance(out);
        }
        ++launches;
    }
    return launches;
}

template int mg_apply_n<4>(const MGPlan&, const double*, double*, const int*, cudaStream_t);
template int mg_apply_n<9>(const MGPlan&, const double*, double*, const int*, cudaStream_t);
template int mg_apply_n<16>(const MGPlan&, const double*, double*, const int*, cudaStream_t);
template int mg_apply_n<25>(const MGPlan&, const double*, double*, const int*, cudaStream_t);

// The V-cycle part of one flexible-CG iteration with the CG vector work
// folded into its first and last level-0 steps (bj_first_update_kernel,
// bj_last_dots_kernel); z = M r as mg_apply computes it, for the residual r
// after the update.
template <int N>
int mg_cg_iteration_n(const MGPlan& m, const CGArgs& a, cudaStream_t s) {
    const int tpb = cg_threads_per_block(N);
    const int nblkR = (m.ne + FaceDims<N>::EPB * kSmoothRows - 1) / (FaceDims<N>::EPB * kSmoothRows);
    float c1[4], c2[4];
    smoother_coeffs(m, c1, c2);
    SmoothState st{m.x0, nullptr, m.x0b};
    bj_first_update_kernel<N, kSmoothRows><<<nblkR, tpb, 0, s>>>(a, m.PinvT, c2[0], st.cur);
    int launches = 1;
    for (int k = 1; k < m.nu0; ++k) {
        float* out = st.next();
        bj_smooth_kernel<float, N, kSmoothRows><<<nblkR, tpb, 0, s>>>(m.ne, m.A, m.PinvT, c1[k], c2[k], a.r, st.cur, st.prev, out,
                                                         a.ctl);
        st.advance(out);
        ++launches;
    }
    bj_residual_kernel<N, kSmoothRows><<<nblkR, tpb, 0, s>>>(m.ne, m.A, m.WdT, a.r, st.cur, m.w4, m.res0,
                                                           m.coarse_pf, m.coarse_npf, a.ctl);
    int lc = 0;
    const float* coarse_out = launch_coarse_cycle(m, m.res0, a.ctl, s, &lc);
    const int rows0 = m.ne * N;
    prolong_q1_kernel<<<(rows0 + 255) / 256, 256, 0, s>>>(m.ne, N, m.vid, m.w4, coarse_out, st.cur, a.ctl);
    launches += 2 + lc;
    st.prev = nullptr;
    for (int k = 0; k < m.nu0; ++k) {
        if (k == m.nu0 - 1) {
            bj_last_dots_kernel<N, kSmoothRows><<<nblkR, tpb, 0, s>>>(a, m.A, m.PinvT, c1[k], c2[k], st.cur, st.prev);
        } else {
            float* out = st.next();
            bj_smooth_kernel<float, N, kSmoothRows><<<nblkR, tpb, 0, s>>>(m.ne, m.A, m.PinvT, c1[k], c2[k], a.r, st.cur, st.prev,
                                                             out, a.ctl);
            st.advance(out);
        }
        ++launches;
    }
    return launches;
}

int mg_cg_iteration(const MGPlan& m, const CGArgs& a, cudaStream_t s) {
    switch (m.n) {
        case 4: return mg_cg_iteration_n<4>(m, a, s);
        case 9: return mg_cg_iteration_n<9>(m, a, s);
        case 16: return mg_cg_iteration_n<16>(m, a, s);
        case 25: return mg_cg_iteration_n<25>(m, a, s);
        default: return 0;
    }
}

}  // namespace smm

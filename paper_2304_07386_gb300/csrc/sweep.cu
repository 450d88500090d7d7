// Persistent wavefront DG S_N sweep (paper Sec. "Transport Discretization").
//
// One warp per (element, ordinate) task; the row i of the local system is
// held by lane i (n = (p+1)^2 <= 25 <= 32).  The local upwind DG operator
//   A = sigma_t M - Omega_x Gx - Omega_y Gy + sum_{outflow f} (Omega_x Fx_f + Omega_y Fy_f)
// is assembled on the fly from the element's angle-independent matrices, the
// right-hand side b = M s - sum_{inflow f} (Omega_x Fx_f + Omega_y Fy_f) psi_up
// takes the upwind neighbour's face values (or the inflow data), and A is
// factored in registers by Gaussian elimination without pivoting (the
// symmetric part of A is positive definite: x^T A x = 1/2 int_dK |Omega.n| x^2
// + sigma_t |x|^2), broadcasting pivot rows with warp shuffles.
//
// Scheduling: tasks are sorted by upwind level and dealt round-robin to the
// warps of a cooperative (co-resident) launch.  A task waits (bounded in
// time) on its upwind neighbours' epoch flags, and publishes its own flag
// with release semantics after its outputs are written.
#include <algorithm>

#include "dfloat.cuh"
#include "kernels.cuh"

namespace smm {

namespace {

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Bounded wait until *flag == epoch.  False on timeout or when another warp
// has already raised the error word.
__device__ bool wait_epoch(const unsigned* flag, unsigned epoch, long long timeout_ns, const int* err) {
    if (ld_acquire(flag) == epoch) return true;
    const long long t0 = global_ns();
    for (unsigned it = 1; it < (1u << 30); ++it) {
        if (ld_acquire(flag) == epoch) return true;
        if ((it & 31u) == 0) {
            if (ld_volatile(err) != DEV_OK) return false;
            if (global_ns() - t0 > timeout_ns) return false;
        }
        __nanosleep(32);
    }
    return false;
}

template <int P>
__device__ __forceinline__ int face_node(int f, int a) {
    constexpr int P1 = P + 1;
    return f == 0 ? a : (f == 1 ? a * P1 + P : (f == 2 ? P * P1 + a : a * P1));
}

template <typename T> __device__ __forceinline__ T ldg_cg(const T* p) { return __ldcg(p); }


}  // namespace

// Moments of element e (Eqs. correction_tensor_disc, broken_Tdiv and
// bdr_correction_factor_disc), formed after the sweep's last task:
//   phi = sum_d w_d psi_d, J = sum_d w_d Omega_d psi_d,
//   T = sum_d w_d Omega_d Omega_d psi_d - phi/3 I        (lane = node),
// accumulated over the ordinates in a fixed order (so the result does not
// depend on which warp forms it), as FP32 pairs against the pair weights in
// FP64 cached mode (split over lane groups for n <= 16) and in FP64 otherwise
// (index order); then, at the Gauss points of each
// boundary face, beta = sum_d w_d |Omega_d . n| psi_d - E_b0 phi (lanes over
// the ordinates, a fixed-order butterfly sum).  The flux loads are issued
// eight ordinates at a time.
template <typename T, int P, bool DF>
__device__ __noinline__ void element_moments(const SweepArgs<T>& a, const int e) {
    constexpr int P1 = P + 1, N = P1 * P1;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int row = lane < N ? lane : 0;
    const int nd = a.nd;
    const size_t st = (size_t)a.ne * N, o = (size_t)e * N + row;
    constexpr int B = 8;  // ordinates whose loads are in flight together
    double phi;
    if constexpr (DF) {
        // with n <= 16 the lanes form KG = 32 / n groups of n rows; group g sums
        // the ordinates d = g (mod KG) and the groups' partial sums are added in
        // group order (p = 4: one group, every ordinate in index order)
        constexpr int KG = 32 / N;
        const int g = KG == 1 ? 0 : (lane < KG * N ? lane / N : KG);
        const int r = KG == 1 ? row : (lane < KG * N ? lane - (lane / N) * N : 0);
        float s[6] = {0, 0, 0, 0, 0, 0}, c[6] = {0, 0, 0, 0, 0, 0};
        const float2* ps = a.psi2 + (size_t)e * nd * N + r;
        if constexpr (KG == 1) {
            for (int d0 = 0; d0 < nd; d0 += B) {
                float2 v[B];
#pragma unroll
                for (int k = 0; k < B; ++k)
                    v[k] = d0 + k < nd ? __ldcg(ps + (size_t)(d0 + k) * N) : make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    if (d0 + k >= nd) break;
#pragma unroll
                    for (int m = 0; m < 6; ++m) {
                        const float2 wk = a.wq2[m * nd + d0 + k];
                        df_acc(s[m], c[m], wk.x, wk.y, v[k].x, v[k].y);
                    }
                }
            }
        } else {
            for (int d0 = 0; d0 < nd; d0 += B * KG) {
                float2 v[B];
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const int d = d0 + k * KG + g;
                    v[k] = g < KG && d < nd ? __ldcg(ps + (size_t)d * N) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const int d = d0 + k * KG + g;
                    if (g >= KG || d >= nd) continue;
#pragma unroll
                    for (int m = 0; m < 6; ++m) {
                        const float2 wk = a.wq2[m * nd + d];
                        df_acc(s[m], c[m], wk.x, wk.y, v[k].x, v[k].y);
                    }
                }
            }
        }
        if constexpr (KG > 1) {
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                float ts = __shfl_sync(FULL, s[m], r), tc = __shfl_sync(FULL, c[m], r);
#pragma unroll
                for (int gg = 1; gg < KG; ++gg)
                    df_add(ts, tc, __shfl_sync(FULL, s[m], r + gg * N), __shfl_sync(FULL, c[m], r + gg * N));
                s[m] = ts;
                c[m] = tc;
            }
        }
        phi = df_to_double(s[0], c[0]);
        if (lane < N) {
            a.mom[o] = phi;
            a.mom[st + o] = df_to_double(s[1], c[1]);
            a.mom[2 * st + o] = df_to_double(s[2], c[2]);
            a.mom[3 * st + o] = df_to_double(s[3], c[3]) - phi / 3.0;
            a.mom[4 * st + o] = df_to_double(s[4], c[4]);
            a.mom[5 * st + o] = df_to_double(s[5], c[5]) - phi / 3.0;
        }
    } else {
        double jx = 0, jy = 0, pxx = 0, pxy = 0, pyy = 0;
        phi = 0;
        const double* ps = a.mpsi + (size_t)e * nd * N + row;
        for (int d0 = 0; d0 < nd; d0 += B) {
            double v[B];
#pragma unroll
            for (int k = 0; k < B; ++k) v[k] = d0 + k < nd ? __ldcg(ps + (size_t)(d0 + k) * N) : 0.0;
#pragma unroll
            for (int k = 0; k < B; ++k) {
                if (d0 + k >= nd) break;
                const int d = d0 + k;
                const double wv = a.w[d] * v[k], x = a.ox[d], y = a.oy[d];
                phi += wv;
                jx += wv * x;
                jy += wv * y;
                pxx += wv * x * x;
                pxy += wv * x * y;
                pyy += wv * y * y;
            }
        }
        if (lane < N) {
            a.mom[o] = phi;
            a.mom[st + o] = jx;
            a.mom[2 * st + o] = jy;
            a.mom[3 * st + o] = pxx - phi / 3.0;
            a.mom[4 * st + o] = pxy;
            a.mom[5 * st + o] = pyy - phi / 3.0;
        }
    }
    if (!a.beta) return;
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        const int b = a.bface_id[e * 4 + f];  // -1 for interior faces
        if (b < 0) continue;
        // face node q of face f is base + q * stride
        const int base = f == 1 ? P : (f == 2 ? P * P1 : 0);
        const int stride = (f == 0 || f == 2) ? 1 : P1;
#pragma unroll 1
        for (int q = 0; q < a.nfq; ++q) {
            const int t = b * a.nfq + q;
            const double* Lq = a.L1 + q * P1;
            const double nx = a.nhat[2 * t], ny = a.nhat[2 * t + 1];
            double B = 0.0;
            for (int d = lane; d < nd; d += 32) {
                double v = 0.0;
#pragma unroll
                for (int k = 0; k < P1; ++k) {
                    const size_t pi = ((size_t)e * nd + d) * N + base + k * stride;
                    double pv;
                    if constexpr (DF) {
                        const float2 pp = __ldcg(a.psi2 + pi);
                        pv = (double)pp.x + (double)pp.y;
                    } else {
                        pv = __ldcg(a.mpsi + pi);
                    }
                    v += Lq[k] * pv;
                }
                B += a.w[d] * fabs(a.ox[d] * nx + a.oy[d] * ny) * v;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) B += __shfl_xor_sync(FULL, B, off);
            double ph = 0.0;
#pragma unroll
            for (int k = 0; k < P1; ++k) ph += Lq[k] * __shfl_sync(FULL, phi, base + k * stride);
            if (lane == 0) a.beta[t] = B - a.eb0[t] * ph;
        }
    }
}

// Grid-wide gate between the sweep's tasks and its moment reductions: every
// warp arrives after its last task and waits (bounded) until all warps have.
// Reductions started while the wavefront's last levels still run would take
// issue slots from their latency-bound tasks.  Returns false if the wait gave
// up or a task's wait did; every warp arrives either way.
__device__ bool sweep_gate(unsigned* gate, unsigned warps, long long timeout_ns, int* err) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    if (lane == 0) {
        __threadfence();
        atomicAdd(gate, 1u);
        if (ld_acquire(gate) != warps) {
            const long long t0 = global_ns();
            ok = false;
            for (unsigned it = 1; it < (1u << 30); ++it) {
                if (ld_acquire(gate) == warps) {
                    ok = true;
                    break;
                }
                if ((it & 31u) == 0 && global_ns() - t0 > timeout_ns) break;
                __nanosleep(256);
            }
            if (!ok) atomicCAS(err, DEV_OK, DEV_TIMEOUT);
        }
        ok = ok && ld_volatile(err) == DEV_OK;
    }
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// One (element, ordinate) task of one problem, executed by a whole warp.
// Returns false if a dependency wait gave up.  EXT compiles in the optional
// parts (negative flux fixup, lagged inflow of a block Jacobi sweep); without
// it the kernel carries neither branch.
template <typename T, int P, int MODE, bool INV, bool EXT>
__device__ __forceinline__ bool sweep_task(const SweepArgs<T>& a, const int task) {
    constexpr int P1 = P + 1, N = P1 * P1;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int row = lane < N ? lane : 0;  // lanes >= N shadow row 0 (results discarded)
    const int ix = row % P1, iy = row / P1;
    const int nd = a.nd;
    {
        const int e = task / nd, d = task - e * nd;
        const T ox = (T)a.ox[d], oy = (T)a.oy[d];
        const char4 dirs = *reinterpret_cast<const char4*>(a.fdir + ((size_t)e * nd + d) * 4);
        const int dir[4] = {dirs.x, dirs.y, dirs.z, dirs.w};

        // ---- cached mode: everything that does not depend on upwind data is
        //      loaded before the wait, so HBM latency overlaps the wavefront ----
        // FP64 cached mode keeps the inverse as FP32 pairs and forms
        // y0 = A^{-1} b_pre (the part of the solution without upwind data)
        // before the wait; after it only the inflow-face columns are added.
        // With n <= 16 the warp's lanes form KG = 32 / n groups of n rows;
        // group g holds columns [g CPG, (g + 1) CPG) of its row of A^{-1} and
        // accumulates their terms, and the groups' partial sums are added in
        // group order at the end (p = 4: one group, the plain row per lane).
        constexpr bool DF = INV && sizeof(T) == 8;
        constexpr int KG = DF ? 32 / N : 1, CPG = (N + KG - 1) / KG;
        // one group: lanes >= n shadow row 0, as in the other modes
        const int dgrp = KG == 1 ? 0 : (lane < KG * N ? lane / N : KG);  // KG: no columns
        const int drow = KG == 1 ? row : (lane < KG * N ? lane - (lane / N) * N : 0);
        T Ainv[(INV && !DF) ? N : 1];
        float2 Adf[DF ? CPG : 1];
        T bpre = 0;
        float ys = 0.0f, yc = 0.0f;  // DF: running pair sum of this lane's columns' terms
        if (INV) {
            if constexpr (DF) {
                const float2* Ai = a.ainv_df + (size_t)task * N * N + drow;
#pragma unroll
                for (int jj = 0; jj < CPG; ++jj) {
                    const int j = dgrp * CPG + jj;
                    Adf[jj] = KG == 1 || j < N ? Ai[(size_t)j * N] : make_float2(0.0f, 0.0f);
                }
            } else {
                const T* Ai = a.ainv + (size_t)task * N * N + row;
#pragma unroll
                for (int j = 0; j < (DF ? 1 : N); ++j) Ainv[j] = Ai[(size_t)j * N];
            }
            if constexpr (DF) {
                // b_pre = M s (+ M q_d) as pairs, y0 = A^{-1} b_pre
                float2 bp;
                if (MODE == SWEEP_SOURCE) {
                    bp = a.msrc2[(size_t)e * N + row];
                    if (a.mq2) {
                        const float2 qv = a.mq2[((size_t)e * nd + d) * N + row];
                        float s0 = bp.x, c0 = bp.y;
                        df_add(s0, c0, qv.x, qv.y);
                        bp = df_norm(s0, c0);
                    }
                } else {
                    bp = make_float2(a.rhs[((size_t)e * nd + d) * N + row], 0.0f);
                }
                // (a zero entry adds an exact zero: the sums are unchanged)
#pragma unroll
                for (int jj = 0; jj < CPG; ++jj) {
                    const int j = KG == 1 ? jj : min(dgrp * CPG + jj, N - 1);
                    df_acc(ys, yc, Adf[jj].x, Adf[jj].y, __shfl_sync(FULL, bp.x, j), __shfl_sync(FULL, bp.y, j));
                }
            } else if (MODE == SWEEP_SOURCE) {
                double bs = a.msrc[(size_t)e * N + row];
                if (a.mq) bs += a.mq[((size_t)e * nd + d) * N + row];
                bpre = (T)bs;
            } else {
                bpre = (T)a.rhs[((size_t)e * nd + d) * N + row];
            }
        }

        // ---- DF: each inflow face's coefficient entry (lane (a, c)) and the
        //      index of its upwind value, formed before the wait; boundary
        //      faces are finished here (ui = -2: cf holds coef * inflow) ----
        //      (p = 4 and the kernel with the optional parts; p <= 3 otherwise packs
        //      its inflow faces below)
        constexpr int FG = 32 / (P1 * P1);            // faces whose lanes fit the warp at once
        constexpr bool FPK = DF && !EXT && FG >= 2;
        float2 cf[4];
        int ui[4];
        unsigned lagm = 0;
        if constexpr (DF && !FPK) {
            const int la = lane / P1, lc = lane - (lane / P1) * P1;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const int df = dir[f];
                cf[f] = make_float2(0.0f, 0.0f);
                ui[f] = -1;
                if ((df < 0 || (EXT && df >= 2)) && lane < P1 * P1) {
                    float2 coef;
                    if (EXT && df >= 2) {
                        coef = a.fmix2[((size_t)a.fmix_id[((size_t)e * nd + d) * 4 + f] * 2 + 1) * P1 * P1 + la * P1 + lc];
                    } else {
                        const size_t fo2 = ((size_t)e * 4 + f) * P1 * P1 + la * P1 + lc;
                        const float2 fx = a.Fx2[fo2], fy = a.Fy2[fo2], o2x = a.ox2[d], o2y = a.oy2[d];
                        float cs = 0.0f, cc = 0.0f;
                        df_acc(cs, cc, o2x.x, o2x.y, fx.x, fx.y);
                        df_acc(cs, cc, o2y.x, o2y.y, fy.x, fy.y);
                        coef = df_norm(cs, cc);
                    }
                    cf[f] = coef;
                    const int nb = a.nbr[e * 4 + f];
                    if (nb >= 0) {
                        const int f2 = a.nbr_face[e * 4 + f];
                        const int c2 = a.nbr_flip[e * 4 + f] ? P - lc : lc;
                        const int node = f2 == 0 ? c2 : (f2 == 1 ? c2 * P1 + P : (f2 == 2 ? P * P1 + c2 : c2 * P1));
                        ui[f] = (int)(((size_t)nb * nd + d) * N + node);
                        if (EXT && (df == -2 || df == 3)) lagm |= 1u << f;
                    } else if (MODE == SWEEP_SOURCE && a.inflow2) {
                        const int bi = a.bface_id[e * 4 + f];
                        const float2 u = a.inflow2[((size_t)bi * nd + d) * P1 + lc];
                        float ts = 0.0f, tc = 0.0f;
                        df_acc(ts, tc, coef.x, coef.y, u.x, u.y);
                        cf[f] = df_norm(ts, tc);
                        ui[f] = -2;
                    }
                }
            }
        }

        // ---- packed inflow faces (FP64 cached mode, p <= 3, no optional parts):
        //      the task's inflow faces (at most three) are dealt to the FG lane
        //      groups of (p+1)^2 lanes, one face per group and round; lane
        //      (h, a, c) of group h forms face f_h's coefficient coef[a][c] and
        //      the index of its upwind value, so all faces' products and sums
        //      over c run in the same instructions ----
        constexpr int RMAX = FPK ? (3 + FG - 1) / FG : 1;
        unsigned flist = 0;  // the inflow faces in order, two bits each
        int nin = 0;
        float2 cfp[RMAX];
        int uip[RMAX];
        if constexpr (FPK) {
#pragma unroll
            for (int f = 0; f < 4; ++f)
                if (dir[f] == -1) flist |= (unsigned)f << (2 * nin++);
            const int h = lane / (P1 * P1), la = (lane % (P1 * P1)) / P1, lc = lane % P1;
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                const int sl = r * FG + h;
                cfp[r] = make_float2(0.0f, 0.0f);
                uip[r] = -1;
                if (h < FG && sl < nin) {
                    const int f = (flist >> (2 * sl)) & 3;
                    const size_t fo2 = ((size_t)e * 4 + f) * P1 * P1 + la * P1 + lc;
                    const float2 fx = a.Fx2[fo2], fy = a.Fy2[fo2], o2x = a.ox2[d], o2y = a.oy2[d];
                    float cs = 0.0f, cc = 0.0f;
                    df_acc(cs, cc, o2x.x, o2x.y, fx.x, fx.y);
                    df_acc(cs, cc, o2y.x, o2y.y, fy.x, fy.y);
                    const float2 coef = df_norm(cs, cc);
                    cfp[r] = coef;
                    const int nb = a.nbr[e * 4 + f];
                    if (nb >= 0) {
                        const int f2 = a.nbr_face[e * 4 + f];
                        const int c2 = a.nbr_flip[e * 4 + f] ? P - lc : lc;
                        const int node = f2 == 0 ? c2 : (f2 == 1 ? c2 * P1 + P : (f2 == 2 ? P * P1 + c2 : c2 * P1));
                        uip[r] = (int)(((size_t)nb * nd + d) * N + node);
                    } else if (MODE == SWEEP_SOURCE && a.inflow2) {
                        const float2 u = a.inflow2[((size_t)a.bface_id[e * 4 + f] * nd + d) * P1 + lc];
                        float ts = 0.0f, tc = 0.0f;
                        df_acc(ts, tc, coef.x, coef.y, u.x, u.y);
                        cfp[r] = df_norm(ts, tc);
                        uip[r] = -2;
                    }
                }
            }
        }

        // ---- wait for the upwind neighbours (lane f waits on face f) ----
        bool ok = true;
        if (lane < 4) {
            const int f = lane;
            const int df = f == 0 ? dir[0] : (f == 1 ? dir[1] : (f == 2 ? dir[2] : dir[3]));
            const int nb = a.nbr[e * 4 + f];
            // (-2, 3: lagged inflow, taken from the previous sweep)
            if ((df == -1 || (EXT && df == 2)) && nb >= 0)
                ok = wait_epoch(a.done + (size_t)nb * nd + d, a.epoch, a.timeout_ns, a.err);
        }
        ok = __all_sync(FULL, ok);
        if (!ok) {
            if (lane == 0) atomicCAS(a.err, DEV_OK, DEV_TIMEOUT);
            return false;
        }

        // ---- right-hand side b (and, without cached inverses, row `row` of A) ----
        const T sig = (T)a.sigma_t[e];
        const size_t mo = ((size_t)e * N + row) * N;
        T A[INV ? 1 : N];
        if (!INV) {
#pragma unroll
            for (int j = 0; j < N; ++j) A[j] = sig * a.M[mo + j] - ox * a.Gx[mo + j] - oy * a.Gy[mo + j];
        }
        T b;
        if (INV) {
            b = bpre;
        } else if (MODE == SWEEP_SOURCE) {
            {
                const double c = a.sigma_s[e] * (1.0 / (4.0 * 3.14159265358979323846));
                const double* q = a.src_angular ? a.src + ((size_t)e * nd + d) * N : a.src + (size_t)e * N;
                T sj = 0;
                if (lane < N) sj = (T)((a.phi ? c * a.phi[(size_t)e * N + lane] : 0.0) + q[lane]);
                T acc = 0;
#pragma unroll
                for (int j = 0; j < N; ++j) acc += a.M[mo + j] * __shfl_sync(FULL, sj, j);
                b = acc;
            }
        } else {
            b = (T)a.rhs[((size_t)e * nd + d) * N + row];
        }

        if constexpr (FPK) {
            // every round's upwind values, loaded together; per round the
            // product, the sum over c within each group of p+1 lanes (valid at
            // lane (h, a, 0)), then every row adds -A^{-1}[row][node(f, a)] v_a
            float2 upp[RMAX], vr[RMAX];
#pragma unroll
            for (int r = 0; r < RMAX; ++r) upp[r] = uip[r] >= 0 ? __ldcg(a.psi2 + uip[r]) : make_float2(0.0f, 0.0f);
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                float2 t;
                if (uip[r] == -2) {
                    t = cfp[r];
                } else {
                    float ts = 0.0f, tc = 0.0f;
                    df_acc(ts, tc, cfp[r].x, cfp[r].y, upp[r].x, upp[r].y);
                    t = df_norm(ts, tc);
                }
                float vs = t.x, vc = t.y;
#pragma unroll
                for (int k = 1; k < P1; ++k)
                    df_add(vs, vc, __shfl_down_sync(FULL, t.x, k), __shfl_down_sync(FULL, t.y, k));
                vr[r] = df_norm(vs, vc);
            }
            int sl = 0;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (dir[f] != -1) continue;
                const int base = (sl % FG) * P1 * P1;
                const float2 v = sl < FG ? vr[0] : vr[RMAX - 1];
#pragma unroll
                for (int aa = 0; aa < P1; ++aa) {
                    const int cn = face_node<P>(f, aa);
                    const float2 col = cn / CPG == dgrp ? Adf[cn % CPG] : make_float2(0.0f, 0.0f);
                    df_acc(ys, yc, -col.x, -col.y, __shfl_sync(FULL, v.x, base + aa * P1),
                           __shfl_sync(FULL, v.y, base + aa * P1));
                }
                ++sl;
            }
        }
        // DF: every inflow face's upwind value, loaded together
        float2 up[4];
        if constexpr (DF && !FPK) {
#pragma unroll
            for (int f = 0; f < 4; ++f)
                up[f] = ui[f] >= 0 ? __ldcg((EXT && ((lagm >> f) & 1u) ? a.psi2_lag : a.psi2) + ui[f])
                                   : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const int df = dir[f];
            const bool on = (f == 0 && iy == 0) || (f == 1 && ix == P) || (f == 2 && iy == P) || (f == 3 && ix == 0);
            const int fa = (f == 0 || f == 2) ? ix : iy;  // position of this row on face f
            const size_t fo = (((size_t)e * 4 + f) * P1 + fa) * P1;
            if (!INV && (df == 1 || (EXT && df >= 2)) && on) {
                const double* fm =
                    EXT && df >= 2 ? a.fmix + ((size_t)a.fmix_id[((size_t)e * nd + d) * 4 + f] * 2 * P1 + fa) * P1
                                   : nullptr;
#pragma unroll
                for (int c = 0; c < P1; ++c) {
                    const T v = fm ? (T)fm[c] : ox * a.Fx[fo + c] + oy * a.Fy[fo + c];
#pragma unroll
                    for (int j = 0; j < (INV ? 1 : N); ++j)
                        if (j == face_node<P>(f, c)) A[j] += v;
                }
            }
            if (DF && !FPK && (df < 0 || (EXT && df >= 2))) {
                // inflow face in pairs: lane (a, c) forms coef[a][c] u[c], the
                // p+1 lanes of group a sum over c, and every row adds
                // -A^{-1}[row][node(f, a)] v_a
                float2 t;
                if (ui[f] == -2) {
                    t = cf[f];
                } else {
                    float ts = 0.0f, tc = 0.0f;
                    df_acc(ts, tc, cf[f].x, cf[f].y, up[f].x, up[f].y);
                    t = df_norm(ts, tc);
                }
                float vs = t.x, vc = t.y;
#pragma unroll
                for (int k = 1; k < P1; ++k)
                    df_add(vs, vc, __shfl_down_sync(FULL, t.x, k), __shfl_down_sync(FULL, t.y, k));
                const float2 v = df_norm(vs, vc);
#pragma unroll
                for (int aa = 0; aa < P1; ++aa) {
                    const int cn = face_node<P>(f, aa);
                    const float2 col =
                        KG == 1 ? Adf[cn] : (cn / CPG == dgrp ? Adf[cn % CPG] : make_float2(0.0f, 0.0f));
                    df_acc(ys, yc, -col.x, -col.y, __shfl_sync(FULL, v.x, aa * P1), __shfl_sync(FULL, v.y, aa * P1));
                }
            } else if (!DF && (df < 0 || (EXT && df >= 2))) {
                // inflow face (warp-uniform branch): the (p+1)^2 products
                // coef[a][c] * psi_up[c] are spread over lanes (a, c), summed
                // over c within each group of p+1 lanes, and handed to the lane
                // of face node a -- every lane does useful FP64 work
                const int la = lane / P1, lc = lane - (lane / P1) * P1;
                T term = 0;
                if (lane < P1 * P1) {
                    const size_t fo2 = ((size_t)e * 4 + f) * P1 * P1 + la * P1 + lc;
                    const T coef = EXT && df >= 2
                                       ? (T)a.fmix[((size_t)a.fmix_id[((size_t)e * nd + d) * 4 + f] * 2 + 1) * P1 * P1 +
                                                   la * P1 + lc]
                                       : ox * a.Fx[fo2] + oy * a.Fy[fo2];
                    const int nb = a.nbr[e * 4 + f];
                    T upv = 0;
                    if (nb >= 0) {
                        const int f2 = a.nbr_face[e * 4 + f];
                        const int c2 = a.nbr_flip[e * 4 + f] ? P - lc : lc;
                        const int node = f2 == 0 ? c2 : (f2 == 1 ? c2 * P1 + P : (f2 == 2 ? P * P1 + c2 : c2 * P1));
                        upv = ldg_cg((EXT && (df == -2 || df == 3) ? a.psi_lag : a.psi) + ((size_t)nb * nd + d) * N + node);
                    } else if (MODE == SWEEP_SOURCE && a.inflow) {
                        const int bi = a.bface_id[e * 4 + f];
                        upv = (T)a.inflow[((size_t)bi * nd + d) * P1 + lc];
                    }
                    term = coef * upv;
                }
                T sum = term;
#pragma unroll
                for (int k = 1; k < P1; ++k) sum += __shfl_down_sync(FULL, term, k);
                const T v = __shfl_sync(FULL, sum, fa * P1);
                if (on) b -= v;
            }
        }

        T x = 0;
        if (INV) {
            if constexpr (DF) {
                if constexpr (KG > 1) {
                    // the row's full sum: its groups' partial sums in group order
                    float ts = __shfl_sync(FULL, ys, drow), tc = __shfl_sync(FULL, yc, drow);
#pragma unroll
                    for (int g = 1; g < KG; ++g)
                        df_add(ts, tc, __shfl_sync(FULL, ys, drow + g * N), __shfl_sync(FULL, yc, drow + g * N));
                    ys = ts;
                    yc = tc;
                }
                x = (T)((double)ys + (double)yc);
            } else {
                // ---- cached inverse: x = A^{-1} b ----
#pragma unroll
                for (int j = 0; j < ((INV && !DF) ? N : 1); ++j) x += Ainv[j] * __shfl_sync(FULL, b, j);
            }
        } else {
            // ---- in-register LU without pivoting (row per lane) ----
            T dinv = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const T inv = T(1) / __shfl_sync(FULL, A[k < (INV ? 1 : N) ? k : 0], k);
                if (lane == k) dinv = inv;
                const T l = A[k < (INV ? 1 : N) ? k : 0] * inv;
                const bool below = lane > k;
#pragma unroll
                for (int j = 0; j < (INV ? 1 : N); ++j) {
                    if (j > k) {
                        const T akj = __shfl_sync(FULL, A[j], k);
                        if (below) A[j] -= l * akj;
                    }
                }
                const T bk = __shfl_sync(FULL, b, k);
                if (below) b -= l * bk;
            }
            // back substitution with the stored pivot reciprocals
#pragma unroll
            for (int k = N - 1; k >= 0; --k) {
                const T xk = __shfl_sync(FULL, b * dinv, k);
                if (lane == k) x = xk;
                if (lane < k) b -= A[k < (INV ? 1 : N) ? k : 0] * xk;
            }
        }

        // ---- zero and scale negative flux fixup (source mode): negative nodal
        //      values are zeroed and the rest scaled so that the element balance
        //      c . x, c = 1^T A (column sums of the local operator), keeps its
        //      value; warp-uniform branch, taken only when a value is negative ----
        bool fixed = false;
        if (EXT && MODE == SWEEP_SOURCE && a.fixup && __any_sync(FULL, lane < N && x < T(0))) {
            double c = 0.0;
            if (lane < N) {
                const size_t eo = (size_t)e * N + lane;
                c = a.sigma_t[e] * a.colM[eo] - a.ox[d] * a.colGx[eo] - a.oy[d] * a.colGy[eo];
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const bool on = (f == 0 && iy == 0) || (f == 1 && ix == P) || (f == 2 && iy == P) ||
                                    (f == 3 && ix == 0);
                    if (dir[f] > 0 && on) {
                        const int fa = (f == 0 || f == 2) ? ix : iy;
                        const size_t fo = ((size_t)e * 4 + f) * P1 + fa;
                        c += a.ox[d] * a.colFx[fo] + a.oy[d] * a.colFy[fo];
                    }
                }
            }
            const double xv = lane < N ? (double)x : 0.0, xp = xv > 0.0 ? xv : 0.0;
            double t = c * xv, tp = c * xp;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                t += __shfl_xor_sync(FULL, t, o);
                tp += __shfl_xor_sync(FULL, tp, o);
            }
            const double alpha = (t > 0.0 && tp > 0.0) ? t / tp : 0.0;
            x = (T)(alpha * xp);
            fixed = true;
        }

        // ---- publish ----
        if (lane < N) {
            const size_t o = ((size_t)e * nd + d) * N + lane;
            if constexpr (DF) a.psi2[o] = fixed ? df_make((double)x) : df_norm(ys, yc);
            else a.psi[o] = x;
            if (MODE == SWEEP_RESIDUAL) a.psi_acc[o] += (double)x;
        }
        // the warp barrier orders every lane's stores before lane 0's release
        // store, whose release semantics make them visible to whoever acquires
        // the flag (no separate full fence: it cost 8 % of the sweep)
        __syncwarp();
        if (lane == 0) st_release(a.done + task, a.epoch);
    }
    return true;
}

// Static round-robin schedule: task t of the level-sorted list goes to warp
// t mod W, so each warp meets its tasks in level order; with every warp
// co-resident (cooperative launch) the task a warp waits for is owned by a
// running warp that reaches it after finishing only earlier-level tasks.
// Cached-inverse sweeps: at least three blocks per SM (five for p <= 3, whose
// lanes hold at most eight inverse entries each in column groups).  They are bound by the latency
// of each task's chain of dependent loads, so resident warps set their
// throughput; the moment reduction after the tasks takes any register spills.
// (The in-register LU keeps its registers: it is bound by its FP64 arithmetic.)
template <typename T, int P, int MODE, bool INV, bool EXT>
__global__ void __launch_bounds__(256, INV ? (P <= 3 ? 5 : 3) : 1) sweep_kernel(SweepArgs<T> a) {
    constexpr bool DF = INV && sizeof(T) == 8;
    const int W = (gridDim.x * blockDim.x) >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    bool ok = true;
    for (int t = gw; t < a.ntask && ok; t += W) ok = sweep_task<T, P, MODE, INV, EXT>(a, a.tasks[t]);
    if (!a.mom) return;
    if (!sweep_gate(a.gate, (unsigned)W, a.timeout_ns, a.err) || !ok) return;
    for (int e = gw; e < a.ne; e += W) element_moments<T, P, DF>(a, e);
}

// Many problems in one launch: the merged list holds (problem, task) pairs
// sorted by each problem's own upwind level, and each task dispatches on its
// problem's order p.  The same schedule argument holds: a task's upwind tasks
// belong to its problem, sit at lower levels and so earlier in the list.
// PMAX: the largest order in the batch (3: the p = 4 path is not compiled in,
// so the kernel takes the registers of p <= 3 and five blocks per SM).
template <typename T, int MODE, bool INV, bool EXT, int PMAX>
__global__ void __launch_bounds__(256, INV ? (PMAX <= 3 ? 5 : 3) : 1) batch_sweep_kernel(const SweepArgs<T>* __restrict__ args,
                                                          const int2* __restrict__ tasks, int ntask,
                                                          const int2* __restrict__ elems, int nelem) {
    const int W = (gridDim.x * blockDim.x) >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // EXT: some problem uses the fixup, tiles or lagged / mixed faces
    constexpr bool DF = INV && sizeof(T) == 8;
    bool ok = true;
    for (int t = gw; t < ntask && ok; t += W) {
        const int2 it = tasks[t];
        const SweepArgs<T>& a = args[it.x];
        switch (a.p) {
            case 1: ok = sweep_task<T, 1, MODE, INV, EXT>(a, it.y); break;
            case 2: ok = sweep_task<T, 2, MODE, INV, EXT>(a, it.y); break;
            case 3: ok = sweep_task<T, 3, MODE, INV, EXT>(a, it.y); break;
            default:
                if constexpr (PMAX >= 4) ok = sweep_task<T, 4, MODE, INV, EXT>(a, it.y);
                break;
        }
    }
    if (!args[0].mom) return;
    if (!sweep_gate(args[0].gate, (unsigned)W, args[0].timeout_ns, args[0].err) || !ok) return;
    // every problem's element moments
    for (int k = gw; k < nelem; k += W) {
        const int2 pe = elems[k];
        const SweepArgs<T>& b = args[pe.x];
        switch (b.p) {
            case 1: element_moments<T, 1, DF>(b, pe.y); break;
            case 2: element_moments<T, 2, DF>(b, pe.y); break;
            case 3: element_moments<T, 3, DF>(b, pe.y); break;
            default:
                if constexpr (PMAX >= 4) element_moments<T, 4, DF>(b, pe.y);
                break;
        }
    }
}

// FP64 transport residual r = b - A psi - (inflow terms) per (element,
// ordinate), independent tasks, one warp each (row per lane).
template <int P>
__global__ void __launch_bounds__(256) residual_kernel(ResidualArgs a) {
    constexpr int P1 = P + 1, N = P1 * P1;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int row = lane < N ? lane : 0;
    const int ix = row % P1, iy = row / P1;
    const int nd = a.nd;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int task = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < a.ntask; task += warps) {
        const int e = task / nd, d = task - e * nd;
        const double ox = a.ox[d], oy = a.oy[d];
        const char4 dirs = *reinterpret_cast<const char4*>(a.fdir + (size_t)task * 4);
        const int dir[4] = {dirs.x, dirs.y, dirs.z, dirs.w};
        const double sig = a.sigma_t[e];
        const double c = a.sigma_s[e] * (1.0 / (4.0 * 3.14159265358979323846));
        const double* q = a.src_angular ? a.src + (size_t)task * N : a.src + (size_t)e * N;
        const double* ps = a.psi + (size_t)task * N;
        const double pj = lane < N ? ps[lane] : 0.0;
        const double sj = lane < N ? (a.phi ? c * a.phi[(size_t)e * N + lane] : 0.0) + q[lane] - sig * pj : 0.0;
        const size_t mo = ((size_t)e * N + row) * N;
        double r = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double sjj = __shfl_sync(FULL, sj, j);
            const double pjj = __shfl_sync(FULL, pj, j);
            r += a.M[mo + j] * sjj + (ox * a.Gx[mo + j] + oy * a.Gy[mo + j]) * pjj;
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const int df = dir[f];
            if (df == 0) continue;
            const bool on = (f == 0 && iy == 0) || (f == 1 && ix == P) || (f == 2 && iy == P) || (f == 3 && ix == 0);
            if (!on) continue;
            const int fa = (f == 0 || f == 2) ? ix : iy;
            const size_t fo = (((size_t)e * 4 + f) * P1 + fa) * P1;
            double acc = 0.0;
            if (df > 0) {
#pragma unroll
                for (int cc = 0; cc < P1; ++cc) acc += (ox * a.Fx[fo + cc] + oy * a.Fy[fo + cc]) * ps[face_node<P>(f, cc)];
            } else {
                const int nb = a.nbr[e * 4 + f];
                if (nb >= 0) {
                    const int f2 = a.nbr_face[e * 4 + f], flip = a.nbr_flip[e * 4 + f];
                    const double* up = a.psi + ((size_t)nb * nd + d) * N;
#pragma unroll
                    for (int cc = 0; cc < P1; ++cc) {
                        const int c2 = flip ? P - cc : cc;
                        const int node = f2 == 0 ? c2 : (f2 == 1 ? c2 * P1 + P : (f2 == 2 ? P * P1 + c2 : c2 * P1));
                        acc += (ox * a.Fx[fo + cc] + oy * a.Fy[fo + cc]) * up[node];
                    }
                } else if (a.inflow) {
                    const int bi = a.bface_id[e * 4 + f];
                    const double* up = a.inflow + ((size_t)bi * nd + d) * P1;
#pragma unroll
                    for (int cc = 0; cc < P1; ++cc) acc += (ox * a.Fx[fo + cc] + oy * a.Fy[fo + cc]) * up[cc];
                }
            }
            r -= acc;
        }
        if (lane < N) a.rhs[(size_t)task * N + lane] = (float)r;
    }
}

// Local inverses A_{K,d}^{-1} by Gauss-Jordan elimination without pivoting,
// one warp per task, row per lane; stored column-major per task.
template <typename T, int P>
__global__ void __launch_bounds__(256) invert_kernel(SweepArgs<T> a, T* __restrict__ out, float2* __restrict__ out2) {
    constexpr int P1 = P + 1, N = P1 * P1;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int row = lane < N ? lane : 0;
    const int ix = row % P1, iy = row / P1;
    const int nd = a.nd;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int task = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < a.ntask; task += warps) {
        const int e = task / nd, d = task - e * nd;
        const T ox = (T)a.ox[d], oy = (T)a.oy[d];
        const char4 dirs = *reinterpret_cast<const char4*>(a.fdir + (size_t)task * 4);
        const int dir[4] = {dirs.x, dirs.y, dirs.z, dirs.w};
        const T sig = (T)a.sigma_t[e];
        const size_t mo = ((size_t)e * N + row) * N;
        T A[N], B[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            A[j] = sig * a.M[mo + j] - ox * a.Gx[mo + j] - oy * a.Gy[mo + j];
            B[j] = (j == row) ? T(1) : T(0);
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const bool on = (f == 0 && iy == 0) || (f == 1 && ix == P) || (f == 2 && iy == P) || (f == 3 && ix == 0);
            if (dir[f] > 0 && on) {
                const int fa = (f == 0 || f == 2) ? ix : iy;
                const size_t fo = (((size_t)e * 4 + f) * P1 + fa) * P1;
                // mixed face: the outflow part of its pointwise face matrix
                const double* fm =
                    dir[f] >= 2 ? a.fmix + ((size_t)a.fmix_id[(size_t)task * 4 + f] * 2 * P1 + fa) * P1 : nullptr;
#pragma unroll
                for (int c = 0; c < P1; ++c) {
                    const T v = fm ? (T)fm[c] : ox * a.Fx[fo + c] + oy * a.Fy[fo + c];
#pragma unroll
                    for (int j = 0; j < N; ++j)
                        if (j == face_node<P>(f, c)) A[j] += v;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T l = A[k] / __shfl_sync(FULL, A[k], k);
            const bool other = lane != k;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                if (j > k) {
                    const T akj = __shfl_sync(FULL, A[j], k);
                    if (other) A[j] -= l * akj;
                }
                const T bkj = __shfl_sync(FULL, B[j], k);
                if (other) B[j] -= l * bkj;
            }
        }
        // row `row` of A is now diagonal: divide
        T dg = 0;
#pragma unroll
        for (int j = 0; j < N; ++j)
            if (j == row) dg = A[j];
        const T inv = T(1) / dg;
        if (lane < N) {
            if (out2) {
                float2* o = out2 + (size_t)task * N * N + lane;
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    float hi, lo;
                    df_split((double)(B[j] * inv), hi, lo);
                    o[(size_t)j * N] = make_float2(hi, lo);
                }
            } else {
                T* o = out + (size_t)task * N * N + lane;
#pragma unroll
                for (int j = 0; j < N; ++j) o[(size_t)j * N] = B[j] * inv;
            }
        }
    }
}

// out[t][i] = sum_j M[e][i][j] in[t][j], t = e*nd + d (FP64 sum, stored as an FP32 pair)
__global__ void mass_apply_kernel(int ne, int nd, int n, const double* __restrict__ M, const double* __restrict__ in,
                                  float2* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ne * nd * n) return;
    const long long task = t / n;
    const int i = (int)(t - task * n);
    const int e = (int)(task / nd);
    const double* m = M + ((size_t)e * n + i) * n;
    const double* v = in + (size_t)task * n;
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += m[j] * v[j];
    out[t] = df_make(s);
}

// msrc[e][i] = sum_j M[e][i][j] (sigma_s/(4 pi) phi[e][j] + q[e][j]) (FP64 sum, stored as an FP32 pair)
__global__ void source_kernel(int ne, int n, const double* __restrict__ M, const double* __restrict__ sigma_s,
                              const double* __restrict__ phi, const double* __restrict__ q, float2* __restrict__ msrc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * n) return;
    const int e = t / n, i = t - e * n;
    const double c = sigma_s[e] * (1.0 / (4.0 * 3.14159265358979323846));
    const double* m = M + ((size_t)e * n + i) * n;
    double s = 0.0;
    for (int j = 0; j < n; ++j)
        s += m[j] * ((phi ? c * phi[(size_t)e * n + j] : 0.0) + (q ? q[(size_t)e * n + j] : 0.0));
    msrc[t] = df_make(s);
}

template <typename T, int P, int MODE, bool INV, bool EXT = false>
static void launch_one(const SweepArgs<T>& a, int grid, cudaStream_t s) {
    SweepArgs<T> arg = a;
    void* params[] = {&arg};
    cudaLaunchCooperativeKernel((const void*)sweep_kernel<T, P, MODE, INV, EXT>, dim3(grid), dim3(256), params, 0,
                                s);
}

template <typename T, int P>
static void launch_p(int mode, const SweepArgs<T>& a, int grid, cudaStream_t s) {
    const bool inv = a.ainv != nullptr || a.ainv_df != nullptr;
    if (mode == SWEEP_SOURCE) {
        if constexpr (sizeof(T) == 8) {
            if (a.fixup || a.psi_lag || a.psi2_lag || a.fmix_id) {
                if (inv) launch_one<T, P, SWEEP_SOURCE, true, true>(a, grid, s);
                else launch_one<T, P, SWEEP_SOURCE, false, true>(a, grid, s);
                return;
            }
        }
        if (inv) launch_one<T, P, SWEEP_SOURCE, true>(a, grid, s);
        else launch_one<T, P, SWEEP_SOURCE, false>(a, grid, s);
    } else {
        if (inv) launch_one<T, P, SWEEP_RESIDUAL, true>(a, grid, s);
        else launch_one<T, P, SWEEP_RESIDUAL, false>(a, grid, s);
    }
}

template <typename T>
void launch_sweep(int p, int mode, const SweepArgs<T>& a, int grid, cudaStream_t s) {
    switch (p) {
        case 1: launch_p<T, 1>(mode, a, grid, s); break;
        case 2: launch_p<T, 2>(mode, a, grid, s); break;
        case 3: launch_p<T, 3>(mode, a, grid, s); break;
        case 4: launch_p<T, 4>(mode, a, grid, s); break;
        default: break;
    }
}

template void launch_sweep<double>(int, int, const SweepArgs<double>&, int, cudaStream_t);
template void launch_sweep<float>(int, int, const SweepArgs<float>&, int, cudaStream_t);

static int residual_grid(long long ntask) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = (int)std::min<long long>((ntask + 7) / 8, (long long)sms * 8);
    return grid < 1 ? 1 : grid;
}

// the kernel of a batch: the optional parts only when a problem uses them (FP64 source mode), the p = 4
// path only when a problem has p = 4
template <typename T, int PMAX>
static const void* batch_kernel_pm(int mode, bool cached, bool ext) {
    if (mode == SWEEP_SOURCE) {
        if constexpr (sizeof(T) == 8) {
            if (ext)
                return cached ? (const void*)batch_sweep_kernel<T, SWEEP_SOURCE, true, true, PMAX>
                              : (const void*)batch_sweep_kernel<T, SWEEP_SOURCE, false, true, PMAX>;
        }
        return cached ? (const void*)batch_sweep_kernel<T, SWEEP_SOURCE, true, false, PMAX>
                      : (const void*)batch_sweep_kernel<T, SWEEP_SOURCE, false, false, PMAX>;
    }
    return cached ? (const void*)batch_sweep_kernel<T, SWEEP_RESIDUAL, true, false, PMAX>
                  : (const void*)batch_sweep_kernel<T, SWEEP_RESIDUAL, false, false, PMAX>;
}

template <typename T>
static const void* batch_kernel_of(int mode, bool cached, bool ext, int pmax) {
    return pmax <= 3 ? batch_kernel_pm<T, 3>(mode, cached, ext) : batch_kernel_pm<T, 4>(mode, cached, ext);
}

template <typename T>
cudaError_t launch_batch_sweep(int mode, bool cached, bool ext, int pmax, const SweepArgs<T>* args, const int2* tasks,
                               int ntask, const int2* elems, int nelem, int grid, int block, cudaStream_t s) {
    void* params[] = {(void*)&args, (void*)&tasks, (void*)&ntask, (void*)&elems, (void*)&nelem};
    return cudaLaunchCooperativeKernel(batch_kernel_of<T>(mode, cached, ext, pmax), dim3(grid), dim3(block), params,
                                       0, s);
}

template cudaError_t launch_batch_sweep<double>(int, bool, bool, int, const SweepArgs<double>*, const int2*, int,
                                                const int2*, int, int, int, cudaStream_t);
template cudaError_t launch_batch_sweep<float>(int, bool, bool, int, const SweepArgs<float>*, const int2*, int,
                                               const int2*, int, int, int, cudaStream_t);

int batch_blocks_per_sm(int mode, bool fp32, bool cached, bool ext, int pmax, int block) {
    int nb = 0;
    const void* f = fp32 ? batch_kernel_of<float>(mode, cached, false, pmax)
                         : batch_kernel_of<double>(mode, cached, ext, pmax);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, block, 0);
    return nb;
}

template <typename T>
void launch_invert(int p, const SweepArgs<T>& a, T* out, cudaStream_t s) {
    const int grid = residual_grid(a.ntask);
    switch (p) {
        case 1: invert_kernel<T, 1><<<grid, 256, 0, s>>>(a, out, nullptr); break;
        case 2: invert_kernel<T, 2><<<grid, 256, 0, s>>>(a, out, nullptr); break;
        case 3: invert_kernel<T, 3><<<grid, 256, 0, s>>>(a, out, nullptr); break;
        case 4: invert_kernel<T, 4><<<grid, 256, 0, s>>>(a, out, nullptr); break;
        default: break;
    }
}

void launch_invert_df(int p, const SweepArgs<double>& a, float2* out, cudaStream_t s) {
    const int grid = residual_grid(a.ntask);
    switch (p) {
        case 1: invert_kernel<double, 1><<<grid, 256, 0, s>>>(a, nullptr, out); break;
        case 2: invert_kernel<double, 2><<<grid, 256, 0, s>>>(a, nullptr, out); break;
        case 3: invert_kernel<double, 3><<<grid, 256, 0, s>>>(a, nullptr, out); break;
        case 4: invert_kernel<double, 4><<<grid, 256, 0, s>>>(a, nullptr, out); break;
        default: break;
    }
}

template void launch_invert<double>(int, const SweepArgs<double>&, double*, cudaStream_t);
template void launch_invert<float>(int, const SweepArgs<float>&, float*, cudaStream_t);

__global__ void pairs_to_f64_kernel(size_t n, const float2* __restrict__ in, double* __restrict__ out) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const float2 v = in[t];
        out[t] = (double)v.x + (double)v.y;
    }
}

void launch_pairs_to_f64(size_t n, const float2* in, double* out, cudaStream_t s) {
    if (n) pairs_to_f64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, in, out);
}

void launch_mass_apply(int ne, int nd, int n, const double* M, const double* in, float2* out, cudaStream_t s) {
    const long long tot = (long long)ne * nd * n;
    mass_apply_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ne, nd, n, M, in, out);
}

void launch_source(int ne, int n, const double* M, const double* sigma_s, const double* phi, const double* q_iso,
                   float2* msrc, cudaStream_t s) {
    const int tot = ne * n;
    source_kernel<<<(tot + 255) / 256, 256, 0, s>>>(ne, n, M, sigma_s, phi, q_iso, msrc);
}

int sweep_blocks_per_sm(int p, int mode, bool fp32, bool cached) {
    // FP64 source mode launches either form (with or without the optional
    // parts), so the grid is sized for the one with the lower occupancy
    int nb = 0, nb_ext = 1 << 30;
#define SMM_OCC(T, PP)                                                                                           \
    do {                                                                                                         \
        if (mode == SWEEP_SOURCE) {                                                                              \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                                       \
                &nb, cached ? (const void*)sweep_kernel<T, PP, SWEEP_SOURCE, true, false>                        \
                            : (const void*)sweep_kernel<T, PP, SWEEP_SOURCE, false, false>, 256, 0);             \
            if (sizeof(T) == 8)                                                                                  \
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                                   \
                    &nb_ext, cached ? (const void*)sweep_kernel<double, PP, SWEEP_SOURCE, true, true>            \
                                    : (const void*)sweep_kernel<double, PP, SWEEP_SOURCE, false, true>, 256, 0); \
        } else {                                                                                                 \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                                       \
                &nb, cached ? (const void*)sweep_kernel<T, PP, SWEEP_RESIDUAL, true, false>                      \
                            : (const void*)sweep_kernel<T, PP, SWEEP_RESIDUAL, false, false>, 256, 0);           \
        }                                                                                                        \
    } while (0)
    switch (p) {
        case 1: if (fp32) SMM_OCC(float, 1); else SMM_OCC(double, 1); break;
        case 2: if (fp32) SMM_OCC(float, 2); else SMM_OCC(double, 2); break;
        case 3: if (fp32) SMM_OCC(float, 3); else SMM_OCC(double, 3); break;
        case 4: if (fp32) SMM_OCC(float, 4); else SMM_OCC(double, 4); break;
        default: break;
    }
#undef SMM_OCC
    nb = std::min(nb, nb_ext);
    return nb > 0 ? nb : 1;
}

void launch_residual(int p, const ResidualArgs& a, cudaStream_t s) {
    const int grid = residual_grid(a.ntask);
    switch (p) {
        case 1: residual_kernel<1><<<grid, 256, 0, s>>>(a); break;
        case 2: residual_kernel<2><<<grid, 256, 0, s>>>(a); break;
        case 3: residual_kernel<3><<<grid, 256, 0, s>>>(a); break;
        case 4: residual_kernel<4><<<grid, 256, 0, s>>>(a); break;
        default: break;
    }
}

}  // namespace smm

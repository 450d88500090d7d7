// Multigrid V-cycle preconditioner for the IP-SMM moment operator.
//
// Level 0: DG-p element blocks, nu0 steps of damped element-block Jacobi
// before and after the coarse correction, in FP32 (the preconditioner only
// has to approximate the inverse; FP64 arithmetic on these blocks is bound by
// the GPU's FP64 rate, FP32 by HBM).  The CG around it is flexible, so the
// rounding of the FP32 cycle does not break its recurrences.  Level 1: continuous bilinear
// functions on the mesh vertices (restriction gathers the four corner
// weights of every element node, prolongation interpolates them back).
// Levels 2..: smoothed-aggregation CSR operators with one damped Jacobi
// step before and after; the coarsest level is a dense inverse.  Levels >= 1
// are stored and applied in FP32 and run as one cluster launch.  The cycle
// is symmetric, so it is a valid CG preconditioner.  Every kernel returns at
// once when the CG control word says the solve has finished.
#include <algorithm>

#include <cooperative_groups.h>

#include "blockops.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace smm {

namespace {

// xout = xin + omega Pinv (b - A xin) in FP32; xin == nullptr means xin = 0;
// b is the FP64 right-hand side, xout is FP32 (inner steps) or FP64 (last step)
template <typename OT, int N>
__global__ void __launch_bounds__(256) bj_smooth_kernel(int ne, FaceOp<float> A, const float* __restrict__ PinvT,
                                                        float omega, const double* __restrict__ b,
                                                        const float* __restrict__ xin, OT* __restrict__ xout,
                                                        const int* ctl) {
    if (cg_finished(ctl)) return;
    constexpr int n = N;
    __shared__ float res[256];
    __shared__ FaceScratch<N, float> sc;
    const int epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    const bool act = e < ne;
    float r = 0.0f, x = 0.0f;
    if (xin) {
        const float ax = faceop_row<N, float, float, float>(A, xin, e, i, act, sc);
        if (act) {
            x = xin[(size_t)e * n + i];
            r = (float)b[(size_t)e * n + i] - ax;
        }
    } else if (act) {
        r = (float)b[(size_t)e * n + i];
    }
    res[threadIdx.x] = r;
    __syncthreads();
    if (act) {
        const float* P = PinvT + (size_t)e * n * n + i;
        const float* re = res + (threadIdx.x / n) * n;
        float z = 0.0f;
#pragma unroll
        for (int j = 0; j < n; ++j) z = fmaf(P[j * n], re[j], z);
        xout[(size_t)e * n + i] = (OT)(x + omega * z);
    }
}

// Level-0 residual res = b - A x (FP32) restricted to the element corners:
// cres[e][c] = sum_i w4[i][c] res[e][i] (the vertex level sums these over the
// elements at each vertex)
template <int N>
__global__ void __launch_bounds__(256) bj_residual_kernel(int ne, FaceOp<float> A, const double* __restrict__ b,
                                                          const float* __restrict__ x, const float* __restrict__ w4,
                                                          float* __restrict__ cres, const int* ctl) {
    if (cg_finished(ctl)) return;
    __shared__ FaceScratch<N, float> sc;
    __shared__ float rs[256];
    const int epb = blockDim.x / N;
    const int e = blockIdx.x * epb + threadIdx.x / N, i = threadIdx.x % N;
    const bool act = e < ne;
    const float ax = faceop_row<N, float, float, float>(A, x, e, i, act, sc);
    rs[threadIdx.x] = act ? (float)b[(size_t)e * N + i] - ax : 0.0f;
    __syncthreads();
    if (act && i < 4) {
        const float* re = rs + (threadIdx.x / N) * N;
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) s = fmaf(w4[j * 4 + i], re[j], s);
        cres[(size_t)e * 4 + i] = s;
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
constexpr int kCoarseThreads = 1024;

struct CoarseArgs {
    int nvert, nlev;
    const float* cres;                          // [ne][4] corner sums of the level-0 residual
    const int* vrp; const int* vinc;
    MGLevelDev lv[12];
    const float* cinv;
};

// rows i and j (j < 0: none) of a CSR matrix times x, with the loads of the two
// rows interleaved so a thread holding two rows waits about as long as one
__device__ __forceinline__ void csr_row2_f(const int* __restrict__ rp, const int* __restrict__ ci,
                                           const float* __restrict__ v, const float* x, int i, int j, float& si,
                                           float& sj) {
    int ki = rp[i], kj = j >= 0 ? rp[j] : 0;
    const int ei = rp[i + 1], ej = j >= 0 ? rp[j + 1] : 0;
    float a0 = 0.0f, a1 = 0.0f, b0 = 0.0f, b1 = 0.0f;
    while (ki < ei || kj < ej) {
        int c[8], d[8];
        float w[8], u[8], xv[8], yv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const bool oi = ki + q < ei, oj = kj + q < ej;
            c[q] = oi ? ci[ki + q] : 0;
            w[q] = oi ? v[ki + q] : 0.0f;
            d[q] = oj ? ci[kj + q] : 0;
            u[q] = oj ? v[kj + q] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            xv[q] = ki + q < ei ? __ldcg(x + c[q]) : 0.0f;
            yv[q] = kj + q < ej ? __ldcg(x + d[q]) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            a0 = fmaf(w[q], xv[q], a0);
            a1 = fmaf(w[q + 1], xv[q + 1], a1);
            b0 = fmaf(u[q], yv[q], b0);
            b1 = fmaf(u[q + 1], yv[q + 1], b1);
        }
        ki += 8;
        kj += 8;
    }
    si = a0 + a1;
    sj = b0 + b1;
}

// launched as one cluster of gridDim.x CTAs (8, or 16 where the GPU allows it)
__global__ void __launch_bounds__(kCoarseThreads) coarse_cycle_kernel(CoarseArgs a, const int* ctl) {
    if (cg_finished(ctl)) return;  // uniform over the cluster: no barrier is left waiting
    cg::cluster_group cl = cg::this_cluster();
    const int T = gridDim.x * kCoarseThreads;
    const int tid = blockIdx.x * kCoarseThreads + threadIdx.x;
    // vertex-level right-hand side: sum of the corner sums of the elements at each vertex
    {
        float* b1 = a.lv[1].b;
        for (int v = tid; v < a.nvert; v += T) {
            float s = 0.0f;
            for (int k = a.vrp[v]; k < a.vrp[v + 1]; ++k) s += a.cres[a.vinc[k]];
            b1[v] = s;
        }
    }
    cl.sync();
    // down: x = omega dinv b ; r = b - A x ; b_{l+1} = R r.  The residual is
    // formed as b - As b with As = A diag(omega dinv) (stored), so x and r come
    // out of one pass over b.
    for (int l = 1; l < a.nlev; ++l) {
        const MGLevelDev& L = a.lv[l];
        for (int i = tid; i < L.n; i += 2 * T) {
            const int j = i + T < L.n ? i + T : -1;
            float si, sj;
            csr_row2_f(L.Arp, L.Aci, L.Asv, L.b, i, j, si, sj);
            const float bi = __ldcg(L.b + i);
            L.r[i] = bi - si;
            L.x[i] = L.omega * L.dinv[i] * bi;
            if (j >= 0) {
                const float bj = __ldcg(L.b + j);
                L.r[j] = bj - sj;
                L.x[j] = L.omega * L.dinv[j] * bj;
            }
        }
        cl.sync();
        const MGLevelDev& Lc = a.lv[l + 1];
        for (int i = tid; i < Lc.n; i += 2 * T) {
            const int j = i + T < Lc.n ? i + T : -1;
            float si, sj;
            csr_row2_f(L.Rrp, L.Rci, L.Rv, L.r, i, j, si, sj);
            Lc.b[i] = si;
            if (j >= 0) Lc.b[j] = sj;
        }
        cl.sync();
    }
    // coarsest: x = Cinv b, one warp per row
    {
        const MGLevelDev& C = a.lv[a.nlev];
        const int lane = threadIdx.x & 31, w = tid >> 5, nw = T >> 5;
        for (int row = w; row < C.n; row += nw) {
            const float* cr = a.cinv + (size_t)row * C.n;
            float s = 0.0f;
            for (int j = lane; j < C.n; j += 32) s = fmaf(cr[j], __ldcg(C.b + j), s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) C.x[row] = s;
        }
    }
    cl.sync();
    // up: x += P x_{l+1} ; t = x + omega dinv (b - A x)
    const float* coarse_out = a.lv[a.nlev].x;
    for (int l = a.nlev - 1; l >= 1; --l) {
        const MGLevelDev& L = a.lv[l];
        for (int i = tid; i < L.n; i += 2 * T) {
            const int j = i + T < L.n ? i + T : -1;
            float si, sj;
            csr_row2_f(L.Prp, L.Pci, L.Pv, coarse_out, i, j, si, sj);
            L.x[i] = __ldcg(L.x + i) + si;
            if (j >= 0) L.x[j] = __ldcg(L.x + j) + sj;
        }
        cl.sync();
        for (int i = tid; i < L.n; i += 2 * T) {
            const int j = i + T < L.n ? i + T : -1;
            float si, sj;
            csr_row2_f(L.Arp, L.Aci, L.Av, L.x, i, j, si, sj);
            L.t[i] = __ldcg(L.x + i) + L.omega * L.dinv[i] * (__ldcg(L.b + i) - si);
            if (j >= 0) L.t[j] = __ldcg(L.x + j) + L.omega * L.dinv[j] * (__ldcg(L.b + j) - sj);
        }
        cl.sync();
        coarse_out = L.t;
    }
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
    if (cudaFuncSetAttribute(coarse_cycle_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        cfg.gridDim = dim3(16, 1, 1);
        cfg.blockDim = dim3(kCoarseThreads, 1, 1);
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

const float* launch_coarse_cycle(const MGPlan& m, const float* cres, const int* ctl, cudaStream_t s) {
    CoarseArgs ca{};
    ca.nvert = m.nvert; ca.nlev = m.nlev; ca.cres = cres; ca.vrp = m.vrp; ca.vinc = m.vinc;
    for (int l = 0; l <= m.nlev; ++l) ca.lv[l] = m.lv[l];
    ca.cinv = m.cinv;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(m.coarse_ctas, 1, 1);
    cfg.blockDim = dim3(kCoarseThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = m.coarse_ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, coarse_cycle_kernel, ca, ctl);
    return m.nlev > 1 ? m.lv[1].t : m.lv[1].x;
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

template <int N>
int mg_apply_n(const MGPlan& m, const double* r, double* z, const int* ctl, cudaStream_t s) {
    int launches = 0;
    const int tpb = cg_threads_per_block(N);
    const int nblk0 = (m.ne + tpb / N - 1) / (tpb / N);
    const size_t shm = 0;
    const float w0 = (float)m.omega0;
    // level 0 pre-smoothing from zero (FP32)
    float* xa = m.x0;
    float* xb = m.x0b;
    bj_smooth_kernel<float, N><<<nblk0, tpb, shm, s>>>(m.ne, m.A, m.PinvT, w0, r, nullptr, xa, ctl);
    ++launches;
    for (int k = 1; k < m.nu0; ++k) {
        bj_smooth_kernel<float, N><<<nblk0, tpb, shm, s>>>(m.ne, m.A, m.PinvT, w0, r, xa, xb, ctl);
        std::swap(xa, xb);
        ++launches;
    }
    bj_residual_kernel<N><<<nblk0, tpb, 0, s>>>(m.ne, m.A, r, xa, m.w4, m.res0, ctl);
    // vertex and aggregation levels and the coarsest solve (one cluster launch)
    const float* coarse_out = launch_coarse_cycle(m, m.res0, ctl, s);
    const int rows0 = m.ne * N;
    prolong_q1_kernel<<<(rows0 + 255) / 256, 256, 0, s>>>(m.ne, N, m.vid, m.w4, coarse_out, xa, ctl);
    launches += 3;
    for (int k = 0; k < m.nu0; ++k) {
        if (k == m.nu0 - 1) {
            bj_smooth_kernel<double, N><<<nblk0, tpb, shm, s>>>(m.ne, m.A, m.PinvT, w0, r, xa, z, ctl);
        } else {
            bj_smooth_kernel<float, N><<<nblk0, tpb, shm, s>>>(m.ne, m.A, m.PinvT, w0, r, xa, xb, ctl);
            std::swap(xa, xb);
        }
        ++launches;
    }
    return launches;
}

template int mg_apply_n<4>(const MGPlan&, const double*, double*, const int*, cudaStream_t);
template int mg_apply_n<9>(const MGPlan&, const double*, double*, const int*, cudaStream_t);
template int mg_apply_n<16>(const MGPlan&, const double*, double*, const int*, cudaStream_t);
template int mg_apply_n<25>(const MGPlan&, const double*, double*, const int*, cudaStream_t);

}  // namespace smm

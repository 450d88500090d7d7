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
// step before and after; the coarsest level is a dense inverse.  The cycle
// is symmetric, so it is a valid CG preconditioner.  Every kernel returns at
// once when the CG control word says the solve has finished.
#include <algorithm>

#include "blockops.cuh"
#include "kernels.cuh"

namespace smm {

namespace {

constexpr int kTPB = 256;

inline int blocks_for(int n) { return std::max(1, (n + kTPB - 1) / kTPB); }

// xout = xin + omega Pinv (b - A xin) in FP32; xin == nullptr means xin = 0;
// b is the FP64 right-hand side, xout is FP32 (inner steps) or FP64 (last step)
template <typename OT, int N>
__global__ void __launch_bounds__(256) bj_smooth_kernel(int ne, const float* __restrict__ AdT,
                                                        const float* __restrict__ AoT, const float* __restrict__ PinvT,
                                                        const int32_t* __restrict__ nbr, float omega,
                                                        const double* __restrict__ b, const float* __restrict__ xin,
                                                        OT* __restrict__ xout, const int* ctl) {
    if (cg_finished(ctl)) return;
    constexpr int n = N;
    __shared__ float res[256];
    const int epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    const bool act = e < ne;
    float r = 0.0f, x = 0.0f;
    if (act) {
        r = (float)b[(size_t)e * n + i];
        if (xin) {
            x = xin[(size_t)e * n + i];
            r -= block_row_n<N, float, float, float>(AdT, AoT, nbr, xin, e, i);
        }
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

// res = b - A x (FP32)
template <int N>
__global__ void bj_residual_kernel(int ne, const float* __restrict__ AdT, const float* __restrict__ AoT,
                                   const int32_t* __restrict__ nbr, const double* __restrict__ b,
                                   const float* __restrict__ x, float* __restrict__ res, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * N) return;
    const int e = t / N, i = t - e * N;
    res[t] = (float)b[t] - block_row_n<N, float, float, float>(AdT, AoT, nbr, x, e, i);
}

// bv[v] = sum over (element, corner) at vertex v of sum_i w4[i][corner] res[e][i]
__global__ void restrict_q1_kernel(int nvert, int n, const int* __restrict__ vrp, const int* __restrict__ vinc,
                                   const double* __restrict__ w4, const float* __restrict__ res,
                                   double* __restrict__ bv, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvert) return;
    double s = 0.0;
    for (int k = vrp[v]; k < vrp[v + 1]; ++k) {
        const int e = vinc[k] >> 2, c = vinc[k] & 3;
        const float* re = res + (size_t)e * n;
        for (int i = 0; i < n; ++i) s += w4[i * 4 + c] * (double)re[i];
    }
    bv[v] = s;
}

// x[e][i] += sum_c w4[i][c] xv[vid[e][c]]
__global__ void prolong_q1_kernel(int ne, int n, const int* __restrict__ vid, const double* __restrict__ w4,
                                  const double* __restrict__ xv, float* __restrict__ x, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * n) return;
    const int e = t / n, i = t - e * n;
    const int* ve = vid + e * 4;
    x[t] += (float)(w4[i * 4] * xv[ve[0]] + w4[i * 4 + 1] * xv[ve[1]] + w4[i * 4 + 2] * xv[ve[2]] +
                    w4[i * 4 + 3] * xv[ve[3]]);
}

__device__ __forceinline__ double csr_row(const int* rp, const int* ci, const double* v, const double* x, int i) {
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
    return s;
}

// x = omega dinv b
__global__ void jac_first_kernel(int n, const double* __restrict__ dinv, double omega, const double* __restrict__ b,
                                 double* __restrict__ x, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = omega * dinv[i] * b[i];
}

// r = b - A x
__global__ void csr_residual_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                    const double* __restrict__ v, const double* __restrict__ b,
                                    const double* __restrict__ x, double* __restrict__ r, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - csr_row(rp, ci, v, x, i);
}

// y = M x   (accumulate: y += M x)
__global__ void csr_spmv_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ y,
                                int accumulate, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = csr_row(rp, ci, v, x, i);
    y[i] = accumulate ? y[i] + s : s;
}

// xout = x + omega dinv (b - A x)
__global__ void jac_step_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                const double* __restrict__ v, const double* __restrict__ dinv, double omega,
                                const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ xout,
                                const int* ctl) {
    if (cg_finished(ctl)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xout[i] = x[i] + omega * dinv[i] * (b[i] - csr_row(rp, ci, v, x, i));
}

// x = Cinv b (dense, row-major), one warp per row
__global__ void dense_solve_kernel(int n, const double* __restrict__ cinv, const double* __restrict__ b,
                                   double* __restrict__ x, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= n) return;
    const double* cr = cinv + (size_t)row * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += cr[j] * b[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = s;
}

}  // namespace

template <int N>
int mg_apply_n(const MGPlan& m, const double* r, double* z, const int* ctl, cudaStream_t s);

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
    const int rows0 = m.ne * N;
    const float w0 = (float)m.omega0;
    // level 0 pre-smoothing from zero (FP32)
    float* xa = m.x0;
    float* xb = m.x0b;
    bj_smooth_kernel<float, N><<<nblk0, tpb, shm, s>>>(m.ne, m.AdT, m.AoT, m.PinvT, m.nbr, w0, r, nullptr, xa, ctl);
    ++launches;
    for (int k = 1; k < m.nu0; ++k) {
        bj_smooth_kernel<float, N><<<nblk0, tpb, shm, s>>>(m.ne, m.AdT, m.AoT, m.PinvT, m.nbr, w0, r, xa, xb, ctl);
        std::swap(xa, xb);
        ++launches;
    }
    bj_residual_kernel<N><<<blocks_for(rows0), kTPB, 0, s>>>(m.ne, m.AdT, m.AoT, m.nbr, r, xa, m.res0, ctl);
    restrict_q1_kernel<<<blocks_for(m.nvert), kTPB, 0, s>>>(m.nvert, N, m.vrp, m.vinc, m.w4, m.res0, m.lv[1].b, ctl);
    launches += 2;
    // down the CSR levels (FP64)
    for (int l = 1; l < m.nlev; ++l) {
        const MGLevelDev& L = m.lv[l];
        jac_first_kernel<<<blocks_for(L.n), kTPB, 0, s>>>(L.n, L.dinv, L.omega, L.b, L.x, ctl);
        csr_residual_kernel<<<blocks_for(L.n), kTPB, 0, s>>>(L.n, L.Arp, L.Aci, L.Av, L.b, L.x, L.r, ctl);
        csr_spmv_kernel<<<blocks_for(m.lv[l + 1].n), kTPB, 0, s>>>(m.lv[l + 1].n, L.Rrp, L.Rci, L.Rv, L.r,
                                                                    m.lv[l + 1].b, 0, ctl);
        launches += 3;
    }
    const MGLevelDev& C = m.lv[m.nlev];
    dense_solve_kernel<<<(C.n * 32 + 255) / 256, 256, 0, s>>>(C.n, m.cinv, C.b, C.x, ctl);
    ++launches;
    const double* coarse_out = C.x;
    // up the CSR levels
    for (int l = m.nlev - 1; l >= 1; --l) {
        const MGLevelDev& L = m.lv[l];
        csr_spmv_kernel<<<blocks_for(L.n), kTPB, 0, s>>>(L.n, L.Prp, L.Pci, L.Pv, coarse_out, L.x, 1, ctl);
        jac_step_kernel<<<blocks_for(L.n), kTPB, 0, s>>>(L.n, L.Arp, L.Aci, L.Av, L.dinv, L.omega, L.b, L.x, L.t, ctl);
        coarse_out = L.t;
        launches += 2;
    }
    // back to level 0: prolongate, post-smooth (the last step writes the FP64 z)
    prolong_q1_kernel<<<blocks_for(rows0), kTPB, 0, s>>>(m.ne, N, m.vid, m.w4, coarse_out, xa, ctl);
    ++launches;
    for (int k = 0; k < m.nu0; ++k) {
        if (k == m.nu0 - 1) {
            bj_smooth_kernel<double, N><<<nblk0, tpb, shm, s>>>(m.ne, m.AdT, m.AoT, m.PinvT, m.nbr, w0, r, xa, z,
                                                             ctl);
        } else {
            bj_smooth_kernel<float, N><<<nblk0, tpb, shm, s>>>(m.ne, m.AdT, m.AoT, m.PinvT, m.nbr, w0, r, xa, xb,
                                                            ctl);
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

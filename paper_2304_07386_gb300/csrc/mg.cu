// Multigrid V-cycle preconditioner for the IP-SMM moment operator (FP64).
//
// Level 0: DG-p element blocks, nu0 steps of damped element-block Jacobi
// before and after the coarse correction.  Level 1: continuous bilinear
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

// xout = xin + omega Pinv (b - A xin); xin == nullptr means xin = 0
__global__ void bj_smooth_kernel(int ne, int n, const double* __restrict__ AdT, const double* __restrict__ AoT,
                                 const double* __restrict__ PinvT, const int32_t* __restrict__ nbr, double omega,
                                 const double* __restrict__ b, const double* __restrict__ xin,
                                 double* __restrict__ xout, const int* ctl) {
    if (cg_finished(ctl)) return;
    extern __shared__ double res[];
    const int epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    const bool act = e < ne;
    double r = 0.0, x = 0.0;
    if (act) {
        r = b[(size_t)e * n + i];
        if (xin) {
            x = xin[(size_t)e * n + i];
            r -= block_row(AdT, AoT, nbr, n, xin, e, i);
        }
    }
    res[threadIdx.x] = r;
    __syncthreads();
    if (act) {
        const double* P = PinvT + (size_t)e * n * n + i;
        const double* re = res + (threadIdx.x / n) * n;
        double z = 0.0;
        for (int j = 0; j < n; ++j) z += P[(size_t)j * n] * re[j];
        xout[(size_t)e * n + i] = x + omega * z;
    }
}

// res = b - A x
__global__ void bj_residual_kernel(int ne, int n, const double* __restrict__ AdT, const double* __restrict__ AoT,
                                   const int32_t* __restrict__ nbr, const double* __restrict__ b,
                                   const double* __restrict__ x, double* __restrict__ res, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * n) return;
    const int e = t / n, i = t - e * n;
    res[t] = b[t] - block_row(AdT, AoT, nbr, n, x, e, i);
}

// bv[v] = sum over (element, corner) at vertex v of sum_i w4[i][corner] res[e][i]
__global__ void restrict_q1_kernel(int nvert, int n, const int* __restrict__ vrp, const int* __restrict__ vinc,
                                   const double* __restrict__ w4, const double* __restrict__ res,
                                   double* __restrict__ bv, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvert) return;
    double s = 0.0;
    for (int k = vrp[v]; k < vrp[v + 1]; ++k) {
        const int e = vinc[k] >> 2, c = vinc[k] & 3;
        const double* re = res + (size_t)e * n;
        for (int i = 0; i < n; ++i) s += w4[i * 4 + c] * re[i];
    }
    bv[v] = s;
}

// x[e][i] += sum_c w4[i][c] xv[vid[e][c]]
__global__ void prolong_q1_kernel(int ne, int n, const int* __restrict__ vid, const double* __restrict__ w4,
                                  const double* __restrict__ xv, double* __restrict__ x, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * n) return;
    const int e = t / n, i = t - e * n;
    const int* ve = vid + e * 4;
    x[t] += w4[i * 4] * xv[ve[0]] + w4[i * 4 + 1] * xv[ve[1]] + w4[i * 4 + 2] * xv[ve[2]] + w4[i * 4 + 3] * xv[ve[3]];
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

// x = Cinv b (dense, row-major), one block
__global__ void dense_solve_kernel(int n, const double* __restrict__ cinv, const double* __restrict__ b,
                                   double* __restrict__ x, const int* ctl) {
    if (cg_finished(ctl)) return;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double* row = cinv + (size_t)i * n;
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += row[j] * b[j];
        x[i] = s;
    }
}

}  // namespace

int mg_apply(const MGPlan& m, const double* r, double* z, const int* ctl, cudaStream_t s) {
    int launches = 0;
    const int tpb = cg_threads_per_block(m.n);
    const int nblk0 = (m.ne + tpb / m.n - 1) / (tpb / m.n);
    const size_t shm = tpb * sizeof(double);
    const int rows0 = m.ne * m.n;
    // level 0 pre-smoothing from zero
    double* xa = m.x0;
    double* xb = m.x0b;
    bj_smooth_kernel<<<nblk0, tpb, shm, s>>>(m.ne, m.n, m.AdT, m.AoT, m.PinvT, m.nbr, m.omega0, r, nullptr, xa, ctl);
    ++launches;
    for (int k = 1; k < m.nu0; ++k) {
        bj_smooth_kernel<<<nblk0, tpb, shm, s>>>(m.ne, m.n, m.AdT, m.AoT, m.PinvT, m.nbr, m.omega0, r, xa, xb, ctl);
        std::swap(xa, xb);
        ++launches;
    }
    bj_residual_kernel<<<blocks_for(rows0), kTPB, 0, s>>>(m.ne, m.n, m.AdT, m.AoT, m.nbr, r, xa, m.res0, ctl);
    restrict_q1_kernel<<<blocks_for(m.nvert), kTPB, 0, s>>>(m.nvert, m.n, m.vrp, m.vinc, m.w4, m.res0, m.lv[1].b, ctl);
    launches += 2;
    // down the CSR levels
    for (int l = 1; l < m.nlev; ++l) {
        const MGLevelDev& L = m.lv[l];
        jac_first_kernel<<<blocks_for(L.n), kTPB, 0, s>>>(L.n, L.dinv, L.omega, L.b, L.x, ctl);
        csr_residual_kernel<<<blocks_for(L.n), kTPB, 0, s>>>(L.n, L.Arp, L.Aci, L.Av, L.b, L.x, L.r, ctl);
        csr_spmv_kernel<<<blocks_for(m.lv[l + 1].n), kTPB, 0, s>>>(m.lv[l + 1].n, L.Rrp, L.Rci, L.Rv, L.r,
                                                                    m.lv[l + 1].b, 0, ctl);
        launches += 3;
    }
    const MGLevelDev& C = m.lv[m.nlev];
    dense_solve_kernel<<<1, 512, 0, s>>>(C.n, m.cinv, C.b, C.x, ctl);
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
    // back to level 0: prolongate, post-smooth (the last step writes z)
    prolong_q1_kernel<<<blocks_for(rows0), kTPB, 0, s>>>(m.ne, m.n, m.vid, m.w4, coarse_out, xa, ctl);
    ++launches;
    for (int k = 0; k < m.nu0; ++k) {
        double* out = (k == m.nu0 - 1) ? z : xb;
        bj_smooth_kernel<<<nblk0, tpb, shm, s>>>(m.ne, m.n, m.AdT, m.AoT, m.PinvT, m.nbr, m.omega0, r, xa, out, ctl);
        std::swap(xa, xb);
        ++launches;
    }
    return launches;
}

}  // namespace smm

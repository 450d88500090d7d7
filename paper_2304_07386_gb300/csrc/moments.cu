// Angular moments, SMM closures, IP-SMM right-hand side and the
// block-Jacobi preconditioned CG of the moment system (FP64).
#include <algorithm>

#include "blockops.cuh"
#include "dfloat.cuh"
#include "kernels.cuh"

namespace smm {

namespace {

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}


}  // namespace

// T (the three correction components, component stride cst) of cnt = elements
// x n dofs into shared memory as pairs, component stride sst.  The rows of K
// and of the face gradient operators sum to zero (the nodal basis is a
// partition of unity), so each element's T enters shifted by its value at the
// element's first node: the pair products then carry the variation of T across
// the element instead of its size, which keeps their cancellation (and so the
// pair rounding) small on fine meshes.
__device__ __forceinline__ void stage_T(float2* sT, const double* __restrict__ t0, size_t cst, int cnt, int sst, int n) {
    for (int k = threadIdx.x; k < 3 * cnt; k += blockDim.x) {
        const int c = k / cnt, r = k - c * cnt;
        const double* tc = t0 + c * cst;
        sT[c * sst + r] = df_make(tc[r] - tc[r - r % n]);
    }
}

// Face traces of the correction tensor per (element, face, Gauss point):
// g = (div T . n ds)/sigma_t, and T n ds (2 components).  A block takes epb
// whole elements, one thread per face point; their T is staged in shared
// memory as FP32 pairs and the gradient sums are pair dot products
// (dfloat.cuh), since FP64 FMAs are the scarce unit here.
template <int N>  // dofs per element, or 0: taken from n_rt
__global__ void rhs_trace_kernel(int ne, int n_rt, int p, int nfq, int epb, const double* __restrict__ mom,
                                 const float2* __restrict__ DfxT, const float2* __restrict__ DfyT,
                                 const double* __restrict__ nds, const double* __restrict__ L1,
                                 const double* __restrict__ sigma_t, double* __restrict__ tr) {
    const int n = N > 0 ? N : n_rt;
    extern __shared__ float2 sT[];  // [3][epb][n]: Txx, Txy, Tyy
    const int e0 = blockIdx.x * epb, ecount = min(epb, ne - e0), cnt = ecount * n;
    const size_t st = (size_t)ne * n;
    stage_T(sT, mom + 3 * st + (size_t)e0 * n, st, cnt, epb * n, n);
    __syncthreads();
    const int fq = 4 * nfq, le = threadIdx.x / fq;
    if (le >= ecount) return;
    const int r = threadIdx.x - le * fq, f = r / nfq, q = r - f * nfq, e = e0 + le;
    const size_t t = (size_t)e * fq + r;
    // the face gradient operators as [element][face][node][point]: the threads of one face read
    // consecutive words
    const float2* dx = DfxT + ((size_t)e * 4 + f) * n * nfq + q;
    const float2* dy = DfyT + ((size_t)e * 4 + f) * n * nfq + q;
    const float2 *txx = sT + le * n, *txy = txx + epb * n, *tyy = txy + epb * n;
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const float2 ax = dx[(size_t)j * nfq], ay = dy[(size_t)j * nfq];
        const float2 a = txx[j], b = txy[j], c = tyy[j];
        df_acc(sx, cx, ax.x, ax.y, a.x, a.y);
        df_acc(sx, cx, ay.x, ay.y, b.x, b.y);
        df_acc(sy, cy, ax.x, ax.y, b.x, b.y);
        df_acc(sy, cy, ay.x, ay.y, c.x, c.y);
    }
    const double divx = df_to_double(sx, cx), divy = df_to_double(sy, cy);
    const double* gxx = mom + 3 * st + (size_t)e * n;
    const double* gxy = mom + 4 * st + (size_t)e * n;
    const double* gyy = mom + 5 * st + (size_t)e * n;
    const int p1 = p + 1;
    double vxx = 0, vxy = 0, vyy = 0;
    for (int a = 0; a < p1; ++a) {
        const int nd_ = f == 0 ? a : (f == 1 ? a * p1 + p : (f == 2 ? p * p1 + a : a * p1));
        const double l = L1[q * p1 + a];
        vxx += l * gxx[nd_];
        vxy += l * gxy[nd_];
        vyy += l * gyy[nd_];
    }
    const double nx = nds[2 * t], ny = nds[2 * t + 1];
    tr[3 * t] = (divx * nx + divy * ny) / sigma_t[e];
    tr[3 * t + 1] = vxx * nx + vxy * ny;
    tr[3 * t + 2] = vxy * nx + vyy * ny;
}

// IP-SMM right-hand side (Eq. ipsmm), element-centric, one thread per dof:
// b = b_fixed - (1/sigma_t)(Kxx Txx + (Kxy+Kyx) Txy + Kyy Tyy)
//   + sum_{interior f} sum_q [ l_a(s_q) (g_K - g_K')/2 + (grad phi_i/sigma_t) . (Tn_K + Tn_K')/2 ]
//   - sum_{boundary f} sum_q ds_q l_a(s_q) beta_q
// A block takes epb whole elements.  It first forms, once per face point, the
// weights that every dof of the face shares: (Tn_K + Tn_K')/(2 sigma_t) as
// pairs and the jump (g_K - g_K')/2, or -ds beta on a boundary face, in FP64.
// The K and face-gradient products are then pair dot products (dfloat.cuh)
// against T staged as pairs; the blocks of K are column-major (entry (i, j)
// at [e][j][i]) so that the n threads of an element read contiguous words.
template <int N>  // dofs per element, or 0: taken from n_rt
__global__ void rhs_assemble_kernel(int ne, int n_rt, int p, int nfq, int epb, const double* __restrict__ mom,
                                    const double* __restrict__ beta, const double* __restrict__ bfixed,
                                    const float2* __restrict__ Kxx, const float2* __restrict__ Ks,
                                    const float2* __restrict__ Kyy, const float2* __restrict__ Dfx,
                                    const float2* __restrict__ Dfy, const double* __restrict__ L1,
                                    const double* __restrict__ sigma_t, const int32_t* __restrict__ nbr,
                                    const int32_t* __restrict__ nbr_face, const int32_t* __restrict__ nbr_flip,
                                    const int32_t* __restrict__ bface_id, const double* __restrict__ b_ds,
                                    const double* __restrict__ tr, double* __restrict__ rhs) {
    const int n = N > 0 ? N : n_rt;
    extern __shared__ float2 sh2[];
    const int nf = 4 * nfq;                     // face points of one element
    float2* sT = sh2;                           // [3][epb][n]: Txx, Txy, Tyy
    float2* sC = sh2 + 3 * epb * n;             // [epb][4 nfq][2]: (Tn_K + Tn_K')/(2 sigma_t)
    double* sG = (double*)(sC + 2 * epb * nf);  // [epb][4 nfq]: jump or boundary weight
    const int e0 = blockIdx.x * epb, ecount = min(epb, ne - e0), cnt = ecount * n;
    const size_t st = (size_t)ne * n;
    stage_T(sT, mom + 3 * st + (size_t)e0 * n, st, cnt, epb * n, n);
    for (int k = threadIdx.x; k < ecount * nf; k += blockDim.x) {
        const int le = k / nf, r = k - le * nf, f = r / nfq, q = r - f * nfq, e = e0 + le;
        const int e2 = nbr[e * 4 + f];
        if (e2 >= 0) {
            const int f2 = nbr_face[e * 4 + f], q2 = nbr_flip[e * 4 + f] ? nfq - 1 - q : q;
            const double* a1 = tr + 3 * ((size_t)e * nf + r);
            const double* a2 = tr + 3 * (((size_t)e2 * 4 + f2) * nfq + q2);
            const double hs = 0.5 / sigma_t[e];
            sC[2 * k] = df_make(hs * (a1[1] + a2[1]));
            sC[2 * k + 1] = df_make(hs * (a1[2] + a2[2]));
            sG[k] = 0.5 * (a1[0] - a2[0]);
        } else {
            const size_t bq = (size_t)bface_id[e * 4 + f] * nfq + q;
            sC[2 * k] = make_float2(0.f, 0.f);
            sC[2 * k + 1] = make_float2(0.f, 0.f);
            sG[k] = -(b_ds[bq] * beta[bq]);
        }
    }
    __syncthreads();
    const int le = threadIdx.x / n;
    if (le >= ecount) return;
    const int i = threadIdx.x - le * n, e = e0 + le;
    const size_t t = (size_t)e * n + i;
    const size_t mo = (size_t)e * n * n + i;
    const float2 *txx = sT + le * n, *txy = txx + epb * n, *tyy = txy + epb * n;
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const float2 kx = Kxx[mo + (size_t)j * n], ks = Ks[mo + (size_t)j * n], ky = Kyy[mo + (size_t)j * n];
        const float2 a = txx[j], b = txy[j], c = tyy[j];
        df_acc(s0, c0, kx.x, kx.y, a.x, a.y);
        df_acc(s1, c1, ks.x, ks.y, b.x, b.y);
        df_acc(s2, c2, ky.x, ky.y, c.x, c.y);
    }
    const int p1 = p + 1, ix = i % p1, iy = i / p1;
    double jump = 0.0;
    for (int f = 0; f < 4; ++f) {
        const int lf = le * nf + f * nfq;
        if (nbr[e * 4 + f] >= 0) {
            const float2* dx = Dfx + ((size_t)e * nf + f * nfq) * n + i;
            const float2* dy = Dfy + ((size_t)e * nf + f * nfq) * n + i;
            for (int q = 0; q < nfq; ++q) {
                const float2 ax = dx[(size_t)q * n], ay = dy[(size_t)q * n];
                const float2 wx = sC[2 * (lf + q)], wy = sC[2 * (lf + q) + 1];
                df_acc(s0, c0, ax.x, ax.y, wx.x, wx.y);
                df_acc(s1, c1, ay.x, ay.y, wy.x, wy.y);
            }
        }
        const bool on = (f == 0 && iy == 0) || (f == 1 && ix == p) || (f == 2 && iy == p) || (f == 3 && ix == 0);
        if (on) {
            const int fa = (f == 0 || f == 2) ? ix : iy;
            for (int q = 0; q < nfq; ++q) jump += L1[q * p1 + fa] * sG[lf + q];
        }
    }
    rhs[t] = bfixed[t] + (df_to_double(s0, c0) + df_to_double(s1, c1) + df_to_double(s2, c2)) + jump;
}

template <int N>
void launch_rhs_n(int ne, int n, int p, int nfq, const double* mom, const double* beta, const double* bfixed,
                  const float2* Kxx, const float2* Ks, const float2* Kyy, const float2* Dfx, const float2* Dfy,
                  const float2* DfxT, const float2* DfyT, const double* nds, const double* L1, const double* sigma_t,
                  const int32_t* nbr, const int32_t* nbr_face, const int32_t* nbr_flip, const int32_t* bface_id,
                  const double* b_ds, double* trace, double* rhs, cudaStream_t s) {
    // trace: whole elements of 4 nfq face points per block (nfq <= 11: at least 5 elements)
    const int fq = 4 * nfq, ept = std::max(1, 256 / fq);
    const size_t sh1 = (size_t)3 * ept * n * sizeof(float2);
    rhs_trace_kernel<N><<<(ne + ept - 1) / ept, (ept * fq + 31) / 32 * 32, sh1, s>>>(ne, n, p, nfq, ept, mom, DfxT,
                                                                                   DfyT, nds, L1, sigma_t, trace);
    // assembly: whole elements of n dofs per block; at most 32 elements keeps the face
    // weights of p = 1 within 48 KB of shared memory
    const int epa = std::max(1, std::min(256 / n, 32));
    const size_t sh2 = (size_t)(3 * epa * n + 2 * epa * fq) * sizeof(float2) + (size_t)epa * fq * sizeof(double);
    rhs_assemble_kernel<N><<<(ne + epa - 1) / epa, (epa * n + 31) / 32 * 32, sh2, s>>>(
        ne, n, p, nfq, epa, mom, beta, bfixed, Kxx, Ks, Kyy, Dfx, Dfy, L1, sigma_t, nbr, nbr_face, nbr_flip, bface_id,
        b_ds, trace, rhs);
}

void launch_rhs(int ne, int n, int p, int nfq, const double* mom, const double* beta, const double* bfixed,
                const float2* Kxx, const float2* Ks, const float2* Kyy, const float2* Dfx, const float2* Dfy,
                const float2* DfxT, const float2* DfyT, const double* nds, const double* L1, const double* sigma_t,
                const int32_t* nbr, const int32_t* nbr_face, const int32_t* nbr_flip, const int32_t* bface_id,
                const double* b_ds, double* trace, double* rhs, cudaStream_t s) {
    // the element sizes of p = 1..4 get fully unrolled dot products
    auto* f = &launch_rhs_n<0>;
    switch (n) {
        case 4: f = &launch_rhs_n<4>; break;
        case 9: f = &launch_rhs_n<9>; break;
        case 16: f = &launch_rhs_n<16>; break;
        case 25: f = &launch_rhs_n<25>; break;
        default: break;
    }
    f(ne, n, p, nfq, mom, beta, bfixed, Kxx, Ks, Kyy, Dfx, Dfy, DfxT, DfyT, nds, L1, sigma_t, nbr, nbr_face, nbr_flip,
      bface_id, b_ds, trace, rhs, s);
}

// ---------------------------------------------------------------------------
// Block-Jacobi PCG on the IP-SMM operator.  Operator blocks are stored
// transposed ([e][j][i]) so that the threads of one element read contiguous
// entries.  Blocks of threads cover whole elements (EPB elements x n rows).
// Scalars are reduced deterministically: per-block partials, then every
// block sums all partials in the same order.
// ---------------------------------------------------------------------------
int cg_threads_per_block(int n) { return std::max(1, 256 / n) * n; }

namespace {

__device__ double sum_partials(const double* part, int nblk, double* sh) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) v += part[i];
    double s = block_sum(v, sh);
    if (threadIdx.x == 0) sh[32] = s;
    __syncthreads();
    s = sh[32];
    __syncthreads();
    return s;
}




// r = b - A x ; z = P r ; p = z ; partials: rz, rr, bb
template <int N>
__global__ void __launch_bounds__(256) cg_init_kernel(CGArgs a) {
    __shared__ double sh[40];
    __shared__ FaceScratch<N, double> sc;
    __shared__ double rs[256];
    constexpr int n = N;
    const int epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    const bool act = e < a.ne;
    const double ax = faceop_row<N, double, double, double>(a.A, a.x, e, i, act, sc);
    double r = 0.0, bv = 0.0;
    if (act) {
        bv = a.b[(size_t)e * n + i];
        r = bv - ax;
        a.r[(size_t)e * n + i] = r;
    }
    rs[threadIdx.x] = r;
    __syncthreads();
    double z = 0.0;
    if (act) {
        const double* P = a.PinvT + (size_t)e * n * n + i;
        const double* re = rs + (threadIdx.x / n) * n;
        for (int j = 0; j < n; ++j) z += P[(size_t)j * n] * re[j];
        a.z[(size_t)e * n + i] = z;
        a.p[(size_t)e * n + i] = z;
    }
    double s0 = block_sum(r * z, sh);
    double s1 = block_sum(r * r, sh);
    double s2 = block_sum(bv * bv, sh);
    if (threadIdx.x == 0) {
        a.part[blockIdx.x] = s0;
        a.part[a.nblk + blockIdx.x] = s1;
        a.part[2 * a.nblk + blockIdx.x] = s2;
    }
}

// dense-operator variants of the two kernels above (runtime n)
__global__ void cg_init_dense_kernel(CGArgs a) {
    __shared__ double sh[40];
    extern __shared__ double rsd[];
    const int n = a.n, epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    const bool act = e < a.ne;
    double r = 0.0, bv = 0.0;
    if (act) {
        bv = a.b[(size_t)e * n + i];
        r = bv - dense_block_row(a.AdT_dense, a.AoT_dense, a.nbr_dense, n, a.x, e, i);
        a.r[(size_t)e * n + i] = r;
    }
    rsd[threadIdx.x] = r;
    __syncthreads();
    double z = 0.0;
    if (act) {
        const double* P = a.PinvT + (size_t)e * n * n + i;
        const double* re = rsd + (threadIdx.x / n) * n;
        for (int j = 0; j < n; ++j) z += P[(size_t)j * n] * re[j];
        a.z[(size_t)e * n + i] = z;
        a.p[(size_t)e * n + i] = z;
    }
    double s0 = block_sum(r * z, sh);
    double s1 = block_sum(r * r, sh);
    double s2 = block_sum(bv * bv, sh);
    if (threadIdx.x == 0) {
        a.part[blockIdx.x] = s0;
        a.part[a.nblk + blockIdx.x] = s1;
        a.part[2 * a.nblk + blockIdx.x] = s2;
    }
}

__global__ void cg_spmv_dense_kernel(CGArgs a) {
    if (*(volatile int*)a.ctl) return;
    __shared__ double sh[40];
    const int n = a.n, epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    double pq = 0.0;
    if (e < a.ne) {
        const double qv = dense_block_row(a.AdT_dense, a.AoT_dense, a.nbr_dense, n, a.p, e, i);
        a.q[(size_t)e * n + i] = qv;
        pq = qv * a.p[(size_t)e * n + i];
    }
    double s = block_sum(pq, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s;
}

__global__ void cg_init_scalars_kernel(CGArgs a, double tol2, int max_iters) {
    __shared__ double sh[40];
    double rz = sum_partials(a.part, a.nblk, sh);
    double rr = sum_partials(a.part + a.nblk, a.nblk, sh);
    double bb = sum_partials(a.part + 2 * a.nblk, a.nblk, sh);
    if (threadIdx.x == 0) {
        a.scal[0] = rz;
        a.scal[2] = rr;
        a.scal[3] = bb;
        a.scal[4] = tol2 * bb;
        a.ctl[1] = 0;
        a.ctl[2] = max_iters;
        a.ctl[3] = (isfinite(rz) && isfinite(rr) && isfinite(bb)) ? 0 : 1;
        a.ctl[0] = (rr <= tol2 * bb || a.ctl[3]) ? 1 : 0;
    }
}

// q = A p ; partial p.q
template <int N>
__global__ void __launch_bounds__(256) cg_spmv_kernel(CGArgs a) {
    if (*(volatile int*)a.ctl) return;
    __shared__ double sh[40];
    __shared__ FaceScratch<N, double> sc;
    constexpr int n = N;
    const int epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    const double qv = faceop_row<N, double, double, double>(a.A, a.p, e, i, e < a.ne, sc);
    double pq = 0.0;
    if (e < a.ne) {
        a.q[(size_t)e * n + i] = qv;
        pq = qv * a.p[(size_t)e * n + i];
    }
    double s = block_sum(pq, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s;
}

// alpha = rz / pq ; x += alpha p ; r -= alpha q ; z = P r ; partials r.z, r.r
__global__ void cg_update_kernel(CGArgs a) {
    if (*(volatile int*)a.ctl) return;
    __shared__ double sh[40];
    extern __shared__ double rs[];
    const double pq = sum_partials(a.part, a.nblk, sh);
    const double alpha = a.scal[0] / pq;
    const int n = a.n, epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    const bool act = e < a.ne;
    double r = 0.0;
    if (act) {
        const size_t o = (size_t)e * n + i;
        a.x[o] += alpha * a.p[o];
        r = a.r[o] - alpha * a.q[o];
        a.r[o] = r;
    }
    rs[threadIdx.x] = r;
    __syncthreads();
    double z = 0.0;
    if (act) {
        const double* P = a.PinvT + (size_t)e * n * n + i;
        const double* re = rs + (threadIdx.x / n) * n;
        for (int j = 0; j < n; ++j) z += P[(size_t)j * n] * re[j];
        a.z[(size_t)e * n + i] = z;
    }
    double s0 = block_sum(r * z, sh);
    double s1 = block_sum(r * r, sh);
    if (threadIdx.x == 0) {
        a.part[a.nblk + blockIdx.x] = s0;
        a.part[2 * a.nblk + blockIdx.x] = s1;
    }
}

// beta = rz_new / rz ; p = z + beta p ; convergence and iteration count
__global__ void cg_direction_kernel(CGArgs a) {
    if (*(volatile int*)a.ctl) return;
    __shared__ double sh[40];
    const double rz_new = sum_partials(a.part + a.nblk, a.nblk, sh);
    const double rr = sum_partials(a.part + 2 * a.nblk, a.nblk, sh);
    const double beta = rz_new / a.scal[0];
    const int n = a.n, epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    if (e < a.ne) {
        const size_t o = (size_t)e * n + i;
        a.p[o] = a.z[o] + beta * a.p[o];
    }
    // every block has read scal[0] above; make the update visible only after
    // all blocks are done with it: block 0 writes into a second slot, the
    // finisher (last block) publishes.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned prev = atomicAdd((unsigned*)(a.ctl + 4), 1u);
        if (prev == (unsigned)gridDim.x - 1) {
            a.ctl[4] = 0;
            a.scal[0] = rz_new;
            a.scal[2] = rr;
            const int it = a.ctl[1] + 1;
            a.ctl[1] = it;
            const bool bad = !(isfinite(rz_new) && isfinite(rr));
            if (bad) a.ctl[3] = 1;
            if (rr <= a.scal[4] || it >= a.ctl[2] || bad) a.ctl[0] = 1;
            __threadfence();
        }
    }
}

// ---- CG with an external preconditioner (multigrid) ----
// r = b - A x ; partials rr -> part[nblk], bb -> part[2 nblk]
template <int N>
__global__ void __launch_bounds__(256) cgx_init_r_kernel(CGArgs a) {
    __shared__ double sh[40];
    __shared__ FaceScratch<N, double> sc;
    constexpr int n = N;
    const int epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    const double ax = faceop_row<N, double, double, double>(a.A, a.x, e, i, e < a.ne, sc);
    double r = 0.0, bv = 0.0;
    if (e < a.ne) {
        bv = a.b[(size_t)e * n + i];
        r = bv - ax;
        a.r[(size_t)e * n + i] = r;
    }
    double s1 = block_sum(r * r, sh);
    double s2 = block_sum(bv * bv, sh);
    if (threadIdx.x == 0) {
        a.part[a.nblk + blockIdx.x] = s1;
        a.part[2 * a.nblk + blockIdx.x] = s2;
    }
}

// p = z ; partial rz -> part[0]
__global__ void cgx_init_p_kernel(CGArgs a) {
    __shared__ double sh[40];
    const int n = a.n, epb = blockDim.x / n;
    const int e = blockIdx.x * epb + threadIdx.x / n, i = threadIdx.x % n;
    double rz = 0.0;
    if (e < a.ne) {
        const size_t o = (size_t)e * n + i;
        const double z = a.z[o];
        a.p[o] = z;
        a.p2[o] = df_make(z);
        rz = z * a.r[o];
    }
    double s = block_sum(rz, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s;
}

// q = A p (FP32-pair arithmetic, FP64 result) ; partial p.q -> part[block];
// the last block reduces the gridDim.x partials: p.q -> scal[1], alpha =
// rz / p.q -> scal[5].  Thread (slot le, row i) handles row i of the R
// elements e0 + k EPB, k < R (e0 = blockIdx.x EPB R + le), as the level-0
// multigrid kernels do.
template <int N, int R>
__global__ void __launch_bounds__(256) cgx_spmv_kernel(CGArgs a) {
    if (*(volatile int*)a.ctl) return;
    constexpr int EPB = FaceDims<N>::EPB, G = FaceDims<N>::G;
    __shared__ double sh[40];
    __shared__ FaceScratchDF<N, EPB * R> sc;
    const int le = threadIdx.x / N, i = threadIdx.x % N;
    const int e0 = blockIdx.x * EPB * R + le;
    float ys[R], yc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        ys[k] = 0.0f;
        yc[k] = 0.0f;
        if (e < a.ne) {
            diag_row_df<N>(a.A2.AdT + (size_t)e * N * N + i, a.p2 + (size_t)e * N, ys[k], yc[k]);
            face_gather_df<N>(a.A2, a.p2, e, i, sc, le + k * EPB);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        if (e < a.ne) face_couple_df<N>(a.A2.CT + (size_t)e * 4 * G * G, a.A2.nbr, e, i, sc, le + k * EPB);
    }
    __syncthreads();
    double pq = 0.0;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int e = e0 + k * EPB;
        if (e < a.ne) {
            const double qv = face_lift_df<N>(a.A2, i, ys[k], yc[k], sc, le + k * EPB);
            a.q[(size_t)e * N + i] = qv;
            pq += qv * a.p[(size_t)e * N + i];
        }
    }
    double s = block_sum(pq, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s;
    if (last_block((unsigned*)(a.ctl + 7))) {
        const double pq_all = sum_partials_cg(a.part, gridDim.x, sh);
        if (threadIdx.x == 0) {
            a.scal[1] = pq_all;
            a.scal[5] = a.scal[0] / pq_all;
            a.ctl[7] = 0;
        }
    }
}

// x += alpha p ; r_old = r ; r -= alpha q ; partial rr -> part[2 nblk]
__global__ void cgx_update_kernel(CGArgs a) {
    if (*(volatile int*)a.ctl) return;
    __shared__ double sh[40];
    // every block reduces the operator product's partials itself (same order
    // everywhere, so every block gets the same alpha)
    const double pq = sum_partials(a.part, a.nblk, sh);
    const double alpha = a.scal[0] / pq;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.scal[1] = pq;
        a.scal[5] = alpha;
    }
    double rr = 0.0;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.nrow; o += gridDim.x * blockDim.x) {
        a.x[o] += alpha * a.p[o];
        const double ro = a.r[o];
        a.rold[o] = ro;
        const double r = ro - alpha * a.q[o];
        a.r[o] = r;
        rr += r * r;
    }
    double s = block_sum(rr, sh);
    if (threadIdx.x == 0) a.pvec[2 * a.nvblk + blockIdx.x] = s;
}

// partials r.z and (r - r_old).z (flexible CG); the last block reduces them
// with the update's r.r partials: beta = (r - r_old).z / rz_old -> scal[6],
// rz, rr, iteration count and convergence
__global__ void cgx_rz_kernel(CGArgs a) {
    if (*(volatile int*)a.ctl) return;
    __shared__ double sh[40];
    double rz = 0.0, dz = 0.0;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.nrow; o += gridDim.x * blockDim.x) {
        const double z = a.z[o], r = a.r[o];
        rz += r * z;
        dz += (r - a.rold[o]) * z;
    }
    double s = block_sum(rz, sh);
    double t = block_sum(dz, sh);
    if (threadIdx.x == 0) {
        a.pvec[a.nvblk + blockIdx.x] = s;
        a.pvec[blockIdx.x] = t;
    }
    if (last_block((unsigned*)(a.ctl + 6))) {
        double dz_all, rz_new, rr;
        sum3_partials_cg(a.pvec, a.nvblk, sh, dz_all, rz_new, rr);
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

// p = z + beta p (flexible beta from scal[6])
__global__ void cgx_direction_kernel(CGArgs a) {
    if (*(volatile int*)a.ctl) return;
    const double beta = a.scal[6];
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.nrow; o += gridDim.x * blockDim.x) {
        const double pn = a.z[o] + beta * a.p[o];
        a.p[o] = pn;
        a.p2[o] = df_make(pn);
    }
}

// max |a - b| and max |a| over rows, plus a non-finite flag
__global__ void diff_kernel(int nrow, const double* __restrict__ x, const double* __restrict__ y, double* part, int* flag) {
    __shared__ double s1[32], s2[32];
    double m1 = 0.0, m2 = 0.0;
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrow; i += gridDim.x * blockDim.x) {
        const double v = x[i];
        bad |= !isfinite(v);
        m1 = fmax(m1, fabs(v - y[i]));
        m2 = fmax(m2, fabs(v));
    }
    if (bad) atomicExch(flag, 1);
    m1 = warp_max(m1);
    m2 = warp_max(m2);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { s1[w] = m1; s2[w] = m2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { m1 = fmax(m1, s1[k]); m2 = fmax(m2, s2[k]); }
        part[2 * blockIdx.x] = m1;
        part[2 * blockIdx.x + 1] = m2;
    }
}

__global__ void diff_final_kernel(int nblk, const double* part, double* out) {
    if (threadIdx.x == 0) {
        double m1 = 0.0, m2 = 0.0;
        for (int k = 0; k < nblk; ++k) { m1 = fmax(m1, part[2 * k]); m2 = fmax(m2, part[2 * k + 1]); }
        out[0] = m1;
        out[1] = m2;
    }
}

}  // namespace

#define SMM_DISPATCH_N(n, KERNEL, ...)                          \
    switch (n) {                                                \
        case 4: KERNEL<4><<<__VA_ARGS__>>>(a); break;           \
        case 9: KERNEL<9><<<__VA_ARGS__>>>(a); break;           \
        case 16: KERNEL<16><<<__VA_ARGS__>>>(a); break;         \
        default: KERNEL<25><<<__VA_ARGS__>>>(a); break;         \
    }

// Flexible-CG pieces shared with the continuous moment solve (grid-stride
// over a.nrow unknowns; the operator-product partials are a.part[0..a.nblk))
void launch_cgx_update(const CGArgs& a, cudaStream_t s) { cgx_update_kernel<<<a.nvblk, 256, 0, s>>>(a); }
void launch_cgx_rz(const CGArgs& a, cudaStream_t s) { cgx_rz_kernel<<<a.nvblk, 256, 0, s>>>(a); }
void launch_cgx_direction(const CGArgs& a, cudaStream_t s) { cgx_direction_kernel<<<(a.nrow + 255) / 256, 256, 0, s>>>(a); }
void launch_cg_init_scalars(const CGArgs& a, double tol, int max_iters, cudaStream_t s) {
    cg_init_scalars_kernel<<<1, 256, 0, s>>>(a, tol * tol, max_iters);
}

void cg_start(const CGArgs& a, double tol, int max_iters, cudaStream_t s) {
    const int tpb = cg_threads_per_block(a.n);
    if (a.AoT_dense) {
        cg_init_dense_kernel<<<a.nblk, tpb, tpb * sizeof(double), s>>>(a);
    } else {
        SMM_DISPATCH_N(a.n, cg_init_kernel, a.nblk, tpb, 0, s)
    }
    cg_init_scalars_kernel<<<1, 256, 0, s>>>(a, tol * tol, max_iters);
}

int cgx_start(const CGArgs& a, double tol, int max_iters, const MGPlan& mg, cudaStream_t s) {
    const int tpb = cg_threads_per_block(a.n);
    SMM_DISPATCH_N(a.n, cgx_init_r_kernel, a.nblk, tpb, 0, s)
    const int l = mg_apply(mg, a.r, a.z, a.ctl, s);
    cgx_init_p_kernel<<<a.nblk, tpb, 0, s>>>(a);
    cg_init_scalars_kernel<<<1, 256, 0, s>>>(a, tol * tol, max_iters);
    return 3 + l;
}

int cgx_iterations(const CGArgs& a, int count, const MGPlan& mg, cudaStream_t s) {
    const int tpb = cg_threads_per_block(a.n);
    int launches = 0;
    for (int k = 0; k < count; ++k) {
        // q = A p and alpha; V-cycle with the update (x, r) and the dots (beta,
        // convergence) folded into its first and last level-0 steps; p = z + beta p
        constexpr int R = 2;   // rows per thread
        const int epb = tpb / a.n, nblkR = (a.ne + epb * R - 1) / (epb * R);
        switch (a.n) {
            case 4: cgx_spmv_kernel<4, R><<<nblkR, tpb, 0, s>>>(a); break;
            case 9: cgx_spmv_kernel<9, R><<<nblkR, tpb, 0, s>>>(a); break;
            case 16: cgx_spmv_kernel<16, R><<<nblkR, tpb, 0, s>>>(a); break;
            default: cgx_spmv_kernel<25, R><<<nblkR, tpb, 0, s>>>(a); break;
        }
        launches += 1 + mg_cg_iteration(mg, a, s);
        // one thread per unknown: every load of the update is in flight at once
        cgx_direction_kernel<<<(a.nrow + 255) / 256, 256, 0, s>>>(a);
        launches += 1;
    }
    return launches;
}

namespace {

// End of one trip of the device-side CG loop (a graph while node): continue
// while the CG has not finished; a hard bound of max_iters + 2 trips (counted
// in ctl[5]) ends the loop even if no kernel has set the finished flag.
__global__ void cg_loop_kernel(cudaGraphConditionalHandle handle, int* ctl) {
    const int trips = ctl[5] + 1;
    ctl[5] = trips;
    const bool stop = *(volatile int*)ctl != 0 || trips >= ctl[2] + 2;
    cudaGraphSetConditional(handle, stop ? 0u : 1u);
}

}  // namespace

void launch_cg_loop_control(cudaGraphConditionalHandle handle, int* ctl, cudaStream_t s) {
    cg_loop_kernel<<<1, 1, 0, s>>>(handle, ctl);
}

void cg_iterations(const CGArgs& a, int count, cudaStream_t s) {
    const int tpb = cg_threads_per_block(a.n);
    for (int k = 0; k < count; ++k) {
        if (a.AoT_dense) {
            cg_spmv_dense_kernel<<<a.nblk, tpb, 0, s>>>(a);
        } else {
            SMM_DISPATCH_N(a.n, cg_spmv_kernel, a.nblk, tpb, 0, s)
        }
        cg_update_kernel<<<a.nblk, tpb, tpb * sizeof(double), s>>>(a);
        cg_direction_kernel<<<a.nblk, tpb, 0, s>>>(a);
    }
}

namespace {

constexpr int kGramBlocks = 256;

__global__ void gram_kernel(int nrow, VecSet vs, double* part) {
    __shared__ double sh[40];
    double acc[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrow; i += gridDim.x * blockDim.x) {
        double x[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) x[a] = a < vs.nv ? vs.v[a][i] : 0.0;
        int k = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) acc[k++] += x[a] * x[b];
    }
    for (int k = 0; k < 21; ++k) {
        const double s = block_sum(acc[k], sh);
        if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void gram_final_kernel(int nblk, const double* part, double* out) {
    const int k = threadIdx.x;
    if (k >= 21) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[k * nblk + b];
    out[k] = s;
}

__global__ void axpby_kernel(int nrow, double alpha, const double* x, double beta, const double* y, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nrow) out[i] = alpha * x[i] + beta * y[i];
}

__global__ void anderson_mix_kernel(int nrow, MixArgs a, double* x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrow) return;
    double v = a.G[0][i];
    for (int j = 0; j < a.m; ++j) v -= a.gamma[j] * (a.G[j][i] - a.G[j + 1][i]);
    x[i] = v;
}

}  // namespace

void launch_gram(int nrow, const VecSet& vs, double* part, double* out, cudaStream_t s) {
    gram_kernel<<<kGramBlocks, 256, 0, s>>>(nrow, vs, part);
    gram_final_kernel<<<1, 32, 0, s>>>(kGramBlocks, part, out);
}

void launch_axpby(int nrow, double alpha, const double* x, double beta, const double* y, double* out, cudaStream_t s) {
    axpby_kernel<<<(nrow + 255) / 256, 256, 0, s>>>(nrow, alpha, x, beta, y, out);
}

void launch_anderson_mix(int nrow, const MixArgs& a, double* x, cudaStream_t s) {
    anderson_mix_kernel<<<(nrow + 255) / 256, 256, 0, s>>>(nrow, a, x);
}

void launch_diff(int nrow, const double* a, const double* b, double* part, double* out, int* flag, cudaStream_t s) {
    const int nblk = 256;
    diff_kernel<<<nblk, 256, 0, s>>>(nrow, a, b, part, flag);
    diff_final_kernel<<<1, 32, 0, s>>>(nblk, part, out);
}

}  // namespace smm

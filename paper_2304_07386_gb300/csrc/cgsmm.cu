// Continuous finite element (CG) SMM moment solve (paper Sec. 5.1).
//
// The CG moment system is Eq. ipsmm with test and trial functions in V_p,
// the continuous degree-p space.  V_p lives on the DG elements' own
// Gauss-Lobatto nodes: a global node is a class of element nodes identified
// across faces, and P: V_p -> Y_p copies a global value to its element nodes.
// Then
//   A_CG = sum_e P_e^T K_e P_e,  K_e = D (Kxx + Kyy) + sigma_a M + Marshak terms,
//   b_CG = P^T b_IP
// (the [u]-weighted face terms of b_IP cancel between the two sides of every
// face once summed over a global node), so the right-hand side reuses the IP
// kernels.  The operator is applied as gather - element block product -
// gather back (element kernel, then a node kernel summing each global node's
// element contributions in a fixed order, so results are deterministic).
//
// Preconditioner: a V-cycle whose level 0 is damped point Jacobi on the
// continuous nodes; its residual is restricted to the element corners
// (weights 1/multiplicity, so each global node counts once) and handed to the
// same vertex-level / aggregation / coarsest cycle as the DG solve, whose
// vertex level is the Galerkin product of K_e with the bilinear weights.
#include <algorithm>

#include "blockops.cuh"
#include "kernels.cuh"

namespace smm {

namespace {

constexpr int kTPB = 256;

__device__ double blk_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) s += sh[i];
    return s;  // valid in thread 0
}

// dst[g] = sum of src over the element nodes of global node g
__global__ void cgc_gather_kernel(int nglob, const int* __restrict__ grp, const int* __restrict__ ginc,
                                  const double* __restrict__ src, double* __restrict__ dst) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nglob) return;
    double s = 0.0;
    for (int k = grp[g]; k < grp[g + 1]; ++k) s += src[ginc[k]];
    dst[g] = s;
}

__global__ void cgc_expand_kernel(int nk, const int* __restrict__ gid, const double* __restrict__ x,
                                  double* __restrict__ dg) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nk) dg[k] = x[gid[k]];
}

__global__ void cgc_pick_kernel(int nglob, const int* __restrict__ gown, const double* __restrict__ dg,
                                double* __restrict__ x) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < nglob) x[g] = dg[gown[g]];
}

// ye[e][i] = sum_j K_e[i][j] v[gid[e][j]]  (blocks column-major: the N threads of
// an element read contiguous words)
template <int N>
__global__ void __launch_bounds__(256) cgc_elem_kernel(int ne, const double* __restrict__ KT,
                                                       const int* __restrict__ gid, const double* __restrict__ v,
                                                       double* __restrict__ ye, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int epb = blockDim.x / N;
    const int e = blockIdx.x * epb + threadIdx.x / N, i = threadIdx.x % N;
    if (e >= ne) return;
    const double* K = KT + (size_t)e * N * N + i;
    const int* g = gid + (size_t)e * N;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) s += K[j * N] * v[g[j]];
    ye[(size_t)e * N + i] = s;
}

enum : int { NODE_SPMV = 0, NODE_INIT_RESIDUAL = 1, NODE_SMOOTH = 2, NODE_RESIDUAL = 3 };

struct NodeArgs {
    int nglob;
    const int* grp;
    const int* ginc;
    const double* ye;
    const double* v;      // SPMV: p (for p.q)
    const double* rhs;    // INIT_RESIDUAL: b; SMOOTH / RESIDUAL: the V-cycle's input r
    const double* xin;    // SMOOTH
    const double* dinv;
    double omega;
    double* out;          // SPMV: q; INIT_RESIDUAL: r; SMOOTH: x out; RESIDUAL: res
    double* part;         // partial sums [3][nblk] (SPMV, INIT_RESIDUAL)
    int nblk;
    const int* ctl;
};

// (A v)[g] = sum of ye over g's element nodes, then per mode:
// SPMV q = A p, partial p.q; INIT_RESIDUAL r = b - A x, partials r.r, b.b;
// SMOOTH x_out = x + omega dinv (r - A x); RESIDUAL res = r - A x
template <int MODE>
__global__ void __launch_bounds__(kTPB) cgc_node_kernel(NodeArgs a) {
    if (cg_finished(a.ctl)) return;
    __shared__ double sh[40];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    double p0 = 0.0, p1 = 0.0;
    if (g < a.nglob) {
        double av = 0.0;
        for (int k = a.grp[g]; k < a.grp[g + 1]; ++k) av += a.ye[a.ginc[k]];
        if (MODE == NODE_SPMV) {
            a.out[g] = av;
            p0 = av * a.v[g];
        } else if (MODE == NODE_INIT_RESIDUAL) {
            const double bg = a.rhs[g], r = bg - av;
            a.out[g] = r;
            p0 = r * r;
            p1 = bg * bg;
        } else if (MODE == NODE_SMOOTH) {
            a.out[g] = a.xin[g] + a.omega * a.dinv[g] * (a.rhs[g] - av);
        } else {
            a.out[g] = a.rhs[g] - av;
        }
    }
    if (MODE == NODE_SPMV) {
        const double s = blk_sum(p0, sh);
        if (threadIdx.x == 0) a.part[blockIdx.x] = s;
    } else if (MODE == NODE_INIT_RESIDUAL) {
        const double s0 = blk_sum(p0, sh);
        const double s1 = blk_sum(p1, sh);
        if (threadIdx.x == 0) {
            a.part[a.nblk + blockIdx.x] = s0;
            a.part[2 * a.nblk + blockIdx.x] = s1;
        }
    }
}

// x = omega dinv r (first smoothing step from zero)
__global__ void cgc_first_smooth_kernel(int nglob, double omega, const double* __restrict__ dinv,
                                        const double* __restrict__ r, double* __restrict__ x, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < nglob) x[g] = omega * dinv[g] * r[g];
}

// cres[e][c] = sum_i w4[i][c] res[gid[e][i]] / mult(gid[e][i])
__global__ void cgc_corner_kernel(int ne, int n, const int* __restrict__ gid, const float* __restrict__ w4,
                                  const float* __restrict__ minv, const double* __restrict__ res,
                                  float* __restrict__ cres, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * 4) return;
    const int e = t >> 2, c = t & 3;
    const int* g = gid + (size_t)e * n;
    float s = 0.0f;
    for (int i = 0; i < n; ++i) s = fmaf(w4[i * 4 + c], (float)res[g[i]] * minv[g[i]], s);
    cres[t] = s;
}

// x[g] += sum_c w4[i][c] xv[vid[e][c]], (e, i) the first element node of g
__global__ void cgc_prolong_kernel(int nglob, int n, const int* __restrict__ gown, const int* __restrict__ vid,
                                   const float* __restrict__ w4, const float* __restrict__ xv,
                                   double* __restrict__ x, const int* ctl) {
    if (cg_finished(ctl)) return;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nglob) return;
    const int k = gown[g], e = k / n, i = k - e * n;
    const int* ve = vid + e * 4;
    const float* w = w4 + i * 4;
    x[g] += (double)(w[0] * xv[ve[0]] + w[1] * xv[ve[1]] + w[2] * xv[ve[2]] + w[3] * xv[ve[3]]);
}

// p = z, p2 = pairs, partial r.z -> part[0..nblk)
__global__ void cgc_init_p_kernel(CGArgs a) {
    __shared__ double sh[40];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    double rz = 0.0;
    if (g < a.nrow) {
        const double z = a.z[g];
        a.p[g] = z;
        const float hi = __double2float_rn(z);
        a.p2[g] = make_float2(hi, __double2float_rn(z - (double)hi));
        rz = z * a.r[g];
    }
    const double s = blk_sum(rz, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s;
}

inline int blocks(int n) { return std::max(1, (n + kTPB - 1) / kTPB); }

template <int N>
void elem_apply(const CGCPlan& c, const double* v, const int* ctl, cudaStream_t s) {
    const int tpb = cg_threads_per_block(N);
    const int nb = (c.ne + tpb / N - 1) / (tpb / N);
    cgc_elem_kernel<N><<<nb, tpb, 0, s>>>(c.ne, c.KT, c.gid, v, c.ye, ctl);
}

void elem_apply_n(const CGCPlan& c, const double* v, const int* ctl, cudaStream_t s) {
    switch (c.n) {
        case 4: elem_apply<4>(c, v, ctl, s); break;
        case 9: elem_apply<9>(c, v, ctl, s); break;
        case 16: elem_apply<16>(c, v, ctl, s); break;
        default: elem_apply<25>(c, v, ctl, s); break;
    }
}

NodeArgs node_args(const CGCPlan& c, const int* ctl) {
    NodeArgs na{};
    na.nglob = c.nglob;
    na.grp = c.grp;
    na.ginc = c.ginc;
    na.ye = c.ye;
    na.dinv = c.dinv;
    na.omega = c.omega;
    na.nblk = c.nblk_node;
    na.ctl = ctl;
    return na;
}

// z = V-cycle(r) on the continuous system; returns the number of launches
int cgc_mg(const CGCPlan& c, const MGPlan& m, const double* r, double* z, const int* ctl, cudaStream_t s) {
    int launches = 0;
    const int nbg = blocks(c.nglob);
    double* xa = c.xa;
    double* xb = c.xb;
    cgc_first_smooth_kernel<<<nbg, kTPB, 0, s>>>(c.nglob, c.omega, c.dinv, r, xa, ctl);
    ++launches;
    NodeArgs na = node_args(c, ctl);
    na.rhs = r;
    for (int k = 1; k < c.nu; ++k) {
        elem_apply_n(c, xa, ctl, s);
        na.xin = xa;
        na.out = xb;
        cgc_node_kernel<NODE_SMOOTH><<<nbg, kTPB, 0, s>>>(na);
        std::swap(xa, xb);
        launches += 2;
    }
    elem_apply_n(c, xa, ctl, s);
    na.out = c.res;
    cgc_node_kernel<NODE_RESIDUAL><<<nbg, kTPB, 0, s>>>(na);
    cgc_corner_kernel<<<blocks(c.ne * 4), kTPB, 0, s>>>(c.ne, c.n, c.gid, m.w4, c.minv, c.res, c.cres, ctl);
    int lc = 0;
    const float* xv = launch_coarse_cycle(m, c.cres, ctl, s, &lc);
    cgc_prolong_kernel<<<nbg, kTPB, 0, s>>>(c.nglob, c.n, c.gown, m.vid, m.w4, xv, xa, ctl);
    launches += 4 + lc;
    for (int k = 0; k < c.nu; ++k) {
        elem_apply_n(c, xa, ctl, s);
        na.xin = xa;
        na.out = (k == c.nu - 1) ? z : xb;
        cgc_node_kernel<NODE_SMOOTH><<<nbg, kTPB, 0, s>>>(na);
        std::swap(xa, xb);
        launches += 2;
    }
    return launches;
}

}  // namespace

void cgc_gather(const CGCPlan& c, const double* b_dg, double* b, cudaStream_t s) {
    cgc_gather_kernel<<<blocks(c.nglob), kTPB, 0, s>>>(c.nglob, c.grp, c.ginc, b_dg, b);
}

void cgc_expand(const CGCPlan& c, const double* x, double* dg, cudaStream_t s) {
    cgc_expand_kernel<<<blocks(c.ne * c.n), kTPB, 0, s>>>(c.ne * c.n, c.gid, x, dg);
}

void cgc_pick(const CGCPlan& c, const double* dg, double* x, cudaStream_t s) {
    cgc_pick_kernel<<<blocks(c.nglob), kTPB, 0, s>>>(c.nglob, c.gown, dg, x);
}

int cgc_start(const CGArgs& a, const CGCPlan& c, const MGPlan& mg, double tol, int max_iters, cudaStream_t s) {
    elem_apply_n(c, a.x, nullptr, s);
    NodeArgs na = node_args(c, nullptr);
    na.rhs = a.b;
    na.out = a.r;
    na.part = a.part;
    cgc_node_kernel<NODE_INIT_RESIDUAL><<<c.nblk_node, kTPB, 0, s>>>(na);
    const int l = cgc_mg(c, mg, a.r, a.z, nullptr, s);
    cgc_init_p_kernel<<<c.nblk_node, kTPB, 0, s>>>(a);
    launch_cg_init_scalars(a, tol, max_iters, s);
    return 4 + l;
}

int cgc_iteration(const CGArgs& a, const CGCPlan& c, const MGPlan& mg, cudaStream_t s) {
    elem_apply_n(c, a.p, a.ctl, s);
    NodeArgs na = node_args(c, a.ctl);
    na.v = a.p;
    na.out = a.q;
    na.part = a.part;
    cgc_node_kernel<NODE_SPMV><<<c.nblk_node, kTPB, 0, s>>>(na);
    launch_cgx_update(a, s);
    const int l = cgc_mg(c, mg, a.r, a.z, a.ctl, s);
    launch_cgx_rz(a, s);
    launch_cgx_direction(a, s);
    return 5 + l;
}

}  // namespace smm

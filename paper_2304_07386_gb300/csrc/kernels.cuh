// Device kernels of the SMM hot path (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace smm {

// Device error word values (first error wins).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_NONFINITE = 2 };

// Sweep modes: SOURCE solves L psi = sigma_s/(4pi) varphi + q with the
// inflow data; RESIDUAL solves L delta = r (r given per element and
// ordinate, homogeneous inflow) and accumulates delta into an FP64 flux.
enum : int { SWEEP_SOURCE = 0, SWEEP_RESIDUAL = 1 };

template <typename T>
struct SweepArgs {
    int ne, nd, ntask, p;
    const int32_t* tasks;      // e*nd + d, sorted by upwind level
    const double* ox;          // [nd]
    const double* oy;          // [nd]
    const double* sigma_t;     // [ne]
    const double* sigma_s;     // [ne]
    const T* M;                // [ne][n][n] row = test function
    const T* Gx;
    const T* Gy;
    const T* Fx;               // [ne][4][p1][p1]
    const T* Fy;
    const int8_t* fdir;        // [ne][nd][4]
    const int32_t* nbr;        // [ne][4]
    const int32_t* nbr_face;
    const int32_t* nbr_flip;
    const int32_t* bface_id;
    const double* phi;         // [ne][n] or nullptr (SOURCE)
    const double* src;         // [ne][n] isotropic or [ne][nd][n] (SOURCE)
    int src_angular;
    const double* inflow;      // [nb][nd][p1] or nullptr (SOURCE)
    const float* rhs;          // [ne][nd][n] (RESIDUAL)
    const T* ainv;             // cached local inverses [ne*nd][n][n] column-major, or nullptr (on-the-fly LU)
    const float2* ainv_df;     // FP64 cached mode: the same inverses as FP32 pairs (hi, lo), hi + lo = entry
    // FP64 cached mode, pair copies: M (s + q_iso) of this sweep [ne][n], M q_d [ne][nd][n] or nullptr,
    // ordinate cosines [nd], face matrices [ne][4][p1][p1], inflow [nb][nd][p1] or nullptr
    const float2* msrc2;
    const float2* mq2;
    const float2* ox2;
    const float2* oy2;
    const float2* Fx2;
    const float2* Fy2;
    const float2* inflow2;
    float2* psi2;              // FP64 cached mode: psi as pairs (read by downwind tasks and the moments)
    // lagged inflow (fdir -2 or 3: across tiles of a block Jacobi sweep, or closing a cycle): the
    // previous sweep's psi
    const T* psi_lag;
    const float2* psi2_lag;
    // faces that are inflow at some quadrature points and outflow at others (fdir 2, or 3 when
    // lagged): id [ne][nd][4] of their pointwise face matrices fmix[id][2][p1][p1] (outflow part,
    // inflow part), FP64 and as FP32 pairs; nullptr when the mesh has none
    const int32_t* fmix_id;
    const double* fmix;
    const float2* fmix2;
    // zero and scale negative flux fixup (source mode): column sums of M, Gx, Gy [ne][n] and of the
    // face matrices Fx, Fy over their test index [ne][4][p1]
    int fixup;
    const double* colM;
    const double* colGx;
    const double* colGy;
    const double* colFx;
    const double* colFy;
    const double* msrc;        // cached mode, SOURCE: [ne][n] M (sigma_s/(4pi) phi + q_iso) of this sweep
    const double* mq;          // cached mode, SOURCE, angular q: [ne][nd][n] M q_d, else nullptr
    T* psi;                    // [ne][nd][n] output, read by downwind tasks (not written in FP64
                               // cached mode, whose flux is psi2)
    double* psi_acc;           // RESIDUAL: psi_acc += psi
    // Angular moments fused into the sweep (Eqs. correction_tensor_disc, bdr_correction_factor_disc):
    // once every warp of the launch has finished its tasks (the gate), warp k forms the moments of
    // elements k, k + warps, ... and the boundary correction at the Gauss points of their boundary
    // faces.  mom == nullptr: no moments.
    unsigned* gate;            // warps arrived after their last task (zero at launch; one per launch)
    const double* w;           // [nd] ordinate weights
    const float2* wq2;         // FP64 cached mode: [6][nd] pairs of w_d (1, Ox, Oy, OxOx, OxOy, OyOy)
    const double* mpsi;        // other modes: the FP64 flux the moments read, [ne][nd][n]
    double* mom;               // [6][ne][n]: phi, Jx, Jy, Txx, Txy, Tyy
    double* beta;              // [nb][nfq]
    int nfq;
    const double* L1;          // [nfq][p1] face nodal values -> Gauss points
    const double* nhat;        // [nb][nfq][2] outward unit normals
    const double* eb0;         // [nb][nfq]
    unsigned* done;            // [ne*nd] epoch flags
    unsigned epoch;
    unsigned* ticket;          // task counter, zero at launch
    int* err;
    long long timeout_ns;
};

struct ResidualArgs {
    int ne, nd, ntask;
    const double* ox;
    const double* oy;
    const double* sigma_t;
    const double* sigma_s;
    const double* M;
    const double* Gx;
    const double* Gy;
    const double* Fx;
    const double* Fy;
    const int8_t* fdir;
    const int32_t* nbr;
    const int32_t* nbr_face;
    const int32_t* nbr_flip;
    const int32_t* bface_id;
    const double* phi;
    const double* src;
    int src_angular;
    const double* inflow;
    const double* psi;         // [ne][nd][n] FP64 current iterate
    float* rhs;                // [ne][nd][n] residual (out)
};

template <typename T>
void launch_sweep(int p, int mode, const SweepArgs<T>& a, int grid, cudaStream_t s);
// many problems in one cooperative launch; tasks: (problem, task) pairs sorted by level; elems:
// (problem, element) of every element of every problem
// ext: some problem uses the fixup, tiles or lagged / mixed faces (the kernel with those parts compiled in)
// pmax: the largest order p among the batch's problems
template <typename T>
cudaError_t launch_batch_sweep(int mode, bool cached, bool ext, int pmax, const SweepArgs<T>* args, const int2* tasks,
                               int ntask, const int2* elems, int nelem, int grid, int block, cudaStream_t s);
int batch_blocks_per_sm(int mode, bool fp32, bool cached, bool ext, int pmax, int block);
// form every local inverse A_{K,d}^{-1} (column-major, type T) in ainv_out
template <typename T>
void launch_invert(int p, const SweepArgs<T>& a, T* ainv_out, cudaStream_t s);
// FP64 local inverses stored as FP32 pairs (hi, lo) with hi + lo = the FP64 entry to 2^-48
void launch_invert_df(int p, const SweepArgs<double>& a, float2* ainv_out, cudaStream_t s);
// out[e][d][i] = scale * sum_j M[e][i][j] in[e][d][j] (+ add[e][i] * scale2 if add) ; nd = 1 for per-element data
void launch_mass_apply(int ne, int nd, int n, const double* M, const double* in, float2* out, cudaStream_t s);
// msrc[e][i] = sum_j M[e][i][j] (c_e phi[e][j] + q[e][j]); phi, q nullable
void launch_source(int ne, int n, const double* M, const double* sigma_s, const double* phi, const double* q_iso,
                   float2* msrc, cudaStream_t s);
void launch_residual(int p, const ResidualArgs& a, cudaStream_t s);
int sweep_blocks_per_sm(int p, int mode, bool fp32, bool cached);

// the FP64 value hi + lo of each of n FP32 pairs
void launch_pairs_to_f64(size_t n, const float2* in, double* out, cudaStream_t s);

void launch_rhs(int ne, int n, int p, int nfq, const double* mom, const double* beta, const double* bfixed,
                const float2* Kxx, const float2* Ks, const float2* Kyy, const float2* Dfx, const float2* Dfy,
                const float2* DfxT, const float2* DfyT, const double* nds, const double* L1, const double* sigma_t,
                const int32_t* nbr, const int32_t* nbr_face, const int32_t* nbr_flip, const int32_t* bface_id,
                const double* b_ds, double* trace, double* rhs, cudaStream_t s);

// IP-SMM moment operator: diagonal blocks plus face-factored neighbour
// blocks A_{e,e2} = E_f^T C_{e,f} E_f2, where E_f extracts the p+1 trace
// values and p+1 reference normal derivatives sum_t wd[t] u(line t) of one
// face (G = 2(p+1) face data)
template <typename T>
struct FaceOp {
    const T* AdT = nullptr;          // [ne][n][n] transposed (col-major per block)
    const T* CT = nullptr;           // [ne][4][G][G], CT[((e*4+f)*G + c)*G + r] = C_{e,f}[r][c]
    const int32_t* nbr = nullptr;    // [ne][4] neighbour element or -1
    const int32_t* nface = nullptr;  // [ne][4] the neighbour's local index of the shared face
    T wd[5] = {};                    // l'_t(0) of the 1D Gauss-Lobatto basis, t < p+1
};

// the same operator with every entry stored as an FP32 pair (hi, lo)
struct FaceOpDF {
    const float2* AdT = nullptr;
    const float2* CT = nullptr;
    const int32_t* nbr = nullptr;
    const int32_t* nface = nullptr;
    float2 wd[5] = {};
};

// block-Jacobi PCG
struct CGArgs {
    int ne, n, nrow, nblk;     // nblk: blocks of the row kernels
    FaceOp<double> A;          // operator (FP64)
    FaceOpDF A2;               // operator as FP32 pairs (flexible-CG product), AdT == nullptr if absent
    float2* p2;                // flexible CG: the direction p as FP32 pairs, kept with p
    // dense alternative (caller-provided blocks, any n <= 64): used when AoT_dense is set
    const double* AdT_dense;   // [ne][n][n] transposed
    const double* AoT_dense;   // [ne][4][n][n] transposed
    const int32_t* nbr_dense;  // [ne][4]
    const double* PinvT;       // [ne][n][n] transposed
    double* x;
    double* r;
    double* z;
    double* p;
    double* q;
    double* rold;              // previous residual (flexible CG), may be nullptr on the block-Jacobi path
    const double* b;
    double* part;              // [3][nblk] partial sums
    double* pvec;              // [3][nvblk] partial sums of the grid-stride vector kernels (flexible CG)
    int nvblk;                 // blocks of the grid-stride vector kernels
    double* scal;              // [8]: rz, pq, rr, bb, thresh2, -, -, -
    int* ctl;                  // [4]: done, iters, max_iters, nonfinite
};
// multigrid preconditioner (device side of an MGHierarchy); levels >= 1 in
// FP32.  Their sparse matrices are stored as k-major ELL: entry k of row i at
// [k * rows + i], every row padded to the longest one with value 0 (column of
// the row's first entry), so that a warp's loads of one k over consecutive
// rows are coalesced and a row's loads are independent of each other.
struct MGLevelDev {
    int n = 0;                                   // unknowns on this level
    int aw = 0;                                  // A: n rows of width aw
    const int* Aci = nullptr; const float* Av = nullptr;
    const float* Asv = nullptr;                  // A diag(omega dinv): the values of A scaled by column
    const float* dinv = nullptr;
    float omega = 0.0f;
    int pw = 0;                                  // P (from level l+1): n rows of width pw
    const int* Pci = nullptr; const float* Pv = nullptr;
    int rw = 0;                                  // R (to level l+1): n_{l+1} rows of width rw
    const int* Rci = nullptr; const float* Rv = nullptr;
    float* b = nullptr; float* x = nullptr; float* r = nullptr; float* t = nullptr;
};
// a 16-byte-aligned span (size a multiple of 16) of read-only device data that a
// kernel prefetches into L2 ahead of the kernel that reads it
struct L2Chunk {
    const void* p;
    unsigned bytes;
    unsigned pad;
};
struct MGPlan {
    bool enabled = false;
    int ne = 0, n = 0, nu0 = 2;
    double omega0 = 0.0;                          // Jacobi damping (4/3) / lambda_max
    bool chebyshev = false;                       // level-0 smoother: Chebyshev polynomial of degree nu0
    FaceOp<float> A;                              // FP32 copy of the operator
    const float* PinvT = nullptr;                 // FP32 block-Jacobi inverses
    const float* WdT = nullptr;                   // [ne][n][4]: w4^T A_d, the diagonal blocks' part of the corner sums
    float* x0 = nullptr; float* x0b = nullptr;   // [ne*n], level 0 works in FP32
    float* res0 = nullptr;                        // [ne][4] element-corner sums of the level-0 residual
    int nvert = 0;
    const int* vid = nullptr; const float* w4 = nullptr;
    int vw = 0;                                   // vertex -> incident (element*4 + corner) as k-major ELL
    const int* vinc = nullptr;                    // [vw][nvert], -1 padding
    int nlev = 0;                                 // levels 1..nlev (nlev = coarsest, dense)
    int coarse_ctas = 8;                          // cluster size of the coarse-level launch
    MGLevelDev lv[12];
    const float* cinv = nullptr;                  // [nc][nc] row-major
    const L2Chunk* coarse_pf = nullptr;           // the coarse levels' read-only data in 32 KB chunks
    int coarse_npf = 0;
};
// cluster size for the coarse-level launch on the current device (8 or 16)
int mg_coarse_cluster_size();
// the coarse part of the V-cycle (vertex level from element-corner residual
// sums cres [ne][4], aggregation levels, coarsest solve) as one cluster
// launch, or, for a large vertex level, that level's stages as grid kernels
// around a cluster launch for the levels below; returns the vertex-level
// correction (device pointer, nvert floats); *launches = kernels launched
const float* launch_coarse_cycle(const MGPlan& m, const float* cres, const int* ctl, cudaStream_t s, int* launches);
bool mg_split_vertex_level(const MGPlan& m);
// z = V-cycle(r); returns the number of kernel launches; the kernels return at once when ctl[0]
// (CG finished) is set
int mg_apply(const MGPlan& m, const double* r, double* z, const int* ctl, cudaStream_t s);
// one flexible-CG iteration's V-cycle with the update and the dot products folded into the level-0
// steps (IP system, element blocks); returns the number of launches
int mg_cg_iteration(const MGPlan& m, const CGArgs& a, cudaStream_t s);

void cg_start(const CGArgs& a, double tol, int max_iters, cudaStream_t s);
// the loop-control kernel that ends a trip of the device-side CG loop (ctl[5] counts the trips)
void launch_cg_loop_control(cudaGraphConditionalHandle handle, int* ctl, cudaStream_t s);
void launch_cgx_update(const CGArgs& a, cudaStream_t s);
void launch_cgx_rz(const CGArgs& a, cudaStream_t s);
void launch_cgx_direction(const CGArgs& a, cudaStream_t s);
void launch_cg_init_scalars(const CGArgs& a, double tol, int max_iters, cudaStream_t s);

// Continuous (CG) moment system, Sec. 5.1: element blocks on the continuous
// node numbering, a V-cycle with point-Jacobi smoothing on the continuous
// nodes over the same vertex / aggregation levels
struct CGCPlan {
    bool enabled = false;
    int ne = 0, n = 0, nglob = 0, nu = 2, nblk_node = 1;
    double omega = 0.0;                           // damping of the point-Jacobi smoother
    const double* KT = nullptr;                   // [ne][n][n] column-major element blocks
    const int* gid = nullptr;                     // [ne][n] global node of each element node
    const int* grp = nullptr;                     // [nglob+1] element nodes of each global node (CSR)
    const int* ginc = nullptr;                    // [ne*n]
    const int* gown = nullptr;                    // [nglob] first element node of each global node
    const float* minv = nullptr;                  // [nglob] 1 / number of element nodes
    const double* dinv = nullptr;                 // [nglob] 1 / diag(A_CG)
    double* ye = nullptr;                         // [ne][n] element products
    double* xa = nullptr;                         // [nglob] V-cycle iterates
    double* xb = nullptr;
    double* res = nullptr;                        // [nglob] level-0 residual
    float* cres = nullptr;                        // [ne][4] its element-corner restriction
};
// b = P^T b_dg (sum over the element nodes of each global node)
void cgc_gather(const CGCPlan& c, const double* b_dg, double* b, cudaStream_t s);
// dg = P x ; x = value of each global node's first element node
void cgc_expand(const CGCPlan& c, const double* x, double* dg, cudaStream_t s);
void cgc_pick(const CGCPlan& c, const double* dg, double* x, cudaStream_t s);
// flexible CG on the continuous system: a.nrow = nglob, a.nblk = c.nblk_node
int cgc_start(const CGArgs& a, const CGCPlan& c, const MGPlan& mg, double tol, int max_iters, cudaStream_t s);
int cgc_iteration(const CGArgs& a, const CGCPlan& c, const MGPlan& mg, cudaStream_t s);
int cgx_start(const CGArgs& a, double tol, int max_iters, const MGPlan& mg, cudaStream_t s);
int cgx_iterations(const CGArgs& a, int count, const MGPlan& mg, cudaStream_t s);
void cg_iterations(const CGArgs& a, int count, cudaStream_t s);
int cg_threads_per_block(int n);

// Anderson acceleration helpers: Gram matrix of up to 6 vectors (21 pairwise
// dots, deterministic two-stage reduction) and the mixing update
struct VecSet {
    const double* v[6];
    int nv;
};
void launch_gram(int nrow, const VecSet& vs, double* part, double* out, cudaStream_t s);
// x = G[0] - sum_j gamma[j] (G[j] - G[j+1]), j = 0..m-1 (G[0] newest)
struct MixArgs {
    const double* G[6];
    double gamma[5];
    int m;
};
void launch_anderson_mix(int nrow, const MixArgs& a, double* x, cudaStream_t s);
// out = alpha x + beta y
void launch_axpby(int nrow, double alpha, const double* x, double beta, const double* y, double* out, cudaStream_t s);

// message returned by smm_last_error() for the calling thread
void set_last_error(const char* msg);

// outer step: diff = max|new - old|, max|new|, nonfinite check
void launch_diff(int nrow, const double* a, const double* b, double* part, double* out, int* flag, cudaStream_t s);

}  // namespace smm

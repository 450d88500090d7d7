// C ABI of the SMM library (include/smm.h): handle, device buffers and the
// outer fixed-point driver (paper Eqs. moment:smm_fp and fixed-point).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/smm.h"
#include "amg.hpp"
#include "kernels.cuh"
#include "setup.hpp"

namespace {

thread_local std::string g_err;

smm_status fail(smm_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

}  // namespace

void smm::set_last_error(const char* msg) { g_err = msg; }

namespace {

#define SMM_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(SMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

struct smm_ctx {
    int ne = 0, m = 1, p = 1, p1 = 2, n = 4, nd = 0, nb = 0, nfq = 0, nlevels = 0, ntask = 0;
    int src_angular = 0, has_inflow = 0;
    bool fp32 = false;
    smm_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0, sms = 1, sweep_grid = 1;
    unsigned epoch = 0;
    std::vector<void*> allocs;
    // quadrature / connectivity
    double *ox = nullptr, *oy = nullptr, *w = nullptr, *sigma_t = nullptr, *sigma_s = nullptr;
    int32_t *tasks = nullptr, *nbr = nullptr, *nbr_face = nullptr, *nbr_flip = nullptr, *bface_id = nullptr;
    int32_t *bface_elem = nullptr, *bface_face = nullptr;
    int8_t* fdir = nullptr;
    unsigned* gate = nullptr;      // the sweep's gate before its moment reductions (one word)
    // sweep matrices
    double *M = nullptr, *Gx = nullptr, *Gy = nullptr, *Fx = nullptr, *Fy = nullptr;
    float *M32 = nullptr, *Gx32 = nullptr, *Gy32 = nullptr, *Fx32 = nullptr, *Fy32 = nullptr;
    double *src = nullptr, *inflow = nullptr;
    bool cached = false;
    float2* ainv_df = nullptr;     // cached local inverses (FP64 sweep), FP32 pairs hi + lo
    // extrapolated CG start (options.cg_guess_extrapolate): the previous outer
    // step's input and the last two successive differences (0: not yet)
    double* phi_old = nullptr;
    double dl1 = 0.0, dl2 = 0.0;
    float* ainv32 = nullptr;       // cached local inverses (FP32 correction sweep)
    // FP64 cached sweep, FP32-pair inputs: M (sigma_s/(4pi) phi + q_iso) of the current sweep [ne][n],
    // M q_d [ne][nd][n] (angular sources), cosines [nd], face matrices, inflow; psi as pairs
    float2* msrc2 = nullptr;
    float2* mq2 = nullptr;
    float2 *ox2 = nullptr, *oy2 = nullptr, *Fx2 = nullptr, *Fy2 = nullptr, *inflow2 = nullptr;
    float2* psi2 = nullptr;
    float2* wq2 = nullptr;         // [6][nd] pairs of w_d (1, Ox, Oy, OxOx, OxOy, OyOy) for the pair moments
    double* psi_lag = nullptr;     // lagged inflow: previous sweep's psi (on-the-fly LU mode)
    float2* psi2_lag = nullptr;    // ... and its pairs (cached-inverse mode)
    bool lagging = false;          // some inflow is lagged (block Jacobi tiles or cycles)
    int64_t n_lagged = 0;          // (element, ordinate, face) inflows lagged to break cycles
    int32_t* fmix_id = nullptr;    // mixed faces: pointwise face matrices (see SweepArgs)
    double* fmix = nullptr;
    float2* fmix2 = nullptr;
    // negative flux fixup: column sums of M, Gx, Gy [ne][n] and of Fx, Fy over the test index [ne][4][p1]
    double *colM = nullptr, *colGx = nullptr, *colGy = nullptr, *colFx = nullptr, *colFy = nullptr;
    std::vector<int32_t> tasks_host, level_start;  // level-sorted task list (for batching)
    // Anderson acceleration: rings of G(x_k) and f_k = G(x_k) - x_k (depth + 1 slots)
    std::vector<double*> aaG, aaF;
    double *aa_part = nullptr, *aa_out = nullptr;
    int aa_k = 0;                  // outer steps in the current Anderson history (0: empty)
    double* phi_io = nullptr;      // device copy of a host iterate passed to smm_iterate
    // state
    double* psi = nullptr;         // [ne][nd][n] FP64 (not kept in FP64 cached mode: psi2 holds the flux)
    float* dpsi = nullptr;         // [ne][nd][n] FP32 correction (refined mode)
    float* res = nullptr;          // [ne][nd][n] FP32 residual (refined mode)
    unsigned* done = nullptr;
    unsigned* ticket = nullptr;
    int* err = nullptr;
    double *mom = nullptr, *beta = nullptr;
    // closures / rhs data
    double *L1 = nullptr, *b_nhat = nullptr, *b_ds = nullptr, *b_eb0 = nullptr;
    double* nds = nullptr;
    // right-hand-side operators as FP32 pairs: K blocks column-major, the face gradient operators
    // point-major (Dfx, Dfy) and node-major (DfxT, DfyT)
    float2 *Kxx = nullptr, *Ks = nullptr, *Kyy = nullptr, *Dfx = nullptr, *Dfy = nullptr;
    float2 *DfxT = nullptr, *DfyT = nullptr;
    double *bfixed = nullptr, *trace = nullptr, *rhs = nullptr;
    // moment operator and CG
    double *AdT = nullptr, *CT = nullptr, *PinvT = nullptr;   // diagonal blocks, face couplings, inverses
    float2 *AdT2 = nullptr, *CT2 = nullptr;                    // the same as FP32 pairs (flexible-CG product)
    float2* p2 = nullptr;                                       // CG direction as FP32 pairs
    double wd[5] = {0, 0, 0, 0, 0};
    double *r = nullptr, *z = nullptr, *pv = nullptr, *qv = nullptr, *part = nullptr, *scal = nullptr;
    double *phi_prev = nullptr, *dpart = nullptr, *dout = nullptr;
    int* ctl = nullptr;
    int* nonfinite = nullptr;
    int cg_nblk = 1;
    int cg_nvblk = 1;              // blocks of the grid-stride CG vector kernels
    int cg_pmax = 1;               // room per partial-sum array
    smm::MGPlan mg;
    smm::CGCPlan cgc;              // continuous (CG) moment system, when selected
    double* bc = nullptr;          // its right-hand side P^T b_IP [nglob]
    double* xc = nullptr;          // its CG iterate [nglob]
    double* rold = nullptr;        // flexible CG: previous residual
    double* xcg = nullptr;         // CG iterate owned by the handle (captured in the iteration graph)
    cudaStream_t cap = nullptr;    // private stream used once to capture the CG iteration graph
    cudaGraphExec_t cg_graph = nullptr;
    cudaGraphExec_t cg_loop = nullptr;   // the whole CG loop (while node over one iteration); null: chunked launches
    int graph_kernels = 0;
    // pinned host scratch
    double* h_scal = nullptr;
    int* h_int = nullptr;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    long long launches = 0;

    // every array carries 16 bytes of slack after its end, so that a bulk
    // prefetch of a span rounded up to 16 bytes stays inside the allocation
    template <class T>
    T* alloc(size_t count) {
        if (count == 0) count = 1;
        void* ptr = nullptr;
        if (cudaMalloc(&ptr, count * sizeof(T) + 16) != cudaSuccess) return nullptr;
        allocs.push_back(ptr);
        return (T*)ptr;
    }
    ~smm_ctx() {
        if (cg_graph) cudaGraphExecDestroy(cg_graph);
        if (cg_loop) cudaGraphExecDestroy(cg_loop);
        if (cap) cudaStreamDestroy(cap);
        for (void* ptr : allocs) cudaFree(ptr);
        if (h_scal) cudaFreeHost(h_scal);
        if (h_int) cudaFreeHost(h_int);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

template <class T>
bool upload(smm_ctx* h, T*& dst, const std::vector<T>& src) {
    dst = h->alloc<T>(src.size());
    if (!dst) return false;
    if (src.empty()) return true;
    return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
}

template <class T>
bool upload_f32(smm_ctx* h, float*& dst, const std::vector<T>& src) {
    std::vector<float> tmp(src.begin(), src.end());
    bool ok = upload(h, dst, tmp);
    return ok && cudaStreamSynchronize(h->stream) == cudaSuccess;
}

// transpose each n x n block ([blk][i][j] -> [blk][j][i])
// k-major ELL copy of a CSR pattern with values val (in CSR order): entry k
// of row i at [k * nrow + i]; width = the longest row; padding entries repeat
// the row's first column (column 0 for an empty row) with value 0
void to_ell(const smm::CSR& A, const std::vector<double>& val, int& width, std::vector<int>& ci,
            std::vector<float>& v) {
    width = 0;
    for (int i = 0; i < A.nrow; ++i) width = std::max(width, A.rp[i + 1] - A.rp[i]);
    ci.assign((size_t)width * A.nrow, 0);
    v.assign((size_t)width * A.nrow, 0.0f);
    for (int i = 0; i < A.nrow; ++i) {
        const int k0 = A.rp[i], len = A.rp[i + 1] - k0;
        for (int k = 0; k < width; ++k) {
            const size_t o = (size_t)k * A.nrow + i;
            ci[o] = k < len ? A.ci[k0 + k] : (len > 0 ? A.ci[k0] : 0);
            v[o] = k < len ? (float)val[k0 + k] : 0.0f;
        }
    }
}

// FP32 pairs (hi, lo) with hi + lo = v to 2^-48
std::vector<float2> to_pairs(const std::vector<double>& v) {
    std::vector<float2> out(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        const float hi = (float)v[i];
        out[i] = make_float2(hi, (float)(v[i] - (double)hi));
    }
    return out;
}

std::vector<double> transpose_blocks(const std::vector<double>& a, int n) {
    std::vector<double> t(a.size());
    const size_t nb = a.size() / ((size_t)n * n);
    for (size_t b = 0; b < nb; ++b)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) t[b * n * n + (size_t)j * n + i] = a[b * n * n + (size_t)i * n + j];
    return t;
}

}  // namespace

namespace {
smm::CGArgs cg_args(smm_handle h, double* x);
smm::CGArgs cgc_args(smm_handle h);
smm_status setup_cg_moment_system(smm_handle h, const smm::Setup& s);
}

extern "C" {

void smm_default_options(smm_options* opt) {
    if (!opt) return;
    opt->sweep_precision = SMM_SWEEP_FP64;
    opt->tol_cg = 1e-12;
    opt->max_cg = 20000;
    opt->kappa_scale = 1.0;
    opt->spin_timeout_s = 2.0;
    opt->precond = SMM_PRECOND_MULTIGRID;
    opt->sweep_solver = SMM_SOLVER_CACHED_INVERSE;
    opt->anderson_depth = 0;
    opt->guess_check = 0;
    opt->mg_smooth_steps = 3;
    opt->moment_discretization = SMM_MOMENT_IP;
    opt->negative_flux_fixup = 0;
    opt->sweep_tiles = 1;
    opt->mg_smoother = SMM_SMOOTHER_CHEBYSHEV;
    opt->cg_device_loop = 1;
    opt->resume_history = 0;
    opt->cycle_lagging = 1;
    opt->cg_tol_adaptive = 0.0;
    opt->cg_guess_extrapolate = 1;
}

const char* smm_last_error(void) { return g_err.c_str(); }

smm_status smm_quadrature(int32_t sn_order, double* omega_out, double* w_out, int32_t* n_ord_out) {
    smm::Quadrature q;
    if (!smm::level_symmetric(sn_order, q)) return fail(SMM_ERR_INVALID_ARG, "unsupported S_N order");
    for (int d = 0; d < q.nd; ++d) {
        if (omega_out) { omega_out[2 * d] = q.ox[d]; omega_out[2 * d + 1] = q.oy[d]; }
        if (w_out) w_out[d] = q.w[d];
    }
    if (n_ord_out) *n_ord_out = q.nd;
    return SMM_OK;
}

smm_status smm_create(const smm_mesh* mesh, int32_t p, int32_t sn_order, const double* sigma_t, const double* sigma_s,
                      int32_t source_kind, const double* q, int32_t inflow_kind, const double* inflow,
                      const smm_options* opt, void* cuda_stream, smm_handle* out) {
    if (!out) return fail(SMM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!mesh) return fail(SMM_ERR_INVALID_ARG, "mesh is NULL");
    if (source_kind != SMM_SOURCE_ISOTROPIC && source_kind != SMM_SOURCE_ANGULAR)
        return fail(SMM_ERR_INVALID_ARG, "bad source kind");
    if (inflow_kind != SMM_INFLOW_VACUUM && inflow_kind != SMM_INFLOW_NODAL)
        return fail(SMM_ERR_INVALID_ARG, "bad inflow kind");
    smm_options o;
    smm_default_options(&o);
    if (opt) o = *opt;
    if (o.sweep_precision != SMM_SWEEP_FP64 && o.sweep_precision != SMM_SWEEP_FP32_REFINED)
        return fail(SMM_ERR_INVALID_ARG, "bad sweep precision");
    if (!(o.tol_cg > 0) || o.max_cg < 1 || !(o.kappa_scale > 0) || !(o.spin_timeout_s > 0) || !(o.cg_tol_adaptive >= 0) ||
        (o.precond != SMM_PRECOND_BLOCK_JACOBI && o.precond != SMM_PRECOND_MULTIGRID) ||
        (o.sweep_solver != SMM_SOLVER_LU && o.sweep_solver != SMM_SOLVER_CACHED_INVERSE) || o.anderson_depth < 0 ||
        o.anderson_depth > 5 || o.mg_smooth_steps < 1 || o.mg_smooth_steps > 4 ||
        (o.moment_discretization != SMM_MOMENT_IP && o.moment_discretization != SMM_MOMENT_CG) ||
        (o.negative_flux_fixup && o.sweep_precision != SMM_SWEEP_FP64) || o.sweep_tiles < 1 || o.sweep_tiles > 64 ||
        (o.sweep_tiles > 1 && o.sweep_precision != SMM_SWEEP_FP64) ||
        (o.mg_smoother != SMM_SMOOTHER_JACOBI && o.mg_smoother != SMM_SMOOTHER_CHEBYSHEV))
        return fail(SMM_ERR_INVALID_ARG, "bad options");

    smm::Input in;
    in.ne = mesh->n_elem; in.m = mesh->geom_order; in.p = p; in.sn = sn_order; in.n_nodes = mesh->n_nodes;
    in.nodes = mesh->nodes; in.elem_nodes = mesh->elem_nodes; in.sigma_t = sigma_t; in.sigma_s = sigma_s;
    in.source_kind = source_kind; in.q = q; in.inflow_kind = inflow_kind; in.inflow = inflow;
    in.kappa_scale = o.kappa_scale;
    in.moment_cg = o.moment_discretization == SMM_MOMENT_CG;
    in.sweep_tiles = o.sweep_tiles;
    in.lag_cycles = o.cycle_lagging ? 1 : 0;
    smm::Setup s;
    std::string err;
    int rc = smm::build_setup(in, s, err);
    if (rc != 0) return fail((smm_status)rc, err);
    if ((s.n_cycle_lagged > 0 || s.n_mixed > 0) &&
        (o.sweep_precision != SMM_SWEEP_FP64 || o.negative_flux_fixup))
        return fail(SMM_ERR_CYCLE, "the upwind graphs have cycles: cycle lagging needs the FP64 sweep without the "
                                   "negative flux fixup");

    smm_ctx* h = new smm_ctx();
    h->opt = o;
    h->stream = (cudaStream_t)cuda_stream;
    h->ne = s.ne; h->m = s.m; h->p = s.p; h->p1 = s.p1; h->n = s.n; h->nd = s.nd; h->nb = s.nb; h->nfq = s.nfq;
    h->nlevels = s.nlevels; h->ntask = (int)s.tasks.size();
    h->tasks_host = s.tasks;
    h->level_start = s.level_start;
    h->src_angular = source_kind == SMM_SOURCE_ANGULAR;
    h->has_inflow = !s.inflow.empty();
    h->fp32 = o.sweep_precision == SMM_SWEEP_FP32_REFINED;
    auto bail = [&](smm_status st, const std::string& msg) { delete h; return fail(st, msg); };
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(SMM_ERR_CUDA, "cudaGetDevice failed");
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);

    bool ok = true;
    ok &= upload(h, h->ox, s.quad.ox) && upload(h, h->oy, s.quad.oy) && upload(h, h->w, s.quad.w);
    ok &= upload(h, h->sigma_t, s.sigma_t) && upload(h, h->sigma_s, s.sigma_s);
    ok &= upload(h, h->tasks, s.tasks) && upload(h, h->fdir, s.fdir);
    ok &= upload(h, h->nbr, s.nbr) && upload(h, h->nbr_face, s.nbr_face) && upload(h, h->nbr_flip, s.nbr_flip);
    ok &= upload(h, h->bface_id, s.bface_id) && upload(h, h->bface_elem, s.bface_elem) && upload(h, h->bface_face, s.bface_face);
    ok &= upload(h, h->M, s.M) && upload(h, h->Gx, s.Gx) && upload(h, h->Gy, s.Gy);
    ok &= upload(h, h->Fx, s.Fx) && upload(h, h->Fy, s.Fy);
    ok &= upload(h, h->src, s.src) && upload(h, h->inflow, s.inflow);
    ok &= upload(h, h->L1, s.L1) && upload(h, h->b_nhat, s.b_nhat) && upload(h, h->b_ds, s.b_ds) && upload(h, h->b_eb0, s.b_eb0);
    // column-major (transposed) blocks, so that the n threads of an element read contiguous entries
    ok &= upload(h, h->Kxx, to_pairs(transpose_blocks(s.Kxx, s.n))) &&
          upload(h, h->Ks, to_pairs(transpose_blocks(s.Ks, s.n))) &&
          upload(h, h->Kyy, to_pairs(transpose_blocks(s.Kyy, s.n)));
    ok &= upload(h, h->Dfx, to_pairs(s.Dfx)) && upload(h, h->Dfy, to_pairs(s.Dfy)) && upload(h, h->nds, s.nds) &&
          upload(h, h->bfixed, s.bfixed);
    {
        // [element][face][node][point] copies for the trace kernel, whose threads are face points
        const int nq = s.nfq, nn = s.n;
        const size_t nb = (size_t)s.ne * 4;
        std::vector<double> tx(s.Dfx.size()), ty(s.Dfy.size());
        for (size_t b = 0; b < nb; ++b)
            for (int q = 0; q < nq; ++q)
                for (int j = 0; j < nn; ++j) {
                    tx[(b * nn + j) * nq + q] = s.Dfx[(b * nq + q) * nn + j];
                    ty[(b * nn + j) * nq + q] = s.Dfy[(b * nq + q) * nn + j];
                }
        ok &= upload(h, h->DfxT, to_pairs(tx)) && upload(h, h->DfyT, to_pairs(ty));
    }
    if (!ok) return bail(SMM_ERR_OOM, "device allocation or upload failed");
    if (o.negative_flux_fixup) {
        const size_t nn = (size_t)s.n * s.n;
        std::vector<double> cm((size_t)s.ne * s.n, 0.0), cgx(cm.size(), 0.0), cgy(cm.size(), 0.0);
        std::vector<double> cfx((size_t)s.ne * 4 * s.p1, 0.0), cfy(cfx.size(), 0.0);
        for (int e = 0; e < s.ne; ++e) {
            for (int i = 0; i < s.n; ++i)
                for (int j = 0; j < s.n; ++j) {
                    cm[(size_t)e * s.n + j] += s.M[e * nn + (size_t)i * s.n + j];
                    cgx[(size_t)e * s.n + j] += s.Gx[e * nn + (size_t)i * s.n + j];
                    cgy[(size_t)e * s.n + j] += s.Gy[e * nn + (size_t)i * s.n + j];
                }
            for (int f = 0; f < 4; ++f)
                for (int a = 0; a < s.p1; ++a)
                    for (int b = 0; b < s.p1; ++b) {
                        const size_t fo = (((size_t)e * 4 + f) * s.p1 + a) * s.p1 + b;
                        cfx[((size_t)e * 4 + f) * s.p1 + b] += s.Fx[fo];
                        cfy[((size_t)e * 4 + f) * s.p1 + b] += s.Fy[fo];
                    }
        }
        ok &= upload(h, h->colM, cm) && upload(h, h->colGx, cgx) && upload(h, h->colGy, cgy) &&
              upload(h, h->colFx, cfx) && upload(h, h->colFy, cfy);
        if (!ok) return bail(SMM_ERR_OOM, "device allocation or upload failed");
    }
    {
        std::vector<double> t = transpose_blocks(s.Adiag, s.n);
        ok &= upload(h, h->AdT, t);
        ok &= upload(h, h->AdT2, to_pairs(t));
        t = transpose_blocks(s.Cface, 2 * s.p1);
        ok &= upload(h, h->CT, t);
        ok &= upload(h, h->CT2, to_pairs(t));
        for (int k = 0; k < s.p1; ++k) h->wd[k] = s.wd[k];
        t = transpose_blocks(s.Pinv, s.n);
        ok &= upload(h, h->PinvT, t);
        ok &= cudaStreamSynchronize(h->stream) == cudaSuccess;
    }
    if (h->fp32) {
        ok &= upload_f32(h, h->M32, s.M) && upload_f32(h, h->Gx32, s.Gx) && upload_f32(h, h->Gy32, s.Gy);
        ok &= upload_f32(h, h->Fx32, s.Fx) && upload_f32(h, h->Fy32, s.Fy);
    }
    if (!ok) return bail(SMM_ERR_OOM, "device allocation or upload failed");
    const size_t nang = (size_t)s.ne * s.nd * s.n, nphi = (size_t)s.ne * s.n;
    const bool pairs_only = o.sweep_solver == SMM_SOLVER_CACHED_INVERSE && o.sweep_precision == SMM_SWEEP_FP64;
    if (!pairs_only) {
        h->psi = h->alloc<double>(nang);
        if (!h->psi) return bail(SMM_ERR_OOM, "device allocation failed");
    }
    h->n_lagged = s.n_cycle_lagged;
    h->lagging = o.sweep_tiles > 1 || s.n_cycle_lagged > 0;
    if (!s.fmix.empty()) {
        if (!upload(h, h->fmix_id, s.fmix_id) || !upload(h, h->fmix, s.fmix) || !upload(h, h->fmix2, to_pairs(s.fmix)))
            return bail(SMM_ERR_OOM, "device allocation failed");
    }
    if (h->lagging && o.sweep_solver != SMM_SOLVER_CACHED_INVERSE) {
        h->psi_lag = h->alloc<double>(nang);
        if (!h->psi_lag) return bail(SMM_ERR_OOM, "device allocation failed");
    }
    if (h->fp32) {
        h->dpsi = h->alloc<float>(nang);
        h->res = h->alloc<float>(nang);
        if (!h->dpsi || !h->res) return bail(SMM_ERR_OOM, "device allocation failed");
    }
    h->gate = h->alloc<unsigned>(1);
    if (!h->gate) return bail(SMM_ERR_OOM, "device allocation failed");
    h->done = h->alloc<unsigned>((size_t)s.ne * s.nd);
    h->ticket = h->alloc<unsigned>(4);
    h->err = h->alloc<int>(4);
    h->mom = h->alloc<double>(6 * nphi);
    h->beta = h->alloc<double>((size_t)s.nb * s.nfq);
    h->trace = h->alloc<double>((size_t)s.ne * 4 * s.nfq * 3);
    h->rhs = h->alloc<double>(nphi);
    h->r = h->alloc<double>(nphi);
    h->z = h->alloc<double>(nphi);
    h->pv = h->alloc<double>(nphi);
    h->qv = h->alloc<double>(nphi);
    h->p2 = h->alloc<float2>(nphi);
    h->phi_prev = h->alloc<double>(nphi);
    h->phi_old = h->alloc<double>(nphi);
    h->phi_io = h->alloc<double>(nphi);
    const int epb = smm::cg_threads_per_block(s.n) / s.n;
    h->cg_nblk = (s.ne + epb - 1) / epb;
    h->cg_nvblk = std::max(1, std::min(2 * h->sms, (int)((nphi + 255) / 256)));
    // partial sums: [4][max(element blocks, continuous-node blocks)] then [3][vector blocks]
    h->cg_pmax = std::max(h->cg_nblk, std::max(1, (s.nglob + 255) / 256));
    h->part = h->alloc<double>(4 * (size_t)h->cg_pmax + 3 * (size_t)h->cg_nvblk);
    h->scal = h->alloc<double>(8);
    h->ctl = h->alloc<int>(8);
    h->dpart = h->alloc<double>(2 * 256);
    h->dout = h->alloc<double>(2);
    h->nonfinite = h->alloc<int>(1);
    if (!h->done || !h->ticket || !h->err || !h->mom || !h->beta || !h->trace || !h->rhs || !h->r || !h->z ||
        !h->pv || !h->qv || !h->p2 || !h->phi_prev || !h->phi_io || !h->part || !h->scal || !h->ctl || !h->dpart || !h->dout || !h->nonfinite)
        return bail(SMM_ERR_OOM, "device allocation failed");
    if ((h->psi && cudaMemsetAsync(h->psi, 0, nang * sizeof(double), h->stream) != cudaSuccess) ||
        cudaMemsetAsync(h->done, 0, (size_t)s.ne * s.nd * sizeof(unsigned), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->err, 0, 4 * sizeof(int), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->mom, 0, 6 * nphi * sizeof(double), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->beta, 0, (size_t)std::max(1, s.nb * s.nfq) * sizeof(double), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->ctl, 0, 8 * sizeof(int), h->stream) != cudaSuccess)
        return bail(SMM_ERR_CUDA, "cudaMemsetAsync failed");
    if (h->fp32 && cudaMemsetAsync(h->dpsi, 0, nang * sizeof(float), h->stream) != cudaSuccess)
        return bail(SMM_ERR_CUDA, "cudaMemsetAsync failed");
    if (cudaMallocHost(&h->h_scal, 32 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&h->h_int, 8 * sizeof(int)) != cudaSuccess)
        return bail(SMM_ERR_OOM, "pinned allocation failed");
    for (auto& e : h->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(SMM_ERR_CUDA, "cudaEventCreate failed");
    const bool cgm = o.moment_discretization == SMM_MOMENT_CG;
    if (o.precond == SMM_PRECOND_MULTIGRID || cgm) {
        const int nc = (s.m + 1) * (s.m + 1);
        std::vector<int> corners((size_t)s.ne * 4);
        const int cidx[4] = {0, s.m, s.m * (s.m + 1), s.m * (s.m + 1) + s.m};
        for (int e = 0; e < s.ne; ++e)
            for (int c = 0; c < 4; ++c) corners[(size_t)e * 4 + c] = mesh->elem_nodes[(size_t)e * nc + cidx[c]];
        std::vector<int> nbr(s.nbr.begin(), s.nbr.end());
        smm::MGHierarchy H;
        std::string merr;
        // the continuous system's hierarchy starts from its element blocks (no
        // neighbour blocks, no level-0 block smoother)
        const bool okmg = cgm ? smm::build_multigrid(s.ne, s.n, s.Kcg, {}, {}, nbr, corners,
                                                     smm::gauss_lobatto01(s.p1).x, H, merr)
                              : smm::build_multigrid(s.ne, s.n, s.Adiag, s.Aoff, s.Pinv, nbr, corners,
                                                     smm::gauss_lobatto01(s.p1).x, H, merr);
        if (!okmg) return bail(SMM_ERR_MESH, merr);
        if ((int)H.lv.size() - 1 > 11) return bail(SMM_ERR_MESH, "multigrid: too many levels");
        smm::MGPlan& P = h->mg;
        P.enabled = true;
        P.ne = s.ne; P.n = s.n; P.nu0 = o.mg_smooth_steps; P.omega0 = H.omega0;
        P.chebyshev = o.mg_smoother == SMM_SMOOTHER_CHEBYSHEV;
        if (!cgm) {
            float *c32 = nullptr, *pi32 = nullptr, *wd32 = nullptr;
            ok &= upload_f32(h, c32, transpose_blocks(s.Cface, 2 * s.p1));
            ok &= upload_f32(h, pi32, transpose_blocks(s.Pinv, s.n));
            // the level-0 residual is needed only as its element-corner sums w4^T (b - A x), so the
            // diagonal blocks enter as W = w4^T A_d, [element][node][corner]
            {
                const int n = s.n;
                std::vector<double> wt((size_t)s.ne * n * 4, 0.0);
#pragma omp parallel for schedule(static)
                for (int e = 0; e < s.ne; ++e)
                    for (int j = 0; j < n; ++j)
                        for (int c = 0; c < 4; ++c) {
                            double acc = 0.0;
                            for (int i = 0; i < n; ++i)
                                acc += H.w4[(size_t)i * 4 + c] * s.Adiag[((size_t)e * n + i) * n + j];
                            wt[((size_t)e * n + j) * 4 + c] = acc;
                        }
                ok &= upload_f32(h, wd32, wt);
            }
            P.A.AdT = nullptr; P.A.CT = c32; P.PinvT = pi32; P.WdT = wd32;
            P.A.nbr = h->nbr; P.A.nface = h->nbr_face;
            for (int k = 0; k < s.p1; ++k) P.A.wd[k] = (float)s.wd[k];
        }
        if (!cgm) {
            P.x0 = h->alloc<float>(nphi); P.x0b = h->alloc<float>(nphi); P.res0 = h->alloc<float>(nphi);
            ok &= P.x0 && P.x0b && P.res0;
        }
        P.nvert = H.nvert;
        int *vid = nullptr, *vinc = nullptr;
        float* w4 = nullptr;
        {
            // vertex incidences as k-major ELL with -1 padding
            int vw = 0;
            for (int v = 0; v < H.nvert; ++v) vw = std::max(vw, H.vrp[v + 1] - H.vrp[v]);
            std::vector<int> ell((size_t)vw * H.nvert, -1);
            for (int v = 0; v < H.nvert; ++v)
                for (int k = H.vrp[v]; k < H.vrp[v + 1]; ++k) ell[(size_t)(k - H.vrp[v]) * H.nvert + v] = H.vinc[k];
            ok &= upload(h, vinc, ell);
            P.vw = vw;
        }
        ok &= upload(h, vid, H.vid) && upload_f32(h, w4, H.w4);
        P.vid = vid; P.vinc = vinc; P.w4 = w4;
        P.nlev = (int)H.lv.size() - 1;
        P.coarse_ctas = smm::mg_coarse_cluster_size();
        for (int l = 1; l <= P.nlev; ++l) {
            const smm::MGLevel& L = H.lv[l];
            smm::MGLevelDev& D = P.lv[l];
            D.n = L.A.nrow;
            D.omega = (float)L.omega;
            D.b = h->alloc<float>(D.n); D.x = h->alloc<float>(D.n); D.r = h->alloc<float>(D.n);
            D.t = h->alloc<float>(D.n);
            ok &= D.b && D.x && D.r && D.t;
            if (l < P.nlev) {
                std::vector<double> asv(L.A.v.size());
                for (int i = 0; i < L.A.nrow; ++i)
                    for (int k = L.A.rp[i]; k < L.A.rp[i + 1]; ++k)
                        asv[k] = L.A.v[k] * L.omega * L.dinv[L.A.ci[k]];
                std::vector<int> ci;
                std::vector<float> v, vs;
                int *aci, *pci, *rci;
                float *av, *asd, *dv, *pv, *rv;
                to_ell(L.A, asv, D.aw, ci, vs);
                to_ell(L.A, L.A.v, D.aw, ci, v);
                ok &= upload(h, aci, ci) && upload(h, av, v) && upload(h, asd, vs) && upload_f32(h, dv, L.dinv);
                to_ell(L.P, L.P.v, D.pw, ci, v);
                ok &= upload(h, pci, ci) && upload(h, pv, v);
                to_ell(L.R, L.R.v, D.rw, ci, v);
                ok &= upload(h, rci, ci) && upload(h, rv, v);
                D.Aci = aci; D.Av = av; D.Asv = asd; D.dinv = dv; D.Pci = pci; D.Pv = pv; D.Rci = rci; D.Rv = rv;
            }
        }
        float* cinv = nullptr;
        ok &= upload_f32(h, cinv, H.coarse_inv);
        P.cinv = cinv;
        // the coarse levels' read-only data in 32 KB chunks, prefetched into L2
        // by the level-0 residual kernel just before the coarse cycle reads it
        // (each span rounded up to 16 bytes stays inside its allocation's slack)
        {
            std::vector<smm::L2Chunk> pf;
            auto span = [&pf](const void* p, size_t bytes) {
                constexpr size_t kChunk = 32768;
                const size_t rb = (bytes + 15) & ~(size_t)15;
                for (size_t o = 0; p && o < rb; o += kChunk)
                    pf.push_back(smm::L2Chunk{(const char*)p + o, (unsigned)std::min(kChunk, rb - o), 0u});
            };
            span(P.vinc, (size_t)P.vw * H.nvert * sizeof(int));
            for (int l = 1; l < P.nlev; ++l) {
                const smm::MGLevel& L = H.lv[l];
                const smm::MGLevelDev& D = P.lv[l];
                const size_t a = (size_t)D.aw * L.A.nrow, pe = (size_t)D.pw * L.P.nrow, re = (size_t)D.rw * L.R.nrow;
                span(D.Aci, a * sizeof(int));
                span(D.Av, a * sizeof(float));
                span(D.Asv, a * sizeof(float));
                span(D.dinv, L.dinv.size() * sizeof(float));
                span(D.Pci, pe * sizeof(int));
                span(D.Pv, pe * sizeof(float));
                span(D.Rci, re * sizeof(int));
                span(D.Rv, re * sizeof(float));
            }
            span(P.cinv, H.coarse_inv.size() * sizeof(float));
            smm::L2Chunk* pfd = nullptr;
            ok &= upload(h, pfd, pf);
            P.coarse_pf = pfd;
            P.coarse_npf = (int)pf.size();
        }
        ok &= cudaStreamSynchronize(h->stream) == cudaSuccess;
        if (!ok) return bail(SMM_ERR_OOM, "multigrid upload failed");
        h->rold = h->alloc<double>(nphi);
        h->xcg = h->alloc<double>(nphi);
        if (!h->rold || !h->xcg) return bail(SMM_ERR_OOM, "device allocation failed");
        if (cgm) {
            smm_status cst = setup_cg_moment_system(h, s);
            if (cst != SMM_OK) {
                delete h;
                return cst;
            }
        }
        // capture one flexible-CG iteration (spmv, update, V-cycle, dots, direction) as a graph
        if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
            return bail(SMM_ERR_CUDA, "cudaStreamCreate failed");
        smm::CGArgs ca = cgm ? cgc_args(h) : cg_args(h, h->xcg);
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bail(SMM_ERR_CUDA, "cudaStreamBeginCapture failed");
        h->graph_kernels = cgm ? smm::cgc_iteration(ca, h->cgc, h->mg, h->cap)
                               : smm::cgx_iterations(ca, 1, h->mg, h->cap);
        if (cudaStreamEndCapture(h->cap, &g) != cudaSuccess || !g)
            return bail(SMM_ERR_CUDA, "CG iteration capture failed");
        const cudaError_t ie = cudaGraphInstantiate(&h->cg_graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return bail(SMM_ERR_CUDA, "CG graph instantiation failed");
        // the whole CG loop as one graph: a while node whose body is one
        // iteration followed by the loop-control kernel, so a solve needs no
        // host round trip between iterations; without it (option off, or a
        // runtime that cannot build it) the solve launches the one-iteration
        // graph in chunks
        if (o.cg_device_loop) {
            cudaGraph_t G = nullptr;
            cudaGraphConditionalHandle hc = 0;
            bool okg = cudaGraphCreate(&G, 0) == cudaSuccess &&
                       cudaGraphConditionalHandleCreate(&hc, G, 1u, cudaGraphCondAssignDefault) == cudaSuccess;
            cudaGraphNodeParams np{};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = hc;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node = nullptr;
            okg = okg && cudaGraphAddNode(&node, G, nullptr, nullptr, 0, &np) == cudaSuccess;
            okg = okg && cudaStreamBeginCaptureToGraph(h->cap, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (okg) {
                if (cgm)
                    smm::cgc_iteration(ca, h->cgc, h->mg, h->cap);
                else
                    smm::cgx_iterations(ca, 1, h->mg, h->cap);
                smm::launch_cg_loop_control(hc, h->ctl, h->cap);
                cudaGraph_t body = nullptr;
                okg = cudaStreamEndCapture(h->cap, &body) == cudaSuccess;
            }
            okg = okg && cudaGraphInstantiate(&h->cg_loop, G, 0) == cudaSuccess;
            if (G) cudaGraphDestroy(G);
            if (!okg) {
                if (h->cg_loop) cudaGraphExecDestroy(h->cg_loop);
                h->cg_loop = nullptr;
                cudaGetLastError();
            }
        }
    }
    if (o.anderson_depth > 0) {
        for (int k = 0; k <= o.anderson_depth; ++k) {
            h->aaG.push_back(h->alloc<double>(nphi));
            h->aaF.push_back(h->alloc<double>(nphi));
            if (!h->aaG.back() || !h->aaF.back()) return bail(SMM_ERR_OOM, "device allocation failed");
        }
        h->aa_part = h->alloc<double>(21 * 256);
        h->aa_out = h->alloc<double>(32);
        if (!h->aa_part || !h->aa_out) return bail(SMM_ERR_OOM, "device allocation failed");
    }
    h->cached = o.sweep_solver == SMM_SOLVER_CACHED_INVERSE;
    if (h->cached) {
        const size_t ninv = (size_t)s.ne * s.nd * s.n * s.n;
        h->msrc2 = h->alloc<float2>(nphi);
        if (!h->msrc2) return bail(SMM_ERR_OOM, "device allocation failed");
        if (h->src_angular) {
            h->mq2 = h->alloc<float2>(nang);
            if (!h->mq2) return bail(SMM_ERR_OOM, "device allocation failed");
            smm::launch_mass_apply(s.ne, s.nd, s.n, h->M, h->src, h->mq2, h->stream);
        }
        if (!h->fp32) {
            bool okp = upload(h, h->ox2, to_pairs(s.quad.ox)) && upload(h, h->oy2, to_pairs(s.quad.oy)) &&
                       upload(h, h->Fx2, to_pairs(s.Fx)) && upload(h, h->Fy2, to_pairs(s.Fy));
            if (okp && !s.inflow.empty()) okp = upload(h, h->inflow2, to_pairs(s.inflow));
            {
                const int nd = s.nd;
                std::vector<double> wq((size_t)6 * nd);
                for (int d = 0; d < nd; ++d) {
                    const double w = s.quad.w[d], x = s.quad.ox[d], y = s.quad.oy[d];
                    wq[d] = w;
                    wq[nd + d] = w * x;
                    wq[2 * nd + d] = w * y;
                    wq[3 * nd + d] = w * x * x;
                    wq[4 * nd + d] = w * x * y;
                    wq[5 * nd + d] = w * y * y;
                }
                okp = okp && upload(h, h->wq2, to_pairs(wq));
            }
            h->psi2 = h->alloc<float2>(nang);
            if (!okp || !h->psi2) return bail(SMM_ERR_OOM, "device allocation failed");
            if (cudaMemsetAsync(h->psi2, 0, nang * sizeof(float2), h->stream) != cudaSuccess)
                return bail(SMM_ERR_CUDA, "cudaMemsetAsync failed");
            if (h->lagging) {
                h->psi2_lag = h->alloc<float2>(nang);
                if (!h->psi2_lag) return bail(SMM_ERR_OOM, "device allocation failed");
            }
        }
        if (h->fp32) {
            h->ainv32 = h->alloc<float>(ninv);
            if (!h->ainv32) return bail(SMM_ERR_OOM, "no device memory for the cached local inverses (use SMM_SOLVER_LU)");
            smm::SweepArgs<float> a{};
            a.ne = s.ne; a.nd = s.nd; a.ntask = h->ntask; a.ox = h->ox; a.oy = h->oy; a.sigma_t = h->sigma_t;
            a.M = h->M32; a.Gx = h->Gx32; a.Gy = h->Gy32; a.Fx = h->Fx32; a.Fy = h->Fy32; a.fdir = h->fdir;
            a.fmix_id = h->fmix_id; a.fmix = h->fmix;
            smm::launch_invert<float>(s.p, a, h->ainv32, h->stream);
        } else {
            h->ainv_df = h->alloc<float2>(ninv);
            if (!h->ainv_df) return bail(SMM_ERR_OOM, "no device memory for the cached local inverses (use SMM_SOLVER_LU)");
            smm::SweepArgs<double> a{};
            a.ne = s.ne; a.nd = s.nd; a.ntask = h->ntask; a.ox = h->ox; a.oy = h->oy; a.sigma_t = h->sigma_t;
            a.M = h->M; a.Gx = h->Gx; a.Gy = h->Gy; a.Fx = h->Fx; a.Fy = h->Fy; a.fdir = h->fdir;
            a.fmix_id = h->fmix_id; a.fmix = h->fmix;
            smm::launch_invert_df(s.p, a, h->ainv_df, h->stream);
        }
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess)
            return bail(SMM_ERR_CUDA, "local inverse construction failed");
    }
    const int bps = smm::sweep_blocks_per_sm(s.p, h->fp32 ? smm::SWEEP_RESIDUAL : smm::SWEEP_SOURCE, h->fp32, h->cached);
    // cooperative launch: never more blocks than can be co-resident
    const long long want = ((long long)h->ntask + 7) / 8;
    h->sweep_grid = (int)std::max(1LL, std::min<long long>((long long)h->sms * bps, want));
    {
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
        if (!coop) return bail(SMM_ERR_CUDA, "device does not support cooperative launches");
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(SMM_ERR_CUDA, "setup upload failed");
    *out = h;
    return SMM_OK;
}

smm_status smm_get_info(smm_handle h, smm_info* info) {
    if (!h || !info) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    info->n_elem = h->ne; info->p = h->p; info->m = h->m; info->n_dof_elem = h->n; info->n_ord = h->nd;
    info->n_bface = h->nb; info->n_fq = h->nfq; info->n_levels = h->nlevels;
    info->n_angular = (int64_t)h->ne * h->n * h->nd;
    info->n_lagged = h->n_lagged;
    return SMM_OK;
}

smm_status smm_destroy(smm_handle h) {
    if (!h) return SMM_OK;
    if (h->stream || true) cudaStreamSynchronize(h->stream);
    delete h;
    return SMM_OK;
}

}  // extern "C"

namespace {

// enqueue one sweep + moments + beta; no host synchronization
// Bump the flag epoch, launch the per-sweep pre-kernels (FP64: source
// products for cached inverses; FP32-refined: the FP64 transport residual) and
// fill the sweep arguments.  Shared by the single and the batched sweep.
template <typename T>
smm_status prepare_sweep(smm_handle h, const double* phi, smm::SweepArgs<T>& a) {
    h->epoch += 1;
    if (h->epoch == 0) {  // wrap: reset flags
        SMM_CUDA(cudaMemsetAsync(h->done, 0, (size_t)h->ne * h->nd * sizeof(unsigned), h->stream));
        h->epoch = 1;
    }
    a = smm::SweepArgs<T>{};
    a.ne = h->ne; a.nd = h->nd; a.ntask = h->ntask; a.p = h->p; a.tasks = h->tasks; a.ox = h->ox; a.oy = h->oy;
    a.sigma_t = h->sigma_t; a.sigma_s = h->sigma_s;
    a.fdir = h->fdir; a.nbr = h->nbr; a.nbr_face = h->nbr_face; a.nbr_flip = h->nbr_flip; a.bface_id = h->bface_id;
    a.fmix_id = h->fmix_id; a.fmix = h->fmix; a.fmix2 = h->fmix2;
    a.done = h->done; a.epoch = h->epoch; a.ticket = h->ticket; a.err = h->err;
    a.timeout_ns = (long long)(h->opt.spin_timeout_s * 1e9);
    SMM_CUDA(cudaMemsetAsync(h->gate, 0, sizeof(unsigned), h->stream));
    a.gate = h->gate; a.w = h->w; a.wq2 = h->wq2; a.mpsi = h->psi; a.mom = h->mom;
    a.beta = h->nb > 0 ? h->beta : nullptr; a.nfq = h->nfq; a.L1 = h->L1; a.nhat = h->b_nhat; a.eb0 = h->b_eb0;
    if constexpr (std::is_same<T, double>::value) {
        a.M = h->M; a.Gx = h->Gx; a.Gy = h->Gy; a.Fx = h->Fx; a.Fy = h->Fy;
        a.phi = phi; a.src = h->src; a.src_angular = h->src_angular; a.inflow = h->has_inflow ? h->inflow : nullptr;
        a.fixup = h->opt.negative_flux_fixup ? 1 : 0;
        a.colM = h->colM; a.colGx = h->colGx; a.colGy = h->colGy; a.colFx = h->colFx; a.colFy = h->colFy;
        a.rhs = nullptr; a.psi = h->psi; a.psi_acc = nullptr;
        if (h->lagging) {
            // lagged inflow (between tiles, or closing a cycle): the previous sweep's psi
            const size_t nang = (size_t)h->ne * h->nd * h->n;
            if (h->cached) {
                SMM_CUDA(cudaMemcpyAsync(h->psi2_lag, h->psi2, nang * sizeof(float2), cudaMemcpyDeviceToDevice,
                                         h->stream));
            } else {
                SMM_CUDA(cudaMemcpyAsync(h->psi_lag, h->psi, nang * sizeof(double), cudaMemcpyDeviceToDevice,
                                         h->stream));
            }
            a.psi_lag = h->psi_lag;
            a.psi2_lag = h->psi2_lag;
        }
        if (h->cached) {
            smm::launch_source(h->ne, h->n, h->M, h->sigma_s, phi, h->src_angular ? nullptr : h->src, h->msrc2,
                               h->stream);
            h->launches += 1;
            a.ainv_df = h->ainv_df; a.msrc2 = h->msrc2; a.mq2 = h->mq2;
            a.ox2 = h->ox2; a.oy2 = h->oy2; a.Fx2 = h->Fx2; a.Fy2 = h->Fy2;
            a.inflow2 = h->has_inflow ? h->inflow2 : nullptr; a.psi2 = h->psi2;
        }
    } else {
        smm::ResidualArgs r{};
        r.ne = h->ne; r.nd = h->nd; r.ntask = h->ntask; r.ox = h->ox; r.oy = h->oy; r.sigma_t = h->sigma_t;
        r.sigma_s = h->sigma_s; r.M = h->M; r.Gx = h->Gx; r.Gy = h->Gy; r.Fx = h->Fx; r.Fy = h->Fy; r.fdir = h->fdir;
        r.nbr = h->nbr; r.nbr_face = h->nbr_face; r.nbr_flip = h->nbr_flip; r.bface_id = h->bface_id; r.phi = phi;
        r.src = h->src; r.src_angular = h->src_angular; r.inflow = h->has_inflow ? h->inflow : nullptr; r.psi = h->psi;
        r.rhs = h->res;
        smm::launch_residual(h->p, r, h->stream);
        h->launches += 1;
        a.M = h->M32; a.Gx = h->Gx32; a.Gy = h->Gy32; a.Fx = h->Fx32; a.Fy = h->Fy32;
        a.phi = nullptr; a.src = nullptr; a.src_angular = 0; a.inflow = nullptr; a.rhs = h->res;
        a.psi = h->dpsi; a.psi_acc = h->psi;
        a.ainv = h->cached ? h->ainv32 : nullptr;
    }
    SMM_CUDA(cudaGetLastError());
    return SMM_OK;
}

// enqueue one sweep (pre-kernels + the wavefront kernel); no host synchronization
smm_status enqueue_sweep(smm_handle h, const double* phi) {
    if (!h->fp32) {
        smm::SweepArgs<double> a;
        smm_status st = prepare_sweep(h, phi, a);
        if (st != SMM_OK) return st;
        SMM_CUDA(cudaEventRecord(h->ev[5], h->stream));
        smm::launch_sweep<double>(h->p, smm::SWEEP_SOURCE, a, h->sweep_grid, h->stream);
    } else {
        smm::SweepArgs<float> a;
        smm_status st = prepare_sweep(h, phi, a);
        if (st != SMM_OK) return st;
        SMM_CUDA(cudaEventRecord(h->ev[5], h->stream));
        smm::launch_sweep<float>(h->p, smm::SWEEP_RESIDUAL, a, h->sweep_grid, h->stream);
    }
    h->launches += 1;
    SMM_CUDA(cudaGetLastError());
    return SMM_OK;
}

smm_status enqueue_rhs(smm_handle h) {
    smm::launch_rhs(h->ne, h->n, h->p, h->nfq, h->mom, h->beta, h->bfixed, h->Kxx, h->Ks, h->Kyy, h->Dfx, h->Dfy,
                    h->DfxT, h->DfyT, h->nds,
                    h->L1, h->sigma_t, h->nbr, h->nbr_face, h->nbr_flip, h->bface_id, h->b_ds, h->trace, h->rhs,
                    h->stream);
    h->launches += 2;
    SMM_CUDA(cudaGetLastError());
    return SMM_OK;
}

// Arguments of the flexible CG on the continuous system (nglob unknowns)
smm::CGArgs cgc_args(smm_handle h) {
    smm::CGArgs a = cg_args(h, h->xc);
    a.nrow = h->cgc.nglob;
    a.nblk = h->cgc.nblk_node;
    a.b = h->bc;
    return a;
}

// Device data of the continuous moment system (Sec. 5.1): element blocks,
// node numbering and incidences, diagonal and point-Jacobi damping
smm_status setup_cg_moment_system(smm_handle h, const smm::Setup& s) {
    const int ne = s.ne, n = s.n, ng = s.nglob;
    const size_t nn = (size_t)n * n;
    smm::CGCPlan& c = h->cgc;
    c.ne = ne; c.n = n; c.nglob = ng; c.nu = h->opt.mg_smooth_steps;
    c.nblk_node = std::max(1, (ng + 255) / 256);
    // assembled diagonal and the largest eigenvalue of D^{-1} A by power iteration
    std::vector<double> diag(ng, 0.0);
    for (int e = 0; e < ne; ++e)
        for (int i = 0; i < n; ++i) diag[s.gid[(size_t)e * n + i]] += s.Kcg[(size_t)e * nn + (size_t)i * n + i];
    std::vector<double> dinv(ng), minv_d(ng);
    for (int g = 0; g < ng; ++g) {
        if (!(diag[g] > 0)) return fail(SMM_ERR_MESH, "continuous moment system: non-positive diagonal");
        dinv[g] = 1.0 / diag[g];
        minv_d[g] = 1.0 / (double)(s.grp[g + 1] - s.grp[g]);
    }
    {
        std::vector<double> x(ng), ye((size_t)ne * n), y(ng);
        for (int g = 0; g < ng; ++g) x[g] = 1.0 + 0.5 * std::sin(0.7 * (double)g + 0.3);
        double lam = 1.0;
        for (int it = 0; it < 30; ++it) {
#pragma omp parallel for schedule(static)
            for (int e = 0; e < ne; ++e)
                for (int i = 0; i < n; ++i) {
                    double acc = 0.0;
                    for (int j = 0; j < n; ++j) acc += s.Kcg[(size_t)e * nn + (size_t)i * n + j] * x[s.gid[(size_t)e * n + j]];
                    ye[(size_t)e * n + i] = acc;
                }
            double xy = 0.0, xdx = 0.0, nrm = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : xy, xdx)
            for (int g = 0; g < ng; ++g) {
                double acc = 0.0;
                for (int k = s.grp[g]; k < s.grp[g + 1]; ++k) acc += ye[s.ginc[k]];
                y[g] = acc;
                xy += x[g] * acc;
                xdx += x[g] * x[g] * diag[g];
            }
            lam = xy / xdx;
            for (int g = 0; g < ng; ++g) {
                y[g] *= dinv[g];
                nrm += y[g] * y[g];
            }
            nrm = std::sqrt(nrm);
            for (int g = 0; g < ng; ++g) x[g] = y[g] / nrm;
        }
        c.omega = (4.0 / 3.0) / (1.05 * lam);
    }
    bool ok = true;
    double *KT = nullptr, *dv = nullptr;
    int *gid = nullptr, *grp = nullptr, *ginc = nullptr, *gown = nullptr;
    float* minv = nullptr;
    ok &= upload(h, KT, transpose_blocks(s.Kcg, n)) && upload(h, dv, dinv);
    ok &= upload(h, gid, s.gid) && upload(h, grp, s.grp) && upload(h, ginc, s.ginc) && upload(h, gown, s.gown);
    ok &= upload_f32(h, minv, minv_d);
    c.KT = KT; c.dinv = dv; c.gid = gid; c.grp = grp; c.ginc = ginc; c.gown = gown; c.minv = minv;
    c.ye = h->alloc<double>((size_t)ne * n);
    c.xa = h->alloc<double>(ng);
    c.xb = h->alloc<double>(ng);
    c.res = h->alloc<double>(ng);
    c.cres = h->alloc<float>((size_t)ne * 4);
    h->bc = h->alloc<double>(ng);
    h->xc = h->alloc<double>(ng);
    ok &= c.ye && c.xa && c.xb && c.res && c.cres && h->bc && h->xc;
    ok &= cudaStreamSynchronize(h->stream) == cudaSuccess;
    if (!ok) return fail(SMM_ERR_OOM, "continuous moment system: device allocation or upload failed");
    c.enabled = true;
    return SMM_OK;
}

smm::CGArgs cg_args(smm_handle h, double* x) {
    smm::CGArgs a{};
    a.ne = h->ne; a.n = h->n; a.nrow = h->ne * h->n; a.nblk = h->cg_nblk;
    a.nvblk = h->cg_nvblk; a.pvec = h->part + 4 * (size_t)h->cg_pmax;
    a.A.AdT = h->AdT; a.A.CT = h->CT; a.A.nbr = h->nbr; a.A.nface = h->nbr_face;
    for (int k = 0; k < 5; ++k) a.A.wd[k] = h->wd[k];
    a.A2.AdT = h->AdT2; a.A2.CT = h->CT2; a.A2.nbr = h->nbr; a.A2.nface = h->nbr_face;
    for (int k = 0; k < 5; ++k) {
        const float hi = (float)h->wd[k];
        a.A2.wd[k] = make_float2(hi, (float)(h->wd[k] - (double)hi));
    }
    a.p2 = h->p2;
    a.PinvT = h->PinvT;
    a.x = x; a.r = h->r; a.z = h->z; a.p = h->pv; a.q = h->qv; a.rold = h->rold; a.b = h->rhs; a.part = h->part;
    a.scal = h->scal;
    a.ctl = h->ctl;
    return a;
}

smm_status check_device_error(smm_handle h) {
    SMM_CUDA(cudaMemcpyAsync(h->h_int, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    SMM_CUDA(cudaStreamSynchronize(h->stream));
    if (h->h_int[0] == smm::DEV_TIMEOUT) {
        cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
        return fail(SMM_ERR_DEVICE_TIMEOUT, "a sweep dependency wait exceeded spin_timeout_s");
    }
    return SMM_OK;
}

// CG from the guess in x to ||r||_2 <= tol ||b||_2; host reads the control word every `chunk` iterations
smm_status run_cg(smm_handle h, double* x, int* iters, double tol) {
    const bool cgm = h->cgc.enabled;
    const bool mg = h->mg.enabled;
    const size_t nphi = (size_t)h->ne * h->n;
    smm::CGArgs a = cgm ? cgc_args(h) : cg_args(h, mg ? h->xcg : x);
    SMM_CUDA(cudaMemsetAsync(h->ctl, 0, 8 * sizeof(int), h->stream));
    if (cgm) {
        // continuous system: b = P^T b_IP, initial guess from the DG iterate
        smm::cgc_gather(h->cgc, h->rhs, h->bc, h->stream);
        smm::cgc_pick(h->cgc, x, h->xc, h->stream);
        h->launches += 2 + smm::cgc_start(a, h->cgc, h->mg, tol, h->opt.max_cg, h->stream);
    } else if (mg) {
        SMM_CUDA(cudaMemcpyAsync(h->xcg, x, nphi * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        h->launches += smm::cgx_start(a, tol, h->opt.max_cg, h->mg, h->stream);
    } else {
        smm::cg_start(a, tol, h->opt.max_cg, h->stream);
        h->launches += 2;
    }
    SMM_CUDA(cudaGetLastError());
    if (mg && h->cg_loop) {
        SMM_CUDA(cudaGraphLaunch(h->cg_loop, h->stream));
        SMM_CUDA(cudaMemcpyAsync(h->h_int, h->ctl, 8 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        SMM_CUDA(cudaStreamSynchronize(h->stream));
        h->launches += (long long)h->h_int[5] * (h->graph_kernels + 1);
    }
    int chunk = mg ? 4 : 8;
    while (!(mg && h->cg_loop)) {
        SMM_CUDA(cudaMemcpyAsync(h->h_int, h->ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        SMM_CUDA(cudaStreamSynchronize(h->stream));
        if (h->h_int[0]) break;
        if (mg) {
            for (int k = 0; k < chunk; ++k) SMM_CUDA(cudaGraphLaunch(h->cg_graph, h->stream));
            h->launches += (long long)chunk * h->graph_kernels;
        } else {
            smm::cg_iterations(a, chunk, h->stream);
            h->launches += 3LL * chunk;
        }
        SMM_CUDA(cudaGetLastError());
        chunk = std::min(chunk * 2, mg ? 16 : 64);
    }
    if (cgm) {
        smm::cgc_expand(h->cgc, h->xc, x, h->stream);  // the DG nodal values P varphi
        h->launches += 1;
    } else if (mg) {
        SMM_CUDA(cudaMemcpyAsync(x, h->xcg, nphi * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    if (iters) *iters = h->h_int[1];
    if (h->h_int[3]) return fail(SMM_ERR_NONFINITE, "non-finite value in the moment solve");
    if (h->h_int[1] >= h->opt.max_cg) {
        // converged exactly at the cap is still convergence
        SMM_CUDA(cudaMemcpyAsync(h->h_scal, h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        SMM_CUDA(cudaStreamSynchronize(h->stream));
        if (!(h->h_scal[2] <= h->h_scal[4])) return fail(SMM_ERR_NOT_CONVERGED, "CG iteration limit reached");
    }
    return SMM_OK;
}

// Anderson acceleration of x = G(x) (depth m): with f_j = G(x_j) - x_j,
// x_{k+1} = G(x_k) - sum_j gamma_j (G_{k-j} - G_{k-j-1}) where gamma minimizes
// || f_k - sum_j gamma_j (f_{k-j} - f_{k-j-1}) ||_2 (normal equations from a
// Gram matrix reduced on the device).  phi holds G(x_k) on entry and
// h->phi_prev holds x_k; phi receives x_{k+1}.
smm_status anderson_step(smm_handle h, int k, double* phi) {
    const int m = h->opt.anderson_depth;
    const int slots = m + 1;
    const size_t nphi = (size_t)h->ne * h->n;
    const int cur = (k - 1) % slots;
    SMM_CUDA(cudaMemcpyAsync(h->aaG[cur], phi, nphi * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    smm::launch_axpby((int)nphi, 1.0, phi, -1.0, h->phi_prev, h->aaF[cur], h->stream);
    h->launches += 1;
    const int mk = std::min(m, k - 1);
    if (mk == 0) return SMM_OK;  // x_{k+1} = G(x_k), already in phi
    smm::VecSet vs{};
    vs.nv = mk + 1;
    for (int j = 0; j <= mk; ++j) vs.v[j] = h->aaF[(cur - j + slots) % slots];
    smm::launch_gram((int)nphi, vs, h->aa_part, h->aa_out, h->stream);
    h->launches += 2;
    SMM_CUDA(cudaMemcpyAsync(h->h_scal, h->aa_out, 21 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SMM_CUDA(cudaStreamSynchronize(h->stream));
    // R[a][b] = f_a . f_b for the vectors of vs (packed upper triangle, row-major)
    double R[6][6];
    {
        int t = 0;
        for (int x = 0; x < 6; ++x)
            for (int y = x; y < 6; ++y) {
                R[x][y] = R[y][x] = h->h_scal[t];
                ++t;
            }
    }
    // dF_i = vs[i] - vs[i+1]:  H_ij = dF_i . dF_j,  g_i = dF_i . f_k
    double H[5][6];
    for (int i = 0; i < mk; ++i) {
        for (int j = 0; j < mk; ++j) H[i][j] = R[i][j] - R[i][j + 1] - R[i + 1][j] + R[i + 1][j + 1];
        H[i][mk] = R[i][0] - R[i + 1][0];
    }
    double tr = 0.0;
    for (int i = 0; i < mk; ++i) tr += H[i][i];
    for (int i = 0; i < mk; ++i) H[i][i] += 1e-13 * tr;
    for (int c = 0; c < mk; ++c) {  // Gaussian elimination with partial pivoting
        int piv = c;
        for (int r = c + 1; r < mk; ++r)
            if (std::fabs(H[r][c]) > std::fabs(H[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j <= mk; ++j) std::swap(H[c][j], H[piv][j]);
        if (H[c][c] == 0.0) return SMM_OK;  // degenerate history: keep the plain update
        for (int r = c + 1; r < mk; ++r) {
            const double l = H[r][c] / H[c][c];
            for (int j = c; j <= mk; ++j) H[r][j] -= l * H[c][j];
        }
    }
    smm::MixArgs mx{};
    mx.m = mk;
    for (int i = mk - 1; i >= 0; --i) {
        double s = H[i][mk];
        for (int j = i + 1; j < mk; ++j) s -= H[i][j] * mx.gamma[j];
        mx.gamma[i] = s / H[i][i];
    }
    for (int j = 0; j <= mk; ++j) mx.G[j] = h->aaG[(cur - j + slots) % slots];
    smm::launch_anderson_mix((int)nphi, mx, phi, h->stream);
    h->launches += 1;
    SMM_CUDA(cudaGetLastError());
    return SMM_OK;
}

}  // namespace

extern "C" {

smm_status smm_sweep(smm_handle h, const double* phi_dev, double* phiT_out) {
    if (!h) return fail(SMM_ERR_INVALID_ARG, "NULL handle");
    smm_status st = enqueue_sweep(h, phi_dev);
    if (st != SMM_OK) return st;
    st = check_device_error(h);
    if (st != SMM_OK) return st;
    if (phiT_out) {
        // component 0 of the moments is phi_T = sum_d w_d psi_d (host or device destination)
        SMM_CUDA(cudaMemcpyAsync(phiT_out, h->mom, (size_t)h->ne * h->n * sizeof(double), cudaMemcpyDefault,
                                 h->stream));
        SMM_CUDA(cudaStreamSynchronize(h->stream));
    }
    return SMM_OK;
}

smm_status smm_moments(smm_handle h, double* moments_dev, double* beta_dev) {
    if (!h) return fail(SMM_ERR_INVALID_ARG, "NULL handle");
    const size_t nphi = (size_t)h->ne * h->n;
    if (moments_dev)
        SMM_CUDA(cudaMemcpyAsync(moments_dev, h->mom, 6 * nphi * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    if (beta_dev && h->nb)
        SMM_CUDA(cudaMemcpyAsync(beta_dev, h->beta, (size_t)h->nb * h->nfq * sizeof(double), cudaMemcpyDeviceToDevice,
                                 h->stream));
    SMM_CUDA(cudaStreamSynchronize(h->stream));
    return SMM_OK;
}

smm_status smm_set_moments(smm_handle h, const double* moments_dev, const double* beta_dev) {
    if (!h || !moments_dev) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    const size_t nphi = (size_t)h->ne * h->n;
    SMM_CUDA(cudaMemcpyAsync(h->mom, moments_dev, 6 * nphi * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    if (h->nb) {
        if (beta_dev)
            SMM_CUDA(cudaMemcpyAsync(h->beta, beta_dev, (size_t)h->nb * h->nfq * sizeof(double),
                                     cudaMemcpyDeviceToDevice, h->stream));
        else
            SMM_CUDA(cudaMemsetAsync(h->beta, 0, (size_t)h->nb * h->nfq * sizeof(double), h->stream));
    }
    SMM_CUDA(cudaStreamSynchronize(h->stream));
    return SMM_OK;
}

smm_status smm_get_psi(smm_handle h, double* psi_dev) {
    if (!h || !psi_dev) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    const size_t nang = (size_t)h->ne * h->nd * h->n;
    if (h->psi) {
        SMM_CUDA(cudaMemcpyAsync(psi_dev, h->psi, nang * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    } else {
        smm::launch_pairs_to_f64(nang, h->psi2, psi_dev, h->stream);  // hi + lo, the FP64 value of each pair
        h->launches += 1;
        SMM_CUDA(cudaGetLastError());
    }
    SMM_CUDA(cudaStreamSynchronize(h->stream));
    return SMM_OK;
}

smm_status smm_moment_solve(smm_handle h, double* phi_dev, int32_t* cg_iters) {
    if (!h || !phi_dev) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    smm_status st = enqueue_rhs(h);
    if (st != SMM_OK) return st;
    int it = 0;
    st = run_cg(h, phi_dev, &it, h->opt.tol_cg);
    if (cg_iters) *cg_iters = it;
    return st;
}

}  // extern "C"

namespace {

// true when p is memory the host addresses directly (pageable or pinned host memory)
bool is_host_pointer(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// the moment solve's tolerance in an outer step whose predecessor changed
// varphi by prev_rel (relative max-norm): options.cg_tol_adaptive
double inner_tol(smm_handle h, double prev_rel) {
    const double eta = h->opt.cg_tol_adaptive;
    return eta > 0 ? std::max(h->opt.tol_cg, eta * prev_rel) : h->opt.tol_cg;
}

// the moment solve's starting point: phi_dev holds varphi_k (also in
// phi_prev); with two earlier steps known it becomes varphi_k + rho (varphi_k
// - varphi_{k-1}), rho = d_{k-1} / d_{k-2} clamped to [0, 0.9]
smm_status extrapolate_start(smm_handle h, double* phi_dev) {
    if (!h->opt.cg_guess_extrapolate || h->opt.anderson_depth > 0 || !(h->dl2 > 0.0)) return SMM_OK;
    const double rho = std::min(0.9, std::max(0.0, h->dl1 / h->dl2));
    smm::launch_axpby(h->ne * h->n, 1.0 + rho, h->phi_prev, -rho, h->phi_old, phi_dev, h->stream);
    h->launches += 1;
    SMM_CUDA(cudaGetLastError());
    return SMM_OK;
}

// after an outer step whose input is in phi_prev and whose successive
// difference is diff: shift the extrapolation history
smm_status record_step(smm_handle h, double diff) {
    h->dl2 = h->dl1;
    h->dl1 = diff;
    SMM_CUDA(cudaMemcpyAsync(h->phi_old, h->phi_prev, (size_t)h->ne * h->n * sizeof(double),
                             cudaMemcpyDeviceToDevice, h->stream));
    return SMM_OK;
}

smm_status iterate_device(smm_handle h, double tol, int32_t relative, int32_t max_outer, double* phi_dev,
                          smm_stats* stats) {
    smm_stats local{};
    local.cg_min = 1 << 30;
    const long long launches0 = h->launches;
    const size_t nphi = (size_t)h->ne * h->n;
    smm_status result = SMM_ERR_NOT_CONVERGED;
    if (!h->opt.resume_history) {
        h->aa_k = 0;
        h->dl1 = h->dl2 = 0.0;
    }
    double prev_rel = 1.0;  // the previous step's relative difference (adaptive inner tolerance)
    for (int k = 1; k <= max_outer; ++k) {
        SMM_CUDA(cudaMemcpyAsync(h->phi_prev, phi_dev, nphi * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        SMM_CUDA(cudaEventRecord(h->ev[0], h->stream));
        smm_status st = enqueue_sweep(h, phi_dev);
        if (st != SMM_OK) return st;
        SMM_CUDA(cudaEventRecord(h->ev[1], h->stream));
        SMM_CUDA(cudaEventRecord(h->ev[2], h->stream));  // the moments are formed inside the sweep
        st = enqueue_rhs(h);
        if (st != SMM_OK) return st;
        SMM_CUDA(cudaEventRecord(h->ev[3], h->stream));
        int it = 0;
        st = extrapolate_start(h, phi_dev);
        if (st != SMM_OK) return st;
        st = run_cg(h, phi_dev, &it, inner_tol(h, prev_rel));
        if (st != SMM_OK && st != SMM_ERR_NOT_CONVERGED) return st;
        SMM_CUDA(cudaEventRecord(h->ev[4], h->stream));
        SMM_CUDA(cudaMemsetAsync(h->nonfinite, 0, sizeof(int), h->stream));
        smm::launch_diff((int)nphi, phi_dev, h->phi_prev, h->dpart, h->dout, h->nonfinite, h->stream);
        h->launches += 2;
        SMM_CUDA(cudaMemcpyAsync(h->h_scal, h->dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        SMM_CUDA(cudaMemcpyAsync(h->h_int + 4, h->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        SMM_CUDA(cudaMemcpyAsync(h->h_int + 5, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        SMM_CUDA(cudaStreamSynchronize(h->stream));
        if (h->h_int[5] == smm::DEV_TIMEOUT) {
            cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
            h->aa_k = 0;
            if (stats) *stats = local;
            return fail(SMM_ERR_DEVICE_TIMEOUT, "a sweep dependency wait exceeded spin_timeout_s");
        }
        float t01 = 0, t12 = 0, t23 = 0, t34 = 0, t05 = 0;
        cudaEventElapsedTime(&t05, h->ev[0], h->ev[5]);
        cudaEventElapsedTime(&t01, h->ev[5], h->ev[1]);
        cudaEventElapsedTime(&t12, h->ev[1], h->ev[2]);
        cudaEventElapsedTime(&t23, h->ev[2], h->ev[3]);
        cudaEventElapsedTime(&t34, h->ev[3], h->ev[4]);
        local.ms_residual += t05; local.ms_sweep += t01; local.ms_moments += t12; local.ms_rhs += t23; local.ms_solve += t34;
        local.outer_iterations = k;
        local.n_launches = h->launches - launches0;
        local.cg_total += it;
        local.cg_min = std::min(local.cg_min, it);
        local.cg_max = std::max(local.cg_max, it);
        const double diff = h->h_scal[0], mx = h->h_scal[1];
        local.last_diff = diff;
        local.last_rel_diff = mx > 0 ? diff / mx : diff;
        prev_rel = local.last_rel_diff;
        st = record_step(h, diff);
        if (st != SMM_OK) return st;
        if (h->h_int[4]) {
            h->aa_k = 0;
            if (stats) *stats = local;
            return fail(SMM_ERR_NONFINITE, "non-finite scalar flux");
        }
        if (k == 1 && h->opt.guess_check && diff > mx) {
            // max|G(x0) - x0| > max|G(x0) - 0|: the given guess is farther from its
            // own image than the zero vector is, so restart from zero with an
            // empty Anderson history (no step from x0 enters it)
            SMM_CUDA(cudaMemsetAsync(phi_dev, 0, nphi * sizeof(double), h->stream));
            local.guess_rejected = 1;
            h->aa_k = 0;
            h->dl1 = h->dl2 = 0.0;
            prev_rel = 1.0;
            continue;
        }
        const double crit = relative ? local.last_rel_diff : diff;
        if (crit < tol) {
            result = SMM_OK;
            break;
        }
        if (h->opt.anderson_depth > 0) {
            h->aa_k += 1;
            smm_status as = anderson_step(h, h->aa_k, phi_dev);
            if (as != SMM_OK) return as;
        }
    }
    if (local.cg_min == (1 << 30)) local.cg_min = 0;
    if (stats) *stats = local;
    if (result != SMM_OK) return fail(result, "outer iteration limit reached");
    return SMM_OK;
}

}  // namespace

extern "C" {

smm_status smm_iterate(smm_handle h, double tol, int32_t relative, int32_t max_outer, double* phi,
                       smm_stats* stats) {
    if (!h || !phi || !(tol > 0) || max_outer < 1) return fail(SMM_ERR_INVALID_ARG, "bad argument");
    if (!is_host_pointer(phi)) return iterate_device(h, tol, relative, max_outer, phi, stats);
    // host iterate: copy in, iterate on the handle's device copy, copy the last iterate back
    const size_t bytes = (size_t)h->ne * h->n * sizeof(double);
    SMM_CUDA(cudaMemcpyAsync(h->phi_io, phi, bytes, cudaMemcpyHostToDevice, h->stream));
    smm_status st = iterate_device(h, tol, relative, max_outer, h->phi_io, stats);
    if (st == SMM_ERR_CUDA) return st;
    const std::string msg = g_err;
    SMM_CUDA(cudaMemcpyAsync(phi, h->phi_io, bytes, cudaMemcpyDeviceToHost, h->stream));
    SMM_CUDA(cudaStreamSynchronize(h->stream));
    if (st != SMM_OK) g_err = msg;
    return st;
}

}  // extern "C"

namespace {

// Checkpoint layout: a header of 16 int64 words, then the handle's state
// arrays, each starting on a 256-byte boundary.
constexpr int64_t kStateMagic = 0x534d4d5354415445LL;  // "SMMSTATE"
constexpr int64_t kStateVersion = 2;

struct StateSection {
    void* dev;
    size_t bytes;
};

std::vector<StateSection> state_sections(smm_handle h) {
    const size_t nang = (size_t)h->ne * h->nd * h->n, nphi = (size_t)h->ne * h->n;
    std::vector<StateSection> v;
    if (h->psi) v.push_back({h->psi, nang * sizeof(double)});
    if (h->psi2) v.push_back({h->psi2, nang * sizeof(float2)});
    v.push_back({h->mom, 6 * nphi * sizeof(double)});
    v.push_back({h->beta, (size_t)h->nb * h->nfq * sizeof(double)});
    v.push_back({h->phi_prev, nphi * sizeof(double)});
    v.push_back({h->phi_old, nphi * sizeof(double)});
    for (size_t k = 0; k < h->aaG.size(); ++k) {
        v.push_back({h->aaG[k], nphi * sizeof(double)});
        v.push_back({h->aaF[k], nphi * sizeof(double)});
    }
    return v;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

int64_t state_bytes(smm_handle h) {
    size_t total = 256;  // header
    for (const auto& sec : state_sections(h)) total += round256(sec.bytes);
    return (int64_t)total;
}

void state_header(smm_handle h, int64_t* hdr) {
    for (int i = 0; i < 32; ++i) hdr[i] = 0;
    hdr[0] = kStateMagic;
    hdr[1] = kStateVersion;
    hdr[2] = h->ne; hdr[3] = h->n; hdr[4] = h->nd; hdr[5] = h->nb; hdr[6] = h->nfq;
    hdr[7] = (h->psi2 ? 1 : 0) | (h->fp32 ? 2 : 0);
    hdr[8] = h->opt.anderson_depth;
    hdr[9] = h->aa_k;
    hdr[10] = state_bytes(h);
    std::memcpy(&hdr[11], &h->dl1, sizeof(double));  // the extrapolation history's differences
    std::memcpy(&hdr[12], &h->dl2, sizeof(double));
}

}  // namespace

extern "C" {

smm_status smm_set_spin_timeout(smm_handle h, double seconds) {
    if (!h || !(seconds > 0)) return fail(SMM_ERR_INVALID_ARG, "bad argument");
    h->opt.spin_timeout_s = seconds;
    return SMM_OK;
}

smm_status smm_state_size(smm_handle h, int64_t* bytes) {
    if (!h || !bytes) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    *bytes = state_bytes(h);
    return SMM_OK;
}

smm_status smm_get_state(smm_handle h, void* buf, int64_t bytes) {
    if (!h || !buf) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    if (bytes < state_bytes(h)) return fail(SMM_ERR_INVALID_ARG, "state buffer smaller than smm_state_size()");
    int64_t* hdr = reinterpret_cast<int64_t*>(h->h_scal);  // 32 pinned words
    state_header(h, hdr);
    char* out = static_cast<char*>(buf);
    SMM_CUDA(cudaMemcpyAsync(out, hdr, 256, cudaMemcpyDefault, h->stream));
    size_t off = 256;
    for (const auto& sec : state_sections(h)) {
        if (sec.bytes) SMM_CUDA(cudaMemcpyAsync(out + off, sec.dev, sec.bytes, cudaMemcpyDefault, h->stream));
        off += round256(sec.bytes);
    }
    SMM_CUDA(cudaStreamSynchronize(h->stream));
    return SMM_OK;
}

smm_status smm_set_state(smm_handle h, const void* buf, int64_t bytes) {
    if (!h || !buf) return fail(SMM_ERR_INVALID_ARG, "NULL argument");
    if (bytes < 256) return fail(SMM_ERR_INVALID_ARG, "state buffer too small");
    int64_t* hdr = reinterpret_cast<int64_t*>(h->h_scal);
    const char* in = static_cast<const char*>(buf);
    SMM_CUDA(cudaMemcpyAsync(hdr, in, 256, cudaMemcpyDefault, h->stream));
    SMM_CUDA(cudaStreamSynchronize(h->stream));
    int64_t want[32];
    state_header(h, want);
    if (hdr[0] != kStateMagic || hdr[1] != kStateVersion) return fail(SMM_ERR_INVALID_ARG, "not an smm state");
    for (int i = 2; i <= 8; ++i)
        if (hdr[i] != want[i]) return fail(SMM_ERR_INVALID_ARG, "state was saved from a handle of another shape or mode");
    if (hdr[10] != want[10] || bytes < want[10]) return fail(SMM_ERR_INVALID_ARG, "state size mismatch");
    if (hdr[9] < 0) return fail(SMM_ERR_INVALID_ARG, "bad Anderson history length");
    const int aa_k = (int)hdr[9];
    size_t off = 256;
    for (const auto& sec : state_sections(h)) {
        if (sec.bytes) SMM_CUDA(cudaMemcpyAsync(sec.dev, in + off, sec.bytes, cudaMemcpyDefault, h->stream));
        off += round256(sec.bytes);
    }
    SMM_CUDA(cudaStreamSynchronize(h->stream));
    h->aa_k = aa_k;
    std::memcpy(&h->dl1, &hdr[11], sizeof(double));
    std::memcpy(&h->dl2, &hdr[12], sizeof(double));
    return SMM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched sweeps: many problems (uneven mesh size, order p and S_N) in one
// cooperative launch over a merged, level-sorted (problem, task) list.
// ---------------------------------------------------------------------------
struct smm_batch_ctx {
    std::vector<smm_handle> hs;
    bool fp32 = false, cached = false;
    cudaStream_t stream = nullptr;
    int ntask = 0, nelem = 0, grid = 1, block = 256, sms = 1;
    double tuned_ms = 0.0;
    int2* tasks = nullptr;
    int2* elems = nullptr;          // (problem, element) of every element of every problem
    bool ext = false;               // some problem uses the fixup, tiles or lagged / mixed faces
    int pmax = 1;                   // the largest order p of the batch
    void* args_dev = nullptr;
    void* args_host = nullptr;  // pinned
    size_t args_bytes = 0;
    int* err = nullptr;
    unsigned* gate = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~smm_batch_ctx() {
        if (tasks) cudaFree(tasks);
        if (elems) cudaFree(elems);
        if (args_dev) cudaFree(args_dev);
        if (args_host) cudaFreeHost(args_host);
        if (err) cudaFree(err);
        if (gate) cudaFree(gate);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

template <typename T>
smm_status batch_enqueue(smm_batch b, const double* const* phis) {
    auto* host = static_cast<smm::SweepArgs<T>*>(b->args_host);
    SMM_CUDA(cudaMemsetAsync(b->gate, 0, sizeof(unsigned), b->stream));
    for (size_t i = 0; i < b->hs.size(); ++i) {
        smm_status st = prepare_sweep<T>(b->hs[i], phis ? phis[i] : nullptr, host[i]);
        if (st != SMM_OK) return st;
        host[i].err = b->err;
        host[i].gate = b->gate;  // one gate for the whole launch
    }
    SMM_CUDA(cudaMemcpyAsync(b->args_dev, b->args_host, b->args_bytes, cudaMemcpyHostToDevice, b->stream));
    SMM_CUDA(smm::launch_batch_sweep<T>(b->fp32 ? smm::SWEEP_RESIDUAL : smm::SWEEP_SOURCE, b->cached, b->ext, b->pmax,
                                         static_cast<const smm::SweepArgs<T>*>(b->args_dev), b->tasks, b->ntask,
                                         b->elems, b->nelem, b->grid, b->block, b->stream));
    b->hs[0]->launches += 1;
    return SMM_OK;
}

smm_status batch_sweep_all(smm_batch b, const double* const* phis) {
    smm_status st = b->fp32 ? batch_enqueue<float>(b, phis) : batch_enqueue<double>(b, phis);
    if (st != SMM_OK) return st;
    int e = 0;
    SMM_CUDA(cudaMemcpyAsync(&e, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    SMM_CUDA(cudaStreamSynchronize(b->stream));
    if (e == smm::DEV_TIMEOUT) {
        cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
        return fail(SMM_ERR_DEVICE_TIMEOUT, "a batched sweep dependency wait exceeded spin_timeout_s");
    }
    return SMM_OK;
}

}  // namespace

extern "C" {

smm_status smm_batch_create(int32_t n, const smm_handle* handles, smm_batch* out) {
    if (!out || n < 1 || !handles) return fail(SMM_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!handles[i]) return fail(SMM_ERR_INVALID_ARG, "NULL handle in batch");
    smm_handle h0 = handles[0];
    for (int i = 1; i < n; ++i) {
        if (handles[i]->fp32 != h0->fp32 || handles[i]->cached != h0->cached)
            return fail(SMM_ERR_INVALID_ARG, "batched problems must share sweep_precision and sweep_solver");
        if (handles[i]->stream != h0->stream || handles[i]->device != h0->device)
            return fail(SMM_ERR_INVALID_ARG, "batched problems must share the device and the stream");
    }
    long long total = 0;  // merged (problem, task) list is indexed with 32-bit integers
    for (int i = 0; i < n; ++i) total += handles[i]->ntask;
    if (total > (long long)INT32_MAX) return fail(SMM_ERR_INVALID_ARG, "batch too large: more than 2^31 - 1 tasks");
    auto* b = new smm_batch_ctx();
    auto bail = [&](smm_status st, const std::string& msg) { delete b; return fail(st, msg); };
    b->hs.assign(handles, handles + n);
    for (smm_handle h : b->hs) {
        b->ext |= h->opt.negative_flux_fixup || h->lagging || h->fmix_id != nullptr;
        b->pmax = std::max(b->pmax, h->p);
    }
    b->fp32 = h0->fp32;
    b->cached = h0->cached;
    b->stream = h0->stream;
    b->sms = h0->sms;
    // merged task list: level by level, problem by problem
    int maxlev = 0;
    for (smm_handle h : b->hs) maxlev = std::max(maxlev, h->nlevels);
    std::vector<int2> merged;
    for (int l = 0; l < maxlev; ++l)
        for (int i = 0; i < n; ++i) {
            smm_handle h = b->hs[i];
            if (l >= h->nlevels) continue;
            for (int t = h->level_start[l]; t < h->level_start[l + 1]; ++t) merged.push_back(make_int2(i, h->tasks_host[t]));
        }
    b->ntask = (int)merged.size();
    // every problem's elements, for the moment reductions after the batched sweep's tasks
    std::vector<int2> elems;
    for (int i = 0; i < n; ++i)
        for (int e = 0; e < b->hs[i]->ne; ++e) elems.push_back(make_int2(i, e));
    b->nelem = (int)elems.size();
    b->args_bytes = (size_t)n * (b->fp32 ? sizeof(smm::SweepArgs<float>) : sizeof(smm::SweepArgs<double>));
    if (cudaMalloc(&b->tasks, merged.size() * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&b->elems, elems.size() * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&b->args_dev, b->args_bytes) != cudaSuccess || cudaMallocHost(&b->args_host, b->args_bytes) != cudaSuccess ||
        cudaMalloc(&b->err, sizeof(int)) != cudaSuccess || cudaMalloc(&b->gate, sizeof(unsigned)) != cudaSuccess)
        return bail(SMM_ERR_OOM, "batch allocation failed");
    if (cudaMemcpyAsync(b->tasks, merged.data(), merged.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->elems, elems.data(), elems.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(b->err, 0, sizeof(int), b->stream) != cudaSuccess)
        return bail(SMM_ERR_CUDA, "batch upload failed");
    for (auto& e : b->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(SMM_ERR_CUDA, "cudaEventCreate failed");
    // autotune the launch shape (threads per block x resident fraction) on live sweeps
    const int mode = b->fp32 ? smm::SWEEP_RESIDUAL : smm::SWEEP_SOURCE;
    double best = 1e300;
    int best_grid = 1, best_block = 256;
    for (int block : {256, 128}) {
        const int bps = smm::batch_blocks_per_sm(mode, b->fp32, b->cached, b->ext, b->pmax, block);
        if (bps < 1) continue;
        for (int frac : {1, 2}) {
            const long long want = ((long long)b->ntask * 32 + block - 1) / block;
            b->grid = (int)std::max(1LL, std::min<long long>((long long)b->sms * bps / frac, want));
            b->block = block;
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                if (cudaEventRecord(b->ev[0], b->stream) != cudaSuccess) return bail(SMM_ERR_CUDA, "event");
                smm_status st = b->fp32 ? batch_enqueue<float>(b, nullptr) : batch_enqueue<double>(b, nullptr);
                if (st != SMM_OK) { delete b; return st; }
                if (cudaEventRecord(b->ev[1], b->stream) != cudaSuccess || cudaEventSynchronize(b->ev[1]) != cudaSuccess)
                    return bail(SMM_ERR_CUDA, "batched sweep failed during tuning");
                cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
            }
            int e = 0;
            cudaMemcpy(&e, b->err, sizeof(int), cudaMemcpyDeviceToHost);
            if (e != 0) return bail(SMM_ERR_DEVICE_TIMEOUT, "batched sweep wait expired during tuning");
            if (ms < best) { best = ms; best_grid = b->grid; best_block = block; }
        }
    }
    b->grid = best_grid;
    b->block = best_block;
    b->tuned_ms = best;
    *out = b;
    return SMM_OK;
}

smm_status smm_batch_schedule(smm_batch b, int32_t* grid, int32_t* block, double* tuned_ms, int64_t* n_tasks) {
    if (!b) return fail(SMM_ERR_INVALID_ARG, "NULL batch");
    if (grid) *grid = b->grid;
    if (block) *block = b->block;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    if (n_tasks) *n_tasks = b->ntask;
    return SMM_OK;
}

smm_status smm_batch_sweep(smm_batch b, const double* const* phi_dev) {
    if (!b) return fail(SMM_ERR_INVALID_ARG, "NULL batch");
    return batch_sweep_all(b, phi_dev);
}

smm_status smm_batch_iterate(smm_batch b, double tol, int32_t relative, int32_t max_outer, double* const* phi_dev,
                             smm_stats* stats) {
    if (!b || !phi_dev || !(tol > 0) || max_outer < 1) return fail(SMM_ERR_INVALID_ARG, "bad argument");
    const int n = (int)b->hs.size();
    std::vector<smm_stats> st(n);
    std::vector<char> done(n, 0);
    for (auto& s : st) s.cg_min = 1 << 30;
    std::vector<const double*> phis(phi_dev, phi_dev + n);
    for (smm_handle h : b->hs)
        if (!h->opt.resume_history) {
            h->aa_k = 0;
            h->dl1 = h->dl2 = 0.0;
        }
    int remaining = n;
    for (int k = 1; k <= max_outer && remaining > 0; ++k) {
        for (int i = 0; i < n; ++i) {
            smm_handle h = b->hs[i];
            SMM_CUDA(cudaMemcpyAsync(h->phi_prev, phi_dev[i], (size_t)h->ne * h->n * sizeof(double),
                                     cudaMemcpyDeviceToDevice, b->stream));
        }
        smm_status s = batch_sweep_all(b, phis.data());
        if (s != SMM_OK) return s;
        for (int i = 0; i < n; ++i) {
            if (done[i]) continue;
            smm_handle h = b->hs[i];
            s = enqueue_rhs(h);
            if (s != SMM_OK) return s;
            int it = 0;
            s = extrapolate_start(h, phi_dev[i]);
            if (s != SMM_OK) return s;
            s = run_cg(h, phi_dev[i], &it, inner_tol(h, k == 1 ? 1.0 : st[i].last_rel_diff));
            if (s != SMM_OK && s != SMM_ERR_NOT_CONVERGED) return s;
            const size_t nphi = (size_t)h->ne * h->n;
            SMM_CUDA(cudaMemsetAsync(h->nonfinite, 0, sizeof(int), h->stream));
            smm::launch_diff((int)nphi, phi_dev[i], h->phi_prev, h->dpart, h->dout, h->nonfinite, h->stream);
            SMM_CUDA(cudaMemcpyAsync(h->h_scal, h->dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            SMM_CUDA(cudaMemcpyAsync(h->h_int + 4, h->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            SMM_CUDA(cudaStreamSynchronize(h->stream));
            if (h->h_int[4]) return fail(SMM_ERR_NONFINITE, "non-finite scalar flux in a batched problem");
            smm_stats& q = st[i];
            q.outer_iterations = k;
            q.cg_total += it;
            q.cg_min = std::min(q.cg_min, it);
            q.cg_max = std::max(q.cg_max, it);
            q.last_diff = h->h_scal[0];
            q.last_rel_diff = h->h_scal[1] > 0 ? h->h_scal[0] / h->h_scal[1] : h->h_scal[0];
            s = record_step(h, q.last_diff);
            if (s != SMM_OK) return s;
            if (k == 1 && h->opt.guess_check && h->h_scal[0] > h->h_scal[1]) {
                // as in smm_iterate: the guess is farther from its image than zero is; restart from zero
                SMM_CUDA(cudaMemsetAsync(phi_dev[i], 0, nphi * sizeof(double), h->stream));
                q.guess_rejected = 1;
                h->aa_k = 0;
                h->dl1 = h->dl2 = 0.0;
                continue;
            }
            const double crit = relative ? q.last_rel_diff : q.last_diff;
            if (crit < tol) {
                done[i] = 1;
                --remaining;
            } else if (h->opt.anderson_depth > 0) {
                h->aa_k += 1;
                s = anderson_step(h, h->aa_k, phi_dev[i]);
                if (s != SMM_OK) return s;
            }
        }
    }
    for (auto& s : st)
        if (s.cg_min == (1 << 30)) s.cg_min = 0;
    if (stats)
        for (int i = 0; i < n; ++i) stats[i] = st[i];
    if (remaining > 0) return fail(SMM_ERR_NOT_CONVERGED, "outer iteration limit reached for some batched problems");
    return SMM_OK;
}

smm_status smm_batch_destroy(smm_batch b) {
    if (!b) return SMM_OK;
    cudaStreamSynchronize(b->stream);
    delete b;
    return SMM_OK;
}

}  // extern "C"

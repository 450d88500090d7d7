// Allocation-free block-Jacobi PCG entry point (see smm_block_pcg_noalloc in
// include/smm.h).
//
// Some callers cannot call cudaMalloc at all: code running under an
// allocator owned by another framework, processes with a fixed memory
// budget, or code paths that must not touch the CUDA allocator.  This entry
// point takes only caller-owned inputs and outputs and keeps every
// temporary vector and reduction slot of the CG iteration in one
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include "../../include/smm.h"
#include "kernels.cuh"

namespace {

constexpr long long kMaxRows = 1LL << 19;            // 524,288 unknowns
constexpr long long kMaxBlocks = kMaxRows / 128 + 2;  // row blocks hold >= 128 rows for n <= 64
// layout (bytes): r, z, p, q [kMaxRows] doubles | partials [3][kMaxBlocks] | scalars [8] | control [8] ints
constexpr long long kScratchBytes = 8LL * (4 * kMaxRows + 3 * kMaxBlocks + 8) + 4LL * 8;

static __device__ __align__(256) unsigned char g_pcg_scratch[kScratchBytes];

smm_status fail(smm_status s, const char* msg) {
    smm::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" smm_status smm_block_pcg_noalloc(int32_t n_elem, int32_t n, const double* diag_blocks,
                                            const double* off_blocks, const int32_t* nbr, const double* pinv_blocks,
                                            const double* b, double* x, double tol, int32_t max_iters,
                                            void* cuda_stream, int32_t* iters_out) {
    if (n_elem <= 0 || n <= 0 || n > 64 || !diag_blocks || !off_blocks || !nbr || !pinv_blocks || !b || !x ||
        !(tol > 0) || max_iters < 1)
        return fail(SMM_ERR_INVALID_ARG, "smm_block_pcg_noalloc: bad argument");
    const long long rows = (long long)n_elem * n;
    if (rows > kMaxRows)
        return fail(SMM_ERR_INVALID_ARG,
                    "smm_block_pcg_noalloc: n_elem * n exceeds the fixed scratch capacity of 524288 unknowns");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(SMM_ERR_CUDA, "smm_block_pcg_noalloc: no current CUDA device");
    // The array's device address in the current device's context, looked up on
    // every call: a cached address would go stale after cudaDeviceReset or in
    // another context of the same device, and the lookup costs microseconds
    // against a CG loop that synchronizes with the host.
    void* base = nullptr;
    if (cudaGetSymbolAddress(&base, g_pcg_scratch) != cudaSuccess || !base)
        return fail(SMM_ERR_CUDA, "smm_block_pcg_noalloc: cudaGetSymbolAddress failed");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* d = (double*)base;
    smm::CGArgs a{};
    a.ne = n_elem;
    a.n = n;
    a.nrow = (int)rows;
    const int epb = smm::cg_threads_per_block(n) / n;
    a.nblk = (n_elem + epb - 1) / epb;
    a.AdT_dense = diag_blocks;
    a.AoT_dense = off_blocks;
    a.nbr_dense = nbr;
    a.PinvT = pinv_blocks;
    a.x = x;
    a.r = d;
    a.z = d + kMaxRows;
    a.p = d + 2 * kMaxRows;
    a.q = d + 3 * kMaxRows;
    a.part = d + 4 * kMaxRows;
    a.scal = a.part + 3 * kMaxBlocks;
    a.ctl = (int*)(a.scal + 8);
    a.b = b;
    // the control words must start at zero; everything else is written before it is read
    if (cudaMemsetAsync(a.ctl, 0, 8 * sizeof(int), s) != cudaSuccess)
        return fail(SMM_ERR_CUDA, "smm_block_pcg_noalloc: cudaMemsetAsync failed");
    smm::cg_start(a, tol, max_iters, s);
    int ctl[4] = {0, 0, 0, 0};
    int chunk = 8;
    while (true) {
        if (cudaGetLastError() != cudaSuccess) return fail(SMM_ERR_CUDA, "smm_block_pcg_noalloc: launch failed");
        if (cudaMemcpyAsync(ctl, a.ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(SMM_ERR_CUDA, "smm_block_pcg_noalloc: synchronization failed");
        if (ctl[0]) break;
        smm::cg_iterations(a, chunk, s);
        chunk = chunk < 64 ? chunk * 2 : 64;
    }
    if (iters_out) *iters_out = ctl[1];
    if (ctl[3]) return fail(SMM_ERR_NONFINITE, "smm_block_pcg_noalloc: non-finite value");
    if (ctl[1] >= max_iters) {
        double sc[8];
        if (cudaMemcpyAsync(sc, a.scal, sizeof(sc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(SMM_ERR_CUDA, "smm_block_pcg_noalloc: synchronization failed");
        if (!(sc[2] <= sc[4])) return fail(SMM_ERR_NOT_CONVERGED, "smm_block_pcg_noalloc: iteration limit reached");
    }
    return SMM_OK;
}

/*
 * smm.h -- C ABI of the GB300 second-moment-method (SMM) transport library.
 *
 * The library solves the mono-energetic, steady, fixed-source transport
 * problem with isotropic scattering and inflow boundary conditions
 * (paper Sec. "Moment Methods for Radiation Transport", Eqs. transport and
 * inflow) by the SMM fixed-point iteration (Eqs. moment:smm_fp and
 * fixed-point):
 *
 *     varphi^{k+1} = D^{-1} b( L^{-1}( sigma_s/(4 pi) varphi^k + q ) ),
 *
 * where L^{-1} is a high-order upwind DG S_N transport sweep on curved
 * quadrilaterals (Sec. "Transport Discretization"), b(.) builds the
 * interior penalty SMM right-hand side from the discrete closures
 * (Eqs. correction_tensor_disc, bdr_correction_factor_disc, eb0_disc,
 * broken_Tdiv, ipsmm) and D is the fixed, symmetric IP diffusion operator
 * (Eq. ipsmm, left-hand side), solved by preconditioned CG.
 *
 * Conventions (all calls):
 *  - Reference element [0,1]^2; nodal points on tensor Gauss-Lobatto points,
 *    lexicographic with x fastest: i = iy*(k+1) + ix.  DG order p: n = (p+1)^2
 *    nodal values per element.  Geometry order m: (m+1)^2 control points.
 *  - Faces: 0 bottom (eta=0), 1 right (xi=1), 2 top (eta=1), 3 left (xi=0);
 *    the face parameter s increases with the reference coordinate that
 *    varies along the face.  Boundary faces are numbered by ascending
 *    (element, face).
 *  - Ordinates (level-symmetric LQ_N, N in {2,4,6,8,10,12}, N(N+2)/2 of them
 *    in 2D) are numbered quadrant-major: (+,+), (-,+), (-,-), (+,-); within
 *    a quadrant by the octant level triple (i,j,k), i then j ascending.
 *    Weights sum to 4 pi.
 *  - Host pointers ("host") are read during the call only; the caller keeps
 *    ownership.  Device pointers ("dev") must be allocated by the caller on
 *    the device of the handle's stream; the library never frees them.
 *  - Every call returns an smm_status; nothing aborts or throws across the
 *    ABI.  smm_last_error() gives a message for the calling thread's most
 *    recent failure.  After SMM_ERR_CUDA the handle must only be destroyed.
 *  - One handle per stream; calls on one handle are not thread safe.
 */
#ifndef SMM_H
#define SMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smm_ctx* smm_handle;

typedef enum {
    SMM_OK = 0,
    SMM_ERR_INVALID_ARG = 1,    /* bad size, NULL where required, unsupported order */
    SMM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    SMM_ERR_OOM = 3,            /* device allocation failed */
    SMM_ERR_MESH = 4,           /* non-positive Jacobian, broken connectivity */
    SMM_ERR_CYCLE = 5,          /* an ordinate's upwind graph has a cycle (a face
                                   that is inflow at some points and outflow at
                                   others makes one) and options.cycle_lagging is
                                   0, or the sweep mode cannot lag it */
    SMM_ERR_NONFINITE = 6,      /* NaN/Inf in an iterate */
    SMM_ERR_NOT_CONVERGED = 7,  /* iteration limit reached; the iterate is kept */
    SMM_ERR_DEVICE_TIMEOUT = 8  /* a bounded device-side wait expired */
} smm_status;

enum { SMM_SOURCE_ISOTROPIC = 0, SMM_SOURCE_ANGULAR = 1 };
enum { SMM_INFLOW_VACUUM = 0, SMM_INFLOW_NODAL = 1 };
enum { SMM_SWEEP_FP64 = 0, SMM_SWEEP_FP32_REFINED = 1 };
enum { SMM_PRECOND_BLOCK_JACOBI = 0, SMM_PRECOND_MULTIGRID = 1 };
enum { SMM_SOLVER_LU = 0, SMM_SOLVER_CACHED_INVERSE = 1 };
enum { SMM_MOMENT_IP = 0, SMM_MOMENT_CG = 1 };
enum { SMM_SMOOTHER_JACOBI = 0, SMM_SMOOTHER_CHEBYSHEV = 1 };

typedef struct {
    int32_t n_elem;             /* number of quadrilaterals */
    int32_t geom_order;         /* m >= 1 */
    int32_t n_nodes;            /* number of control points */
    const double* nodes;        /* host [n_nodes][2] control point coordinates */
    const int32_t* elem_nodes;  /* host [n_elem][(m+1)^2] control point ids,
                                   lexicographic Gauss-Lobatto order; elements
                                   must be positively oriented (J > 0) and
                                   neighbours share face control points */
} smm_mesh;

typedef struct {
    int32_t sweep_precision;    /* SMM_SWEEP_FP64 (default): local solves in
                                   FP64.  SMM_SWEEP_FP32_REFINED: each sweep
                                   solves for a correction in FP32 from an FP64
                                   transport residual (moments, CG, checks stay
                                   FP64). */
    double tol_cg;              /* CG stop: ||r||_2 <= tol_cg ||b||_2 (default 1e-12) */
    int32_t max_cg;             /* CG iteration cap per moment solve (default 20000) */
    double kappa_scale;         /* multiplies the IP penalty (default 1) */
    double spin_timeout_s;      /* bound on every device-side wait (default 2 s) */
    int32_t precond;            /* moment-solve preconditioner: SMM_PRECOND_MULTIGRID
                                   (default) or SMM_PRECOND_BLOCK_JACOBI */
    int32_t sweep_solver;       /* SMM_SOLVER_CACHED_INVERSE (default): every local
                                   operator A_{K,d} is inverted once at create
                                   (it does not change between sweeps) and a sweep
                                   task is an n x n matrix-vector product;
                                   needs n_elem * n_ord * n^2 words of device
                                   memory.  SMM_SOLVER_LU: assemble and factor
                                   every local system in registers per sweep. */
    int32_t anderson_depth;     /* smm_iterate: 0 (default) plain fixed point
                                   varphi^{k+1} = G(varphi^k); 1..5 Anderson
                                   acceleration of that depth (paper Sec. "The
                                   Moment Method Algorithm"; depth 2 in its
                                   crooked-pipe runs), with moment-sized history */
    int32_t guess_check;        /* smm_iterate: if nonzero and the first outer step
                                   from the given guess x0 moves it farther than
                                   its image is from zero, i.e.
                                   max|G(x0) - x0| > max|G(x0) - 0|, the guess is
                                   rejected and the iteration restarts from zero
                                   with an empty Anderson history.  This compares
                                   the guess with the zero vector as starting
                                   points for the same image G(x0); it stands in
                                   for the first residual of the zero guess,
                                   max|G(0)|, which would cost one more outer
                                   step (default 0) */
    int32_t mg_smooth_steps;    /* multigrid preconditioner: smoothing steps on
                                   the DG level before and after the coarse
                                   correction (the Chebyshev degree with
                                   SMM_SMOOTHER_CHEBYSHEV), 1..4 (default 3);
                                   also the point-Jacobi steps of the
                                   continuous system's V-cycle */
    int32_t moment_discretization; /* SMM_MOMENT_IP (default): interior penalty
                                   moment system on the DG space (paper Eq.
                                   ipsmm).  SMM_MOMENT_CG: the continuous
                                   finite element system (Sec. "Discontinuous
                                   Galerkin and Continuous Finite Element"):
                                   Eq. ipsmm with test and trial space V_p,
                                   solved by flexible CG with a V-cycle of
                                   point-Jacobi smoothing on the continuous
                                   nodes (any `precond`); varphi is still
                                   passed as DG nodal values, and the solve
                                   returns P varphi (equal values at shared
                                   nodes). */
    int32_t negative_flux_fixup; /* nonzero: the zero and scale negative flux
                                   fixup inside the sweep (paper Sec. "Crooked
                                   Pipe"): after each element solve, negative
                                   nodal values are set to zero and the rest
                                   scaled so that the element's particle
                                   balance (local system tested with v = 1)
                                   keeps its value (zero if that value is not
                                   positive).  FP64 sweeps only
                                   (INVALID_ARG with SMM_SWEEP_FP32_REFINED).
                                   Default 0: SMM closures need no positivity. */
    int32_t sweep_tiles;        /* T > 1: parallel block Jacobi sweep (paper Sec.
                                   "Weak Scaling"): the mesh's bounding box is
                                   cut into T x T tiles, an element belongs to
                                   the tile holding the mean of its four corner
                                   control points, every tile sweeps its own
                                   elements, and inflow across tile borders is
                                   taken from the previous sweep (zero at
                                   first).  Shortens the sweep's dependency
                                   chains; the outer iteration needs more steps
                                   and converges to the same fixed point.
                                   1..64, default 1 (exact sweep); FP64 sweeps
                                   only. */
    int32_t mg_smoother;        /* level-0 smoother of the IP-SMM multigrid
                                   preconditioner: SMM_SMOOTHER_CHEBYSHEV
                                   (default: the Chebyshev polynomial of degree
                                   mg_smooth_steps in Pinv A on
                                   [lambda_max / 60, lambda_max]) or
                                   SMM_SMOOTHER_JACOBI (damped element-block
                                   Jacobi, omega = (4/3) / lambda_max); the
                                   same cost per step.  lambda_max is a
                                   power-iteration estimate times 1.05. */
    int32_t cg_device_loop;     /* multigrid CG: nonzero (default) runs the
                                   whole CG loop as one graph launch (a
                                   device-controlled while node over one
                                   iteration); 0 launches the one-iteration
                                   graph in chunks checked by the host (for
                                   profilers that do not see kernels inside
                                   conditional graph nodes).  The same
                                   arithmetic either way. */
    int32_t resume_history;     /* smm_iterate / smm_batch_iterate: 0 (default)
                                   starts every call with an empty Anderson
                                   history (and no extrapolation history, see
                                   cg_guess_extrapolate); nonzero continues the
                                   history that
                                   the previous call on the handle left (or that
                                   smm_set_state restored), so that an iteration
                                   split over several calls, or restarted from a
                                   checkpoint, takes the same steps as one
                                   uninterrupted call.  The caller passes the
                                   iterate the previous call returned. */
    int32_t cycle_lagging;      /* nonzero (default): cycles of the ordinates'
                                   upwind graphs are lagged, as the paper does on
                                   its distorted mesh (Sec. "Thick Diffusion
                                   Limit"): when no element is left whose upwind
                                   neighbours are all swept, the lowest-numbered
                                   remaining element is swept next and its
                                   inflow from neighbours not yet swept is taken
                                   from the previous sweep (zero before the
                                   first).  A face that is inflow at some
                                   quadrature points and outflow at others is
                                   upwinded pointwise.  The iteration converges
                                   to the same fixed point in more outer steps.
                                   FP64 sweeps without the fixup only (else
                                   SMM_ERR_CYCLE).  0: a cycle is SMM_ERR_CYCLE. */
    double cg_tol_adaptive;     /* smm_iterate / smm_batch_iterate: eta > 0 solves
                                   the moment system of outer step k only to
                                   ||r||_2 <= max(tol_cg, eta d_{k-1}) ||b||_2,
                                   d_{k-1} the previous step's relative
                                   successive difference (1 before the first):
                                   an inexact inner solve that tightens as the
                                   outer iteration converges (the paper's
                                   crooked-pipe runs solve the moment system
                                   to 1e-8 for an outer tolerance of 1e-6).
                                   Default 0: every solve to tol_cg. */
    int32_t cg_guess_extrapolate; /* smm_iterate / smm_batch_iterate without
                                   Anderson acceleration: nonzero (default)
                                   starts the moment solve of outer step k
                                   from varphi_k + rho (varphi_k - varphi_{k-1}),
                                   rho = d_{k-1} / d_{k-2} (the ratio of the last
                                   two successive differences, clamped to
                                   [0, 0.9]) instead of from varphi_k, once two
                                   steps of this call (or, with resume_history,
                                   of earlier calls) exist: the outer iteration
                                   converges linearly, so the extrapolation
                                   starts the CG closer to its solution.  The
                                   same fixed point; 0: start from varphi_k. */
} smm_options;

typedef struct {
    int32_t n_elem, p, m, n_dof_elem, n_ord, n_bface, n_fq, n_levels;
    int64_t n_angular;          /* n_elem * n_dof_elem * n_ord */
    int64_t n_lagged;           /* (element, ordinate, face) inflows lagged to break cycles */
} smm_info;

typedef struct {
    int32_t outer_iterations;
    int32_t cg_total, cg_min, cg_max; /* CG iterations over the outer steps */
    double last_diff;           /* max |varphi^{k+1} - varphi^k| of the last step */
    double last_rel_diff;       /* last_diff / max |varphi^{k+1}| */
    double ms_residual;         /* FP64 transport residual kernel (refined mode) */
    double ms_sweep;            /* sweep kernel alone */
    double ms_moments, ms_rhs, ms_solve; /* moments + beta, RHS, CG (accumulated, ms) */
    int64_t n_launches;         /* kernels this library launched during the call */
    int32_t guess_rejected;     /* 1 if guess_check restarted the iteration from zero */
} smm_stats;

/* Fill *opt with the defaults listed above. */
void smm_default_options(smm_options* opt);

/* The library's level-symmetric quadrature for S_N order sn_order
 * (paper: "Level Symmetric S_N", not printed; LQ_N construction).
 * omega_out: host [n_ord][2] (may be NULL), w_out: host [n_ord] (may be
 * NULL), n_ord_out: number of ordinates N(N+2)/2.
 * Errors: SMM_ERR_INVALID_ARG for unsupported orders. */
smm_status smm_quadrature(int32_t sn_order, double* omega_out, double* w_out, int32_t* n_ord_out);

/* Build a solver for the transport problem of Eqs. transport and inflow
 * (Sec. "Moment Methods for Radiation Transport") on a mesh of curved
 * quadrilaterals with the DG discretization of Sec. "Transport
 * Discretization" (nodal Q_p on Gauss-Lobatto points, upwind fluxes) and the
 * IP-SMM moment system of Eq. ipsmm (penalty kappa of Sec. "Results"):
 * geometry factors, element and face matrices, upwind level lists per
 * ordinate, the IP-SMM operator blocks and its preconditioner; uploads
 * everything to the device of cuda_stream (NULL = legacy default stream of
 * the current device).  The handle owns all device memory it allocates.
 *   p: DG order 1..4.  sn_order: see smm_quadrature.
 *   sigma_t, sigma_s: host [n_elem], piecewise constant, sigma_t > 0,
 *     0 <= sigma_s <= sigma_t.
 *   source_kind SMM_SOURCE_ISOTROPIC: q host [n_elem][n] nodal values per
 *     steradian; SMM_SOURCE_ANGULAR: q host [n_ord][n_elem][n].
 *   inflow_kind SMM_INFLOW_VACUUM: inflow ignored (may be NULL);
 *     SMM_INFLOW_NODAL: inflow host [n_ord][n_bface][p+1], psibar at the face
 *     nodal points in increasing s (used only where the ordinate enters).
 *   opt: NULL for defaults.
 * Errors: INVALID_ARG (also when n_elem times the ordinates, the control
 * points or the dofs per element exceeds 2^31 - 1: those ids are 32-bit),
 * MESH (J <= 0 at a quadrature point, a face shared by more than two
 * elements), CYCLE (see above), OOM, CUDA. */
smm_status smm_create(const smm_mesh* mesh, int32_t p, int32_t sn_order,
                      const double* sigma_t, const double* sigma_s,
                      int32_t source_kind, const double* q,
                      int32_t inflow_kind, const double* inflow,
                      const smm_options* opt, void* cuda_stream, smm_handle* out);

smm_status smm_get_info(smm_handle h, smm_info* info);

/* One transport sweep psi = L^{-1}(sigma_s/(4 pi) varphi + q) over all
 * ordinates (Sec. "Transport Discretization"), followed by the angular
 * moments and the boundary correction (Eqs. correction_tensor_disc,
 * bdr_correction_factor_disc), kept in the handle.
 *   phi_dev: dev [n_elem][n] FP64, or NULL for varphi = 0.
 *   phiT_out: NULL, or host or device [n_elem][n] FP64 that receives the
 *     transport scalar flux phi_T = sum_d w_d psi_d of this sweep.
 * In SMM_SWEEP_FP32_REFINED mode the sweep corrects the handle's current
 * angular flux (zero after create) and repeated calls converge to the FP64
 * result.  Errors: DEVICE_TIMEOUT (the handle stays usable; the next sweep
 * starts afresh), CUDA. */
smm_status smm_sweep(smm_handle h, const double* phi_dev, double* phiT_out);

/* Copy the moments of the last sweep.  moments_dev: dev [6][n_elem][n]
 * (phi, Jx, Jy, Txx, Txy, Tyy), or NULL; beta_dev: dev [n_bface][n_fq]
 * boundary correction beta at the face Gauss points, or NULL. */
smm_status smm_moments(smm_handle h, double* moments_dev, double* beta_dev);

/* Replace the handle's closures (the state a sweep would leave): used to
 * solve the moment system with given T and beta (paper's isolated MMS
 * study) and to restore a checkpoint.  Same layouts as smm_moments. */
smm_status smm_set_moments(smm_handle h, const double* moments_dev, const double* beta_dev);

/* Copy the angular flux of the last sweep: psi_dev dev [n_elem][n_ord][n] FP64. */
smm_status smm_get_psi(smm_handle h, double* psi_dev);

/* Solve the IP-SMM moment system (Eq. ipsmm) with the handle's closures by
 * preconditioned flexible CG: a multigrid V-cycle (Chebyshev or damped
 * element-block Jacobi smoothing on Y_p, options.mg_smoother; Galerkin coarse
 * level of continuous bilinear functions on the mesh vertices, smoothed
 * aggregation below it, dense coarsest solve), the iterations run as one
 * device-side graph loop (options.cg_device_loop), or element-block Jacobi
 * alone (options.precond).  phi_dev: dev [n_elem][n], in: initial
 * guess, out: solution.  cg_iters (host, may be NULL): iterations used.
 * Errors: NOT_CONVERGED (phi_dev holds the last iterate), NONFINITE, CUDA. */
smm_status smm_moment_solve(smm_handle h, double* phi_dev, int32_t* cg_iters);

/* The SMM fixed-point iteration of Eqs. moment:smm_fp and fixed-point
 * (Sec. "The Moment Method Algorithm"), varphi^{k+1} = G(varphi^k): sweep,
 * moments, right-hand side, moment solve, until
 * max|varphi^{k+1}-varphi^k| < tol (relative == 0) or
 * max|varphi^{k+1}-varphi^k| / max|varphi^{k+1}| < tol (relative != 0), or
 * max_outer steps; with options.anderson_depth > 0 the steps are Anderson
 * accelerated.
 *   phi: host or device [n_elem][n] FP64 (the library tells them apart from
 *     the pointer): the guess on entry, the last iterate on return (also
 *     after NOT_CONVERGED and NONFINITE).  A host array is copied to the
 *     device once before the first step and back once after the last.
 *   stats: host, may be NULL.
 * Errors: INVALID_ARG, NOT_CONVERGED, NONFINITE, DEVICE_TIMEOUT, CUDA. */
smm_status smm_iterate(smm_handle h, double tol, int32_t relative, int32_t max_outer, double* phi,
                       smm_stats* stats);

/* Change the bound on every device-side wait of the handle's later sweeps
 * (options.spin_timeout_s; Sec. "Transport Discretization" orders the sweep
 * by upwind dependencies, whose waits these are).  seconds > 0, else
 * INVALID_ARG.  After a wait expires (DEVICE_TIMEOUT) the handle stays
 * usable: the next sweep uses a new flag epoch, so flags left by the aborted
 * sweep are never taken for finished work. */
smm_status smm_set_spin_timeout(smm_handle h, double seconds);

/* ---- Checkpoint ----
 * The state a later call depends on besides its arguments: the angular flux
 * of the last sweep (which the next FP32-refined sweep corrects and a block
 * Jacobi sweep lags), the moments and boundary correction (the next moment
 * solve's closures), the previous iterate, the Anderson history with its
 * length and the extrapolated CG start's history (the input of the step
 * before and the last two successive differences).  Restoring it into a handle created with the same mesh, data and
 * options makes the following calls return bit for bit what they would have
 * returned on the saved handle.  The buffer is opaque (a 256-byte header,
 * then the arrays), host or device memory alike, owned by the caller.
 *   smm_state_size: *bytes = the size of the state.
 *   smm_get_state: write it to buf (at least that many bytes).
 *   smm_set_state: restore it from buf.
 * Errors: INVALID_ARG (small buffer; a state of another shape or mode),
 * CUDA. */
smm_status smm_state_size(smm_handle h, int64_t* bytes);
smm_status smm_get_state(smm_handle h, void* buf, int64_t bytes);
smm_status smm_set_state(smm_handle h, const void* buf, int64_t bytes);

smm_status smm_destroy(smm_handle h);

/* ---- Batched problems ----
 * Many problems of uneven mesh size, order p and S_N order swept in one
 * cooperative launch: their level-sorted task lists are merged level by level
 * and every task dispatches on its problem's p.  Problems keep their own
 * state; only the sweep is shared.  The launch shape (threads per block,
 * resident blocks per SM) is autotuned on live sweeps at creation. */
typedef struct smm_batch_ctx* smm_batch;

/* handles: n problems created with the same sweep_precision, sweep_solver,
 * device and stream; they must outlive the batch.  Creation runs a few
 * sweeps with varphi = 0 to tune the launch (the handles' sweep state
 * changes as by smm_sweep).  Errors: INVALID_ARG (also for more than
 * 2^31 - 1 element-ordinate tasks in all), OOM, CUDA, DEVICE_TIMEOUT. */
smm_status smm_batch_create(int32_t n, const smm_handle* handles, smm_batch* out);

/* Chosen launch shape and the tuned time of one batched sweep (ms). */
smm_status smm_batch_schedule(smm_batch b, int32_t* grid, int32_t* block, double* tuned_ms, int64_t* n_tasks);

/* One sweep of every problem (as smm_sweep for each) in one launch.
 * phi_dev: host array of n device pointers (entries NULL for varphi = 0). */
smm_status smm_batch_sweep(smm_batch b, const double* const* phi_dev);

/* smm_iterate for every problem, sharing the batched sweep: each outer step
 * runs one batched sweep, then each unconverged problem's moment solve
 * (with each handle's anderson_depth, guess_check and resume_history).
 * phi_dev: host array of n device pointers (guesses in, iterates out);
 * stats: NULL or n entries.  Errors as smm_iterate. */
smm_status smm_batch_iterate(smm_batch b, double tol, int32_t relative, int32_t max_outer, double* const* phi_dev,
                             smm_stats* stats);

smm_status smm_batch_destroy(smm_batch b);

/* ---- Learned initial guess (not part of the paper's method) ----
 * A convolutional encoder-decoder on an H x W element grid (H, W even)
 * mapping 3 input channels (normalized sigma_t, scattering ratio, source) to
 * n_out output channels (normalized nodal varphi), trained and evaluated by
 * the library's own tensor-core kernels: BF16 weights, activations and stored
 * gradients, FP32 accumulation, FP32 master weights, Adam, mean squared
 * error.  Layers: a1 = relu(conv3x3(x, 3 -> c1)), a2 = relu(conv3x3 stride 2
 * (a1, c1 -> c2)), a3 = relu(conv3x3(a2, c2 -> c2)), a4 = relu(conv3x3(up2(a3),
 * c2 -> c1)), a5 = relu(conv3x3([a4, a1], 2 c1 -> c1)), y = conv1x1(a5, c1 ->
 * n_out); parameters flat, layer by layer: weights [cout][cin][ky][kx], then
 * biases [cout].  Layouts: inputs dev [batch][3][H][W] FP32, outputs and
 * targets dev [batch][n_out][H][W] FP32.  The network only proposes a starting
 * point: smm_iterate still runs to the same tolerance, and options.guess_check
 * makes it fall back to the zero guess when the proposal raises the first
 * residual. */
typedef struct smm_guess_ctx* smm_guess;

/* c1, c2: the widths (24 / 32 for a small network, 64 / 384 for about two
 * million parameters); max_batch: largest batch of later calls (the
 * activations of max_batch samples are allocated here); seed: weight
 * initialization.  SMM_ERR_INVALID_ARG for odd or tiny grids, widths outside
 * 1..1024, or max_batch x H x W x width beyond 2^31; SMM_ERR_OOM when the
 * device allocations fail. */
smm_status smm_guess_create(int32_t height, int32_t width, int32_t n_out, int32_t c1, int32_t c2, int32_t max_batch,
                            uint64_t seed, void* cuda_stream, smm_guess* out);
smm_status smm_guess_num_params(smm_guess g, int64_t* n);
smm_status smm_guess_forward(smm_guess g, int32_t batch, const float* in_dev, float* out_dev);
/* One Adam step (learning rate lr) on the batch; loss_host (may be NULL) gets the batch loss before the step. */
smm_status smm_guess_train_step(smm_guess g, int32_t batch, const float* in_dev, const float* target_dev, float lr,
                                float* loss_host);
/* Loss and parameter gradients (host, n_params floats; may be NULL) without updating the weights. */
smm_status smm_guess_gradients(smm_guess g, int32_t batch, const float* in_dev, const float* target_dev,
                               float* grad_host, float* loss_host);
/* FP32 master weights to / from a host buffer of n_params floats (checkpoint). */
smm_status smm_guess_get_params(smm_guess g, float* host);
smm_status smm_guess_set_params(smm_guess g, const float* host);
smm_status smm_guess_destroy(smm_guess g);

/* Allocation-free block-Jacobi preconditioned CG.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code that runs under another framework's allocator, inside
 * a fixed memory budget, or on a path that must not touch the CUDA
 * allocator.  It solves A x = b for a symmetric positive definite operator
 * made of n x n blocks on an element graph (the layout smm uses for the
 * IP-SMM operator) and allocates nothing: the CG vectors and reduction
 * slots live in one fixed __device__ array of about 16.9 MB that every GPU
 * which loads the library holds until the process exits.
 *   n_elem, n: blocks of n unknowns (1 <= n <= 64); n_elem * n must not
 *     exceed 524288 (else SMM_ERR_INVALID_ARG).
 *   diag_blocks: dev [n_elem][n][n], off_blocks: dev [n_elem][4][n][n] (block
 *     coupling element e to its neighbour across face f), pinv_blocks: dev
 *     [n_elem][n][n] (inverse of each diagonal block); every block is stored
 *     column-major: entry (i, j) at [j*n + i].
 *   nbr: dev [n_elem][4] neighbour element ids, -1 where there is none.
 *   b: dev [n_elem*n]; x: dev [n_elem*n], in: initial guess, out: solution.
 *   Stops when ||r||_2 <= tol ||b||_2 or after max_iters iterations.
 *   cuda_stream: stream of the current device (NULL = legacy default);
 *   iters_out (host, may be NULL): iterations used.
 * Every call looks up the array's device address in the current device's
 * context (so a device reset or another context needs nothing from the
 * caller); the first call on a device may load the library's device code,
 * so make it before any stream capture.  All
 * calls share the array and it keeps the last call's contents; calls that
 * overlap on the GPU (other streams, other threads) race and must be
 * serialized by the caller.
 * Errors: INVALID_ARG, NOT_CONVERGED (x holds the last iterate), NONFINITE, CUDA. */
smm_status smm_block_pcg_noalloc(int32_t n_elem, int32_t n, const double* diag_blocks, const double* off_blocks,
                                 const int32_t* nbr, const double* pinv_blocks, const double* b, double* x,
                                 double tol, int32_t max_iters, void* cuda_stream, int32_t* iters_out);

/* Message of the calling thread's most recent error ("" if none); valid
 * until the next call on that thread. */
const char* smm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SMM_H */

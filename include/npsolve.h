/*
 * npsolve.h -- C ABI of the B300 (sm_103a) neural-preconditioned Poisson
 * solver: NPSDO (Sec. 4.1, Algorithm 1 of arXiv 2310.00177) with the
 * image-conditioned multilevel network P_net of Sec. 4.2 (Algorithm 2).
 *
 * The problem (Sec. 3.2): a voxel grid of nx*ny*nz cells, each labelled
 * fluid, air (Dirichlet p = 0) or solid (Neumann; the region outside the grid
 * counts as solid).  A is the masked 7-point Laplacian on the fluid cells
 * (stencil points outside the fluid dropped, diagonal = number of fluid-or-air
 * neighbours, rows/columns of non-fluid cells empty).  Every vector is stored
 * on the full grid, x fastest: index p = (z*ny + y)*nx + x; entries at
 * non-fluid cells are ignored on input and written as 0 on output (this is
 * the paper's reduced system A~ x~ = b~ without the gather/scatter).
 *
 * Labels: uint8, 0 = solid, 1 = fluid, 2 = air (0 is solid so that a
 * zero-filled halo is the paper's solid padding, Sec. 4.2.1).  Any other code
 * is rejected with NPSOLVE_BAD_LABELS.
 *
 * Memory and ownership: unless a name ends in _host, every array argument is
 * a DEVICE pointer on the current CUDA device, owned by the caller, and must
 * stay valid until the call returns (all calls are synchronous with respect
 * to the host; work is issued on `stream`, a cudaStream_t, 0 = legacy default
 * stream).  Device arrays are accessed with 8- and 16-byte vector loads and
 * stores, so every device pointer must be 16-byte aligned (cudaMalloc and
 * framework allocators return far larger alignments; an offset view into one
 * may not be): a misaligned one is rejected with NPSOLVE_BAD_ARG.  The handle owns its scratch memory (Krylov state, image pyramid,
 * network intermediates), allocates it on first use for a grid size, reuses
 * it for equal or smaller grids, and frees it in npsolve_destroy.  There is
 * no CPU fallback: without a usable sm_103a device every call fails with
 * NPSOLVE_CUDA_ERROR.
 *
 * Errors: every int-returning call returns an npsolve_status; on failure a
 * message is available from npsolve_last_error(handle) (or
 * npsolve_last_error(NULL) for errors of calls without a handle, per thread).
 * A handle must not be used from two host threads at once.
 */
#ifndef NPSOLVE_H
#define NPSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct npsolve *npsolve_t;

typedef enum {
  NPSOLVE_OK = 0,
  NPSOLVE_BAD_ARG = 1,        /* null pointer, bad tolerance, non-finite b, ... */
  NPSOLVE_BAD_DIMS = 2,       /* a dimension not divisible by 2^(L-1) (Sec. 4.2.1) */
  NPSOLVE_BAD_LABELS = 3,     /* a label outside {0, 1, 2} */
  NPSOLVE_NO_CONVERGENCE = 4, /* max_iter reached; x, iters, residual still written */
  NPSOLVE_BREAKDOWN = 5,      /* d^T A d <= 0 or non-finite in Alg. 1; x so far written */
  NPSOLVE_OOM = 6,            /* device allocation failed */
  NPSOLVE_CUDA_ERROR = 7      /* a CUDA call failed (message has the CUDA error) */
} npsolve_status;

enum { NPSOLVE_LABEL_SOLID = 0, NPSOLVE_LABEL_FLUID = 1, NPSOLVE_LABEL_AIR = 2 };

/* Precision forms of the network evaluation.  Vectors are FP32, dot products
 * and orthogonalisation coefficients FP64 and x FP64 in both forms. */
enum {
  NPSOLVE_FP32 = 0, /* per-cell kernels generated and applied to FP32 accuracy (on the tensor cores: the
                       FP32 weights split into three BF16 terms, FP32 accumulation) */
  NPSOLVE_BF16 = 1  /* CConv weights rounded to BF16, kernels accumulated in FP32 and stored/used as BF16
                       values, applied with FP32 accumulation; vectors, Aff coefficients and the solver
                       as in the FP32 form */
};

/* Residual update of Alg. 1. */
enum {
  NPSOLVE_RESIDUAL_RECURRENCE = 0, /* r_k = r_{k-1} - alpha_k A d_k; on exit the FP64 true residual
                                      is checked and, if above tolerance, r is replaced by b - A x and
                                      the iteration continues (at most 4 times) */
  NPSOLVE_RESIDUAL_EXPLICIT = 1    /* r_k = b - A x_k every iteration, as printed in Alg. 1 */
};

/* How CConv obtains its per-cell kernels K_a(p) (Sec. 4.2.1). */
enum {
  NPSOLVE_PATH_CACHED = 0,    /* default: once per solve, the kernels of the cells whose 3x3x3 image window
                                 is not uniform are generated and cached (a uniform window gives the exact
                                 closed form Bp + nF*SWf + nA*SWa); every iteration then runs a z-marching
                                 27-point stencil with fused pooling / interpolation / combination */
  NPSOLVE_PATH_CUDA_CORE = 1, /* every iteration regenerates every kernel with FP32 FMAs; reference path */
  NPSOLVE_PATH_TENSOR = 2     /* every iteration regenerates every kernel on the tcgen05 tensor cores
                                 (levels 1-3, BF16 operands, FP32 accumulation), CUDA cores beyond */
};

/* The Krylov method that npsolve_solve runs with the network as preconditioner
 * (Sec. 4.1 and the solver-variant comparison of the appendix). */
enum {
  NPSOLVE_METHOD_NPSDO = 0, /* Alg. 1: steepest descent with A-orthogonalisation against n_ortho directions */
  NPSOLVE_METHOD_PCG = 1,   /* preconditioned CG (Shewchuk's form): z_k = P(r_k), rho_k = r_k^T z_k,
                               d_k = z_k + (rho_k / rho_{k-1}) d_{k-1}, alpha_k = rho_k / d_k^T A d_k */
  NPSOLVE_METHOD_FPCG = 2   /* flexible PCG (Polak-Ribiere form for a non-symmetric preconditioner):
                               beta_k = z_k^T (r_k - r_{k-1}) / rho_{k-1}, otherwise as PCG */
};

typedef struct {
  int levels;        /* L, number of network levels, 1..7 (paper: 6; L = 4 ~ 16k parameters) */
  int n_ortho;       /* directions to A-orthogonalise against, 0..4 (paper: 2, Sec. 4.1); NPSDO only */
  int precision;     /* NPSOLVE_FP32 or NPSOLVE_BF16 */
  int residual_mode; /* NPSOLVE_RESIDUAL_RECURRENCE or NPSOLVE_RESIDUAL_EXPLICIT */
  int kernel_path;   /* NPSOLVE_PATH_CACHED, NPSOLVE_PATH_CUDA_CORE or NPSOLVE_PATH_TENSOR */
  int method;        /* NPSOLVE_METHOD_NPSDO (0, the paper's solver), _PCG or _FPCG */
  int symmetric;     /* 0: the preconditioner is P_net; 1: the symmetric variant P_sym,1 = P_net^T P_net
                        of the paper's symmetry analysis (appendix), with any method */
} npsolve_config;

/* Number of FP32 network parameters for L levels (Alg. 2): for each level
 * l < L the blocks CConv1 (W 27x3x27, B 27), CConv2 (same), Aff1 (Wbar 3x27,
 * Bbar 1), Aff2 (same), in that order, then CConv1 of level L.
 * W[a][c][l]: a = output tap, c = image channel (0 fluid, 1 air, 2 solid),
 * l = image window offset; taps/offsets t = 9(dz+1) + 3(dy+1) + (dx+1).
 * L = 4 gives 15,990; L = 6 gives 25,174. */
size_t npsolve_weight_count(int levels);

/* Create a solver handle on the current device.  `weights_host` (host
 * memory, n_weights == npsolve_weight_count(cfg->levels) floats) is copied.
 * Returns NPSOLVE_BAD_ARG for an invalid config, NPSOLVE_CUDA_ERROR when no
 * sm_103a device is usable. */
int npsolve_create(const npsolve_config *cfg, const float *weights_host, size_t n_weights, npsolve_t *out);

/* Replace / read back the network weights (host memory, FP32). */
int npsolve_set_weights(npsolve_t h, const float *weights_host, size_t n_weights);
int npsolve_get_weights(npsolve_t h, float *weights_host, size_t n_weights);

/* Release the handle and all device memory it owns.  NULL is ignored. */
void npsolve_destroy(npsolve_t h);

/* Last error message of the handle (or of this thread for h == NULL);
 * valid until the next call on the same handle/thread. */
const char *npsolve_last_error(npsolve_t h);

/* Solve A x = b with NPSDO (Alg. 1): x_0 = 0, r_0 = b; while ||r_k|| >=
 * tol*||b||: d_k = P_net(I, r_{k-1}/||r_{k-1}||) (Alg. 2), A-orthogonalise
 * d_k against the last n_ortho directions, exact line search
 * alpha_k = r_{k-1}^T d_k / d_k^T A d_k, x_k = x_{k-1} + alpha_k d_k.
 *   labels [nz][ny][nx] uint8 (device); b [nz][ny][nx] FP32 (device);
 *   tol relative tolerance (> 0; the paper uses 1e-6, Sec. 5);
 *   max_iter iteration cap (>= 0); stream cudaStream_t;
 *   x [nz][ny][nx] FP64 (device, written; 0 off fluid);
 *   iters (host, written) network applications performed;
 *   rel_residual (host, written) FP64 ||b - A x|| / ||b|| of the returned x.
 * Each dimension must be divisible by 2^(L-1).  Returns NPSOLVE_OK,
 * NPSOLVE_NO_CONVERGENCE or NPSOLVE_BREAKDOWN with all outputs written, or an
 * argument/CUDA error with outputs unspecified.
 * With cfg.method = NPSOLVE_METHOD_PCG or _FPCG the same call runs PCG or
 * flexible PCG with the network as preconditioner, z_k = ||r_k|| P_net(I,
 * r_k/||r_k||) (the network is linear in r); n_ortho is then not used.  Their
 * BREAKDOWN also covers rho_k = r_k^T z_k = 0 or non-finite (the network is
 * not symmetric positive definite, so rho_k can vanish).  After a residual
 * replacement both restart with beta = 0. */
int npsolve_solve(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *b, double tol,
                  int max_iter, void *stream, double *x, int *iters, double *rel_residual);

/* npsolve_solve on HOST buffers: labels_host, b_host are copied to the device,
 * the solve runs, and x_host (FP64) is copied back, all inside the call.
 * Pinned (page-locked) host memory gives the fastest copies. */
int npsolve_solve_host(npsolve_t h, const uint8_t *labels_host, int nx, int ny, int nz, const float *b_host,
                       double tol, int max_iter, void *stream, double *x_host, int *iters, double *rel_residual);

/* Per-iteration residual norms ||r_k|| (FP64, k = 0..iters) of the last
 * solve on this handle, copied to `hist_host` (at most `cap` entries).
 * Returns the number of entries written in *count. */
int npsolve_residual_history(npsolve_t h, double *hist_host, int cap, int *count);

/* One evaluation of the network z = P_net(I, r) (Alg. 2): r is zeroed off
 * fluid before use (the reduced vector padded with zeros) and z is written
 * as 0 off fluid.  labels, r (FP32), z (FP32) are device arrays. */
int npsolve_apply_network(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *r, float *z,
                          void *stream);

/* One network evaluation, returning an intermediate of level `level`
 * (1..L) instead of z (for per-level parity checks of Alg. 2):
 *   which = 0 x1^l (CConv1 output), 1 r2^l (interpolated input of CConv2),
 *           2 x2^l (CConv2 output), 3 x^l (combined output), 4 r1^l (CConv1 input).
 * out has (nx>>(l-1))*(ny>>(l-1))*(nz>>(l-1)) FP32 entries (device).
 * c12_host (2 doubles, may be NULL) receives Aff1^l, Aff2^l. */
int npsolve_network_intermediate(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *r,
                                 int level, int which, float *out, double *c12_host, void *stream);

/* The adjoint of npsolve_apply_network: out = P_net^T g = mask_fluid(N^T(mask_fluid(g)))
 * for the network z = mask_fluid(N(mask_fluid(r))) of Alg. 2, which is
 * linear in r (Sec. 4.2): the reverse of Alg. 2 without weight gradients
 * (combinations, CConv^T, trilinear interpolation^T, pooling^T), FP32 on
 * CUDA cores with the per-cell kernels materialised (27 FP32 per cell of
 * each level).  g, out: [nz][ny][nx] FP32 device buffers (out written,
 * 0 off fluid); synchronous on `stream`.  The symmetric variant
 * P_sym,1 = P_net^T P_net of the paper's symmetry analysis (appendix) is
 * npsolve_network_transpose(npsolve_apply_network(r)). */
int npsolve_network_transpose(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *g, float *out,
                              void *stream);

/* The relative asymmetry measure of the paper's symmetry analysis
 * (appendix): S(x, y; I) = |x.P(y) - y.P(x)| / sqrt(|x.P(x)| |y.P(y)|)
 * with P = P_net of this handle (two network applications; FP64 dots of
 * the FP32 vectors).  x, y: [nz][ny][nx] FP32 device buffers; *S (host)
 * written; dots_host (optional, host, 4 doubles) receives x.P(y), x.P(x),
 * y.P(x), y.P(y).  S = 0 when the denominator is 0. */
int npsolve_asymmetry(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *x, const float *y,
                      void *stream, double *S, double *dots_host);

/* q = A d, the masked 7-point Laplacian of Sec. 3.2, FP32 (device arrays). */
int npsolve_apply_laplacian(const uint8_t *labels, int nx, int ny, int nz, const float *d, float *q, void *stream);

/* FP64 relative residual ||b - A x|| / ||b|| over the fluid cells (device
 * arrays; result on the host). */
int npsolve_true_residual(const uint8_t *labels, int nx, int ny, int nz, const float *b, const double *x,
                          double *rel_residual, void *stream);

/* Jacobi-preconditioned CG (M = diag(A) on fluid cells) with the same
 * conventions as npsolve_solve; the same-device comparison solver. */
int npsolve_jacobi_pcg(const uint8_t *labels, int nx, int ny, int nz, const float *b, double tol, int max_iter,
                       void *stream, double *x, int *iters, double *rel_residual);

/* Reverse mode of the network (the hand-written backward of Alg. 2): for the
 * output cotangent gz of z = P_net(I, r), the gradient of <gz, z> with
 * respect to the weights (host, npsolve_weight_count(L) floats, raw blob
 * layout) and, if grad_r != NULL, with respect to r (device, zero off fluid).
 * Intermediates are stored during the forward pass; the per-cell kernels are
 * regenerated from the image for each level of the backward pass. */
int npsolve_network_vjp(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *r, const float *gz,
                        float *grad_w_host, float *grad_r, void *stream);

/* Training loss of Sec. 4.2.3 for one system, Loss = || b - A P_net(I, b) ||_2
 * (b as given, zeroed off fluid), and its weight gradient (host floats, may
 * be NULL). */
int npsolve_loss_grad(npsolve_t h, const uint8_t *labels, int nx, int ny, int nz, const float *b, void *stream,
                      double *loss, float *grad_w_host);

/* One optimisation step on a batch: the mean of the per-system losses of
 * npsolve_loss_grad over `batch` systems (labels[i], b[i] device pointers,
 * dims[3i..3i+2] = nx, ny, nz of system i, each divisible by 2^(L-1)), then
 * an Adam update (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) of the
 * handle's weights.  *loss receives the mean loss before the update.  Train
 * with an FP32-form handle; the Adam state lives in the handle. */
int npsolve_train_step(npsolve_t h, int batch, const uint8_t *const *labels, const int *dims, const float *const *b,
                       float lr, void *stream, double *loss);

/* Training right-hand sides from Ritz vectors (Sec. 4.2.3): m Lanczos steps
 * on the masked Laplacian A of the grid from `start` (device, zeroed off
 * fluid; project out the constant on pure-Neumann components first), with
 * full reorthogonalisation; the k lowest Ritz vectors; `count` random
 * normalised combinations of them (coefficients N(0,1) from a 64-bit
 * Mersenne twister seeded with `seed`) written to out (device, count x n
 * floats, zero off fluid; with k = m, every Ritz vector, the combinations are
 * drawn directly in the Lanczos basis, which has the same distribution).
 * ritz_values_host (may be NULL) receives the k
 * lowest Ritz values.  2 <= m <= 2048, 1 <= k <= m; the basis takes
 * (m + 1) n floats of device memory (13 GB for m = 1600 at 128^3). */
int npsolve_lanczos_rhs(const uint8_t *labels, int nx, int ny, int nz, const float *start, int m, int k, int count,
                        unsigned long long seed, float *out, double *ritz_values_host, void *stream);

/* npsolve_true_residual without any device allocation (the paper has no
 * counterpart; this is a library service).  npsolve_true_residual allocates
 * its reduction scratch on every call; callers that must not allocate device
 * memory where they check a solution -- for example a simulation loop that
 * reserves all GPU memory at start-up and forbids allocation inside a frame,
 * or a plug-in whose host application owns the device memory -- use this
 * variant, which keeps the scratch in a fixed device array inside the library.
 * Same arguments and result as npsolve_true_residual (FP64 ||b - A x|| / ||b||
 * over the fluid cells; labels, b, x device arrays; result on the host).
 * Limits: grids of at most 16,777,216 cells (one 256^3 grid; the array is
 * 128 KB per device, held until the process exits); larger grids return
 * NPSOLVE_BAD_DIMS with a message (npsolve_last_error(NULL)).  All calls on a
 * device share the array and overwrite what they use, so nothing needs
 * clearing, but calls that overlap on the GPU (unordered streams) race on
 * it.  The first call on a device looks the array up with that device
 * current; make it before any stream capture. */
int npsolve_true_residual_noalloc(const uint8_t *labels, int nx, int ny, int nz, const float *b, const double *x,
                                  double *rel_residual, void *stream);

/* Continuous-batching solve server (the serving pattern of the deployment
 * setting; the paper has no serving layer).  Requests are queued as they
 * arrive and admitted to solver slots as slots and HBM budget become free;
 * each slot owns a solver handle (workspace, Krylov state and image pyramid
 * on the device), a non-blocking stream and a worker thread, so solves of
 * different sizes overlap on the GPU.  A slot's reservation against the
 * budget is its measured device footprint (an upper estimate of 256 bytes
 * per cell + 64 MB before its first solve at a size); idle slots keep their
 * workspace and its reservation.  Admission is first-fit in arrival order.
 * Results are identical to a solve of the same request on its own.
 *   npsolve_server_create   config and weights as npsolve_create; hbm_budget_bytes > 0;
 *                           1 <= max_active <= 64 concurrent solves
 *   npsolve_server_submit   queues the solve of labels_host / b_host (host memory; pinned
 *                           memory gives the fastest copies) with x written to x_host
 *                           (host FP64, may be NULL); the three buffers are the caller's
 *                           and must stay valid until the request's result has been read;
 *                           submit and result allocate nothing.  Returns the request id;
 *                           a request larger than the whole budget fails with NPSOLVE_OOM
 *   npsolve_server_poll     ids of requests finished since the last poll (non-blocking)
 *   npsolve_server_result   iterations, FP64 true relative residual, the solve's status,
 *                           the time spent queued and in service (ms); releases the request
 *   npsolve_server_stats    reserved and peak reserved bytes, active and queued requests
 *   npsolve_server_destroy  waits for running solves, drops queued ones, frees everything */
typedef struct npsolve_server *npsolve_server_t;
int npsolve_server_create(const npsolve_config *cfg, const float *weights_host, size_t n_weights,
                          size_t hbm_budget_bytes, int max_active, npsolve_server_t *out);
int npsolve_server_submit(npsolve_server_t s, const uint8_t *labels_host, int nx, int ny, int nz, const float *b_host,
                          double *x_host, double tol, int max_iter, long long *request_id);
int npsolve_server_poll(npsolve_server_t s, long long *ids, int cap, int *count);
int npsolve_server_result(npsolve_server_t s, long long id, int *iters, double *rel_residual, int *solve_status,
                          double *queue_ms, double *service_ms);
int npsolve_server_stats(npsolve_server_t s, size_t *reserved_bytes, size_t *peak_reserved_bytes, int *active,
                         int *queued);
void npsolve_server_destroy(npsolve_server_t s);
const char *npsolve_server_last_error(npsolve_server_t s);

/* Optional per-kernel-class timing of solves on a handle.  While profiling
 * is on, npsolve_solve runs one iteration at a time (no CUDA graph) and
 * records a CUDA event pair on the solve's stream around every launch of each
 * kernel class; the totals accumulate until profiling is switched on again.
 *   npsolve_profile_count()     number of classes
 *   npsolve_profile_name(c)     name of class c ("cconv_l1", "lap_alpha", ...)
 *   npsolve_get_profile(h, ms, launches)  per class: total device ms and the
 *                               number of timed launch groups (host arrays of
 *                               npsolve_profile_count() entries). */
int npsolve_profile_count(void);
/* Number of CUDA kernels this handle has enqueued since it was created
 * (solves, network evaluations; graph replays count their kernels). */
long long npsolve_launch_count(npsolve_t h);
/* Device bytes held by the handle's solve workspace (Krylov state, pyramid,
 * network intermediates, kernel cache, staging buffers). */
size_t npsolve_workspace_bytes(npsolve_t h);
/* Cells of level `level` whose 3x3x3 image window was not uniform in the last
 * setup of the cached path (their kernels are generated and cached; all other
 * cells use the closed form of a uniform window); -1 when not available. */
long long npsolve_mixed_cells(npsolve_t h, int level);
/* Work of the level-1 CConvs in the last solve setup (occupancy-aware
 * sparsity: only the units of 32 x 8 cells x a chunk of planes that have work
 * are processed): which = 0 the CConv1 (cells with fluid within one tile or
 * plane), 1 the CConv2 (units holding fluid).  *cells = level-1 cells of the
 * processed units, *mixed = their mixed-window cells (whose cached kernels are
 * read).  Returns NPSOLVE_BAD_ARG before the first solve on the cached path. */
int npsolve_level1_work(npsolve_t h, int which, long long *cells, long long *mixed);
const char *npsolve_profile_name(int cls);
int npsolve_set_profiling(npsolve_t h, int on);
int npsolve_get_profile(npsolve_t h, double *ms_host, long long *launches_host);

/* Self-test of the tensor-core data path (tcgen05.mma with the A operand in
 * tensor memory and the B operand in shared memory, as used by CConv): one
 * 128 x 32 x 64 BF16 product of exactly representable values, compared with
 * the CUDA-core result.  *max_abs_err (host) receives the largest absolute
 * difference (0 when the path is correct).  Returns NPSOLVE_CUDA_ERROR if the
 * device is not sm_103a or the MMA did not complete within 1 s. */
int npsolve_selftest_tensor_core(double *max_abs_err);

#ifdef __cplusplus
}
#endif

#endif /* NPSOLVE_H */

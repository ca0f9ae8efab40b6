/*
 * purify.h -- C ABI of the GB300 (sm_103a) SDMM-SARA imaging library.
 *
 * The library computes the hot path of PURIFY (Carrillo, McEwen & Wiaux,
 * arXiv:1307.4370): the measurement operator Phi = G F D Z of §5 eq. opmodel
 * and its adjoint, the SARA dictionary of §3.3, the proximity operators of
 * §4.4 eqs. prox1-prox3, the conjugate-gradient x-update of §4.4 and the
 * SDMM iteration of Algorithm 1 for problem eq. delta.  Every numerical step
 * runs in hand-written CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by every call
 * --------------------------------
 * Complex vectors are interleaved float32 pairs (re, im) ("complex64").
 * An image is n x n, row-major; element [r][c] is the pixel at offset
 * l = (r - n/2, c - n/2).  A visibility frequency is a float32 pair
 * (u0, u1) in radians per pixel, u0 paired with the row offset; Phi
 * approximates (1/(2n)) sum_l x_l exp(-i u.l).  The oversampled grid is
 * 2n x 2n; F is the unitary 2-D DFT; G interpolates with a Kaiser-Bessel
 * kernel of J x J cells (J even, 2..8) whose first cell per axis is
 * floor(kappa) - J/2 + 1, kappa = u 2n / (2 pi).
 *
 * SARA coefficients are q planes of n x n complex values, one per basis
 * selected by bases_mask (bit 0 Dirac, bit p Daubechies-p, p = 1..8), in
 * increasing bit order; each wavelet plane holds a periodic orthonormal
 * DWT with `levels` levels in Mallat layout (low-low block top-left).  The
 * dictionary is scaled by 1/sqrt(q) so that Psi Psi^H = I (§4.4 needs a
 * Parseval frame for Q = Phi^H Phi + 2I).
 *
 * Memory and ownership
 * --------------------
 * Unless a parameter says otherwise, every array argument is a DEVICE
 * pointer owned by the caller, on the device that was current when the
 * context was created.  The library never frees caller memory.  A context
 * owns its device scratch (the oversampled grid, the sorted visibility
 * table, reduction buffers); an SDMM state owns its iteration variables.
 * Scalars a call produces on the device are written to caller device
 * pointers (never synchronously returned) unless the name says "host".
 *
 * Streams
 * -------
 * Every call that takes a purify_stream_t enqueues its work on that CUDA
 * stream (a cudaStream_t; NULL = the legacy default stream) and returns
 * without synchronising, except where noted.  Calls that use the same
 * context or state must not overlap on the GPU: they share its scratch.
 *
 * Errors
 * ------
 * Every call returns a purify_status; PURIFY_OK is 0, failures are
 * negative.  Argument checks happen before anything is enqueued; a call
 * that fails an argument check has no effect.  PURIFY_E_CUDA reports an
 * error from the CUDA runtime (launch or allocation), after which the
 * context should be destroyed.  purify_status_string() names each code.
 */
#ifndef PURIFY_H
#define PURIFY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* purify_stream_t; /* same type as cudaStream_t */
typedef struct purify_ctx purify_ctx;
typedef struct purify_sdmm_state purify_sdmm_state;

typedef enum {
  PURIFY_OK = 0,
  PURIFY_E_INVALID_ARG = -1,    /* NULL where an array is required, bad enum */
  PURIFY_E_SIZE = -2,           /* a size outside the supported range */
  PURIFY_E_NOT_DEVICE_PTR = -3, /* an argument that must be device memory is not */
  PURIFY_E_ALLOC = -4,          /* device or host allocation failed */
  PURIFY_E_CUDA = -5,           /* CUDA runtime error (launch, copy) */
  PURIFY_E_TIMEOUT = -6,        /* a bounded device wait gave up */
  PURIFY_E_UNSUPPORTED = -7     /* grid side with a prime factor other than 2, 3 */
} purify_status;

/* Visibility storage formats of the measured data y (SDMM data only). */
/* Interpolation kernel of G (§5): Kaiser-Bessel, or the paper's Gaussian
 * g(t) = exp(-b t^2), b = pi (alpha - 1/2) / (alpha J / 2) with alpha = 2,
 * D dividing by the transform of the untruncated Gaussian. */
typedef enum {
  PURIFY_KERNEL_KB = 0,
  PURIFY_KERNEL_GAUSS = 1
} purify_kernel;

/* Prior of the SDMM problem: SARA (eq. delta, the context's dictionary) or
 * the (weighted) TV of eq. tvproblem with positivity (§3.3, §5, §6 "TV" and
 * "RWTV"). */
typedef enum {
  PURIFY_PRIOR_SARA = 0,
  PURIFY_PRIOR_TV = 1
} purify_prior;

typedef enum {
  PURIFY_VIS_C64 = 0,       /* complex64 */
  PURIFY_VIS_BF16_BLOCK = 1 /* bf16 (re, im) pairs, one float32 scale per 4096 */
} purify_vis_format;

/* Problem description (§3.1 eq. ri4, §5 eq. opmodel, §3.3).
 *   n           image side; N = n*n; a multiple of 2^levels; 2n must factor
 *               as 2^a 3^b with b <= 1; 8 <= n <= 2048.
 *   M           number of visibilities, 1 <= M <= 2^31 - 1.
 *   J           kernel support per axis: 2, 4, 6 or 8.
 *   oversample  must be 2 (§6 uses k = 2; the grid is 2n x 2n).
 *   levels      wavelet levels of each Daubechies basis, 1..6 (4 in §6).
 *   bases_mask  bit 0 Dirac, bit p db_p (p = 1..8); SARA is 0x1FF.
 *   tile        side of the grid tiles that organise G and G^T (a schedule
 *               choice, not part of the method): 0 picks a default from the
 *               grid size; otherwise 8, 16, 32 or 64, at least J and dividing
 *               2n.  The autotuner of the Python package measures the
 *               candidates.
 *   kernel      a purify_kernel (0, the zero-initialised default, is
 *               Kaiser-Bessel).  */
typedef struct {
  int32_t n;
  int64_t M;
  int32_t J;
  int32_t oversample;
  int32_t levels;
  uint32_t bases_mask;
  int32_t tile;
  int32_t kernel;
} purify_desc;

/* Create a context for one u-v coverage (§5: G depends only on the
 * frequencies, so it is set up once).  uv holds M float32 pairs and may be
 * a host or a device pointer; it is read during the call and not kept.
 * Set-up sorts the visibilities by grid tile and builds the tile lists of
 * the gridding adjoint and its stored gather walk (one 32-bit item per
 * visibility and 2 x 2 cell block its footprint meets, about 12 per
 * visibility for J = 6, so ~50 bytes of device memory per visibility besides
 * the grids and tables).  For the grid tiles whose lists are dense it also
 * computes G^T G restricted to them (§5: G^H G precomputed for the CG
 * solve), on the host in double with a pool of threads, and keeps it on the
 * device as float stencils: (2J - 1)^2 values per cell, or about half that
 * when the stencils fit a quarter of L2 (at most 4 (2J - 1)^2 bytes per grid
 * cell of the dense tiles; 200 MB for the 1024 x 1024, M = 2^21 workload).
 * This call synchronises `stream`.  PURIFY_E_SIZE if a gridding work unit
 * does not fit the walk's encoding (not reached for the supported sizes),
 * PURIFY_E_ALLOC if device or host memory runs out.
 * *out receives the context, or NULL on failure. */
int purify_create(purify_ctx** out, const purify_desc* desc, const float* uv,
                  purify_stream_t stream);

/* Release a context and its device memory (synchronises the device). */
void purify_destroy(purify_ctx* ctx);

/* Name of a status code (static string). */
const char* purify_status_string(int status);

/* Description of the last CUDA runtime error that a call made on this host
 * thread reported as PURIFY_E_CUDA ("no CUDA error" if none); a static
 * string. */
const char* purify_last_error(void);

/* Primary beam B of Phi = G F D Z B (§5 eq. opmodel): a real n x n map
 * (N float32, row-major like the image; host or device pointer), copied
 * into the context during the call; NULL restores B = I (every experiment
 * of §6).  Every later Phi, Phi^H, CG and SDMM call of this context applies
 * it; SDMM states, and batches holding one of them, re-capture their
 * iteration graph on their next step.  Do not call it while work of this
 * context is in flight on other streams.  Synchronises `stream`.
 * PURIFY_E_INVALID_ARG for a null context. */
int purify_set_beam(purify_ctx* ctx, const float* beam, purify_stream_t stream);

/* The l2 bound of problem eq. delta for i.i.d. complex Gaussian noise (§6):
 * eps^2 = (2M + 4 sqrt(M)) sigma_n^2 / 2, the mean of the chi^2 distribution
 * with 2M degrees of freedom plus two standard deviations, where
 * sigma_n^2 / 2 is the variance of the real and of the imaginary part of the
 * noise.  Host arithmetic (no device, no context); *eps receives the bound.
 * PURIFY_E_INVALID_ARG for M < 1, sigma_n < 0 or a NULL eps. */
int purify_l2_bound(int64_t M, double sigma_n, double* eps);

/* Sizes of a context: N = n*n, M, q = number of bases, D = q*N. */
int purify_sizes(const purify_ctx* ctx, int64_t* N, int64_t* M, int32_t* q,
                 int64_t* D);

/* y = Phi x (§5 eq. opmodel; B = I unless purify_set_beam gave one): x is N complex64 (device), y is M
 * complex64 (device), visibilities in the order of the uv array given to
 * purify_create. */
int purify_phi(purify_ctx* ctx, const float* x, float* y, purify_stream_t stream);

/* y = Phi x without allocating anything and without a context.  The paper
 * has no counterpart: this is for callers that cannot allocate device memory
 * at the point where they need Phi -- a process whose GPU memory is already
 * reserved in full by another allocator, or a latency-critical loop that
 * cannot afford cudaMalloc and the device synchronisation it implies
 * (purify_create allocates its tables and scratch).  Same arithmetic as
 * purify_phi, visibilities gathered in the given order.
 *   n   image side, 8 <= n <= 256, even, 2n = 2^a 3^b with b <= 1
 *   J   Kaiser-Bessel support: 2, 4, 6 or 8;  M >= 1 visibilities
 *   uv  M float32 pairs, x N = n*n complex64, y M complex64 (all device,
 *       owned by the caller).
 * Scratch: one fixed array (about 3 MiB) in the library's device memory,
 * held by every GPU that loads the library until the process exits.  All
 * calls share it and it keeps the last call's contents: calls that overlap on
 * the GPU race; order them on one stream.  The first call on a device looks
 * up the array's device address with that device current, so make it before
 * any stream capture.  Sizes beyond the limits return PURIFY_E_SIZE (or
 * PURIFY_E_UNSUPPORTED for the grid side). */
int purify_phi_static(int32_t n, int32_t J, int64_t M, const float* uv, const float* x,
                      float* y, purify_stream_t stream);

/* x = Phi^H y = Z^T D F^H G^T y: y is M complex64, x is N complex64. */
int purify_phi_adj(purify_ctx* ctx, const float* y, float* x, purify_stream_t stream);

/* alpha = Psi^H x (§3.3, §4.3 L1 = Psi^H): x is N complex64, alpha is D
 * complex64 (q planes of n x n). */
int purify_sara_analysis(purify_ctx* ctx, const float* x, float* alpha,
                         purify_stream_t stream);

/* x = Psi alpha: alpha is D complex64, x is N complex64. */
int purify_sara_synthesis(purify_ctx* ctx, const float* alpha, float* x,
                          purify_stream_t stream);

/* Weighted complex soft threshold, the prox of gamma ||W .||_1 (§4.4 eq.
 * prox1): out_j = a_j/|a_j| (|a_j| - gamma w_j)^+ (0 where a_j = 0).
 * in, out: `count` complex64 (may alias); w: `count` float32 weights >= 0,
 * or NULL for w = 1. */
int purify_prox_l1_reweighted(purify_ctx* ctx, int64_t count, const float* in,
                              const float* w, float gamma, float* out,
                              purify_stream_t stream);

/* Projection onto the l2 ball B = {r : ||r - y||_2 <= eps} of §4.3 (the
 * formula printed as eq. prox2 is read as this projection):
 * out = y + min(1, eps/||in - y||) (in - y).  in, y, out: `count`
 * complex64 (in and out may alias).  ||in - y|| is accumulated in FP64
 * and written to *norm_out (a device double) when norm_out is not NULL. */
int purify_proj_l2ball(purify_ctx* ctx, int64_t count, const float* in,
                       const float* y, double eps, float* out, double* norm_out,
                       purify_stream_t stream);

/* Projection onto the positive orthant of §4.4 eq. prox3, complex vectors
 * treated as real pairs (§4.1): out = max(Re in, 0) + 0i.  May alias. */
int purify_proj_positive(purify_ctx* ctx, int64_t count, const float* in,
                         float* out, purify_stream_t stream);

/* `iters` conjugate-gradient steps on Q x = b, Q = Phi^H Phi + 2I (§4.4),
 * starting from the x passed in (overwritten with the result).  b and x are
 * N complex64.  Inner products and step sizes are FP64.  When resid_out is
 * not NULL the recurrence residual ||r|| is written there (device double). */
int purify_cg_solve(purify_ctx* ctx, const float* b, float* x, int32_t iters,
                    double* resid_out, purify_stream_t stream);

/* SDMM parameters (§4.4). */
typedef struct {
  int32_t max_iters;  /* T_max per reweighting round */
  int32_t cg_iters;   /* CG steps per x-update */
  int32_t rounds;     /* reweighting rounds (1 = no reweighting) */
  int32_t check_every;/* evaluate the halting test every this many
                         iterations (needs one 48-byte device-to-host copy);
                         0 = never (run exactly max_iters per round) */
  double beta;        /* gamma = beta ||Psi^H Phi^H y||_inf; 1e-3 in §4.4 */
  double xi;          /* bound on the relative change of f1; 1e-3 */
  double tau;         /* tolerance on nu = ||y - Phi x||/eps; 0.1 */
  int32_t use_graph;  /* 1: purify_sdmm_step replays one CUDA graph of the
                         whole iteration (captured at its first call on a
                         private stream); 0: launches kernel by kernel */
} purify_sdmm_params;

/* Defaults of §4.4: T = 300, k = 10, 1 round, no halting checks,
 * beta = xi = 1e-3, tau = 0.1; use_graph = 1. */
void purify_sdmm_default_params(purify_sdmm_params* p);

/* Halting quantities after the last iteration (§4.4). */
typedef struct {
  int64_t iters;      /* SDMM iterations run so far */
  double f1;          /* ||W Psi^H x_hat||_1 */
  double zeta;        /* |f1(t) - f1(t-1)| / |f1(t-1)| (inf while f1(t-1) = 0) */
  double nu;          /* ||y - Phi x_hat|| / eps */
  double gamma;       /* penalty parameter */
  double cg_residual; /* CG recurrence residual of the last x-update */
  double nu_min;      /* distributed form: the smallest block's nu (nu is the
                         largest); equal to nu for a single ball */
} purify_report;

/* Allocate the iteration variables of Algorithm 1 for a context. */
int purify_sdmm_state_create(purify_ctx* ctx, purify_sdmm_state** out);
void purify_sdmm_state_destroy(purify_sdmm_state* st);

/* Load the data: y (M complex64, HOST or DEVICE pointer, in uv order) and
 * eps; resets the state to Algorithm 1 steps 1-3 with x_hat(0) = 0 and
 * weights w = 1, and computes gamma = beta ||Psi^H Phi^H y||_inf. */
int purify_sdmm_init(purify_ctx* ctx, purify_sdmm_state* st, const float* y,
                     double eps, const purify_sdmm_params* params,
                     purify_stream_t stream);

/* Replace the data vector y (HOST or DEVICE pointer) without touching the
 * iteration variables. */
int purify_sdmm_set_data(purify_ctx* ctx, purify_sdmm_state* st, const float* y,
                         purify_stream_t stream);

/* Replace the data vector y (HOST or DEVICE complex64, caller order) and keep
 * it in the state as bf16 (re, im) pairs with one float32 scale per block of
 * 4096 visibilities of the library's internal visibility order:
 * scale_b = max |component| over the block (1 if the block is zero), stored
 * value = round-to-nearest-even bf16 of component / scale_b.  The l2 branch
 * of the SDMM step (the only reader of y) then reads 4 bytes per visibility
 * instead of 8; its norms stay FP64. */
int purify_sdmm_set_data_bf16(purify_ctx* ctx, purify_sdmm_state* st, const float* y,
                              purify_stream_t stream);

/* One SDMM iteration (Algorithm 1 steps 5-9). */
int purify_sdmm_step(purify_ctx* ctx, purify_sdmm_state* st, purify_stream_t stream);

/* Prior of an SDMM state (default PURIFY_PRIOR_SARA).  PURIFY_PRIOR_TV runs
 * Algorithm 1 with L1 = I and f1 = ||W grad x||_1 (isotropic forward
 * differences, zero on the last row and column; W the state's N weights, 1
 * until reweighted by purify_sdmm_reweight with delta / (delta + |grad x_hat|));
 * its prox is `fgp_iters` (1..1000) iterations of Beck & Teboulle's fast
 * gradient projection on the dual (§5), and gamma = beta max |grad Phi^H y|.
 * Call before purify_sdmm_init.  Allocates the prox scratch (7 N complex64)
 * on the context.  PURIFY_E_INVALID_ARG for an unknown prior or iteration
 * count. */
int purify_sdmm_set_prior(purify_ctx* ctx, purify_sdmm_state* st, int32_t prior,
                          int32_t fgp_iters);

/* prox of lambda ||W grad .||_1 (§5): out = argmin 1/2 ||x - in||^2 +
 * lambda ||W grad x||_1 by `iters` FGP iterations (0 returns in).  in, out:
 * N complex64 (device, may not alias); w: N float32 weights > 0 (device) or
 * NULL for W = I; lambda >= 0.  Uses the context's TV scratch (allocated on
 * first use). */
int purify_prox_tv(purify_ctx* ctx, const float* in, const float* w, float lambda,
                   int32_t iters, float* out, purify_stream_t stream);

/* Distributed-block form (§4.5 eqs. blocks, dbp1, dbp2): the visibilities,
 * in the caller's order, are cut into R consecutive blocks y_1 .. y_R with
 * offsets[0] = 0 < offsets[1] < ... < offsets[R] = M (host array of R + 1),
 * and block i must satisfy ||y_i - Phi_i x|| <= eps[i] (host array of R,
 * all > 0) in place of the single ball of purify_sdmm_init.  SDMM then runs
 * with S = R + 2 functions; Q = Phi^H Phi + 2I is unchanged, the data
 * branch projects every block onto its own ball (factors and nu_i in FP64),
 * and the report's nu / nu_min are the largest / smallest nu_i (the halting
 * test of purify_sdmm_solve asks every nu_i to lie in the band).
 * 1 <= R <= 4096; R = 0 (offsets, eps may be NULL) returns to the single
 * ball.  The setting belongs to the state, survives purify_sdmm_init and
 * is not part of purify_sdmm_export.  Synchronises `stream`.
 * PURIFY_E_INVALID_ARG for offsets that are not increasing from 0 to M or a
 * bound that is not positive. */
int purify_sdmm_set_blocks(purify_ctx* ctx, purify_sdmm_state* st, int32_t R,
                           const int64_t* offsets, const double* eps,
                           purify_stream_t stream);

/* Start a new reweighting round (§3.3): w_j = delta / (delta + |alpha_j|),
 * alpha = Psi^H x_hat, delta = max(10^-round ||alpha||_inf,
 * 1e-6 ||alpha||_inf); round >= 1.  Iteration variables carry over. */
int purify_sdmm_reweight(purify_ctx* ctx, purify_sdmm_state* st, int32_t round,
                         purify_stream_t stream);

/* Set the weights directly (D float32, device pointer). */
int purify_sdmm_set_weights(purify_ctx* ctx, purify_sdmm_state* st, const float* w,
                            purify_stream_t stream);

/* Copy x_hat (N complex64) to x_out, a HOST or DEVICE pointer.  A host copy
 * synchronises `stream`. */
int purify_sdmm_get_image(purify_ctx* ctx, purify_sdmm_state* st, float* x_out,
                          purify_stream_t stream);

/* Read the halting quantities (synchronises `stream`). */
int purify_sdmm_get_report(purify_ctx* ctx, purify_sdmm_state* st,
                           purify_report* report, purify_stream_t stream);

/* Run the whole method: init, then `rounds` reweighting rounds of up to
 * max_iters iterations, stopping a round early when check_every > 0 and
 * the halting test of §4.4 holds.  y: HOST or DEVICE; x_out: HOST or
 * DEVICE.  Synchronises `stream` before returning. */
int purify_sdmm_solve(purify_ctx* ctx, const float* y, double eps,
                      const purify_sdmm_params* params, float* x_out,
                      purify_report* report, purify_stream_t stream);

/* Checkpoint / resume: the variables (x_hat, r, p, z1, z2, z3, x1, w and the
 * scalars) as one opaque byte blob.  purify_sdmm_state_bytes gives its size;
 * export writes it to a HOST buffer, import reads one back (same context
 * sizes).  Both synchronise `stream`. */
int purify_sdmm_state_bytes(purify_ctx* ctx, size_t* bytes);
int purify_sdmm_export(purify_ctx* ctx, purify_sdmm_state* st, void* host_buf,
                       size_t bytes, purify_stream_t stream);
int purify_sdmm_import(purify_ctx* ctx, purify_sdmm_state* st, const void* host_buf,
                       size_t bytes, purify_stream_t stream);

/* Batched SDMM: `count` independent problems (eq. delta), each with its own
 * context and state and of any sizes, advanced together.  §4.5 discusses
 * parallel evaluation of SDMM's independent parts; here whole problems run
 * side by side.  One batch iteration is one CUDA graph with one branch per
 * problem (captured at the first step, recaptured when any problem's
 * cg_iters, data format, prior, data blocks, beam or imported state changed
 * since), so the kernels of the problems overlap on the GPU.
 * Contexts and states must be distinct, on one device, and already
 * initialised (purify_sdmm_init).  purify_batch_step runs `iters` iterations
 * of every problem on `stream`; each state can be read as usual afterwards.
 * The batch does not own the contexts or states. */
typedef struct purify_batch purify_batch;
int purify_batch_create(purify_batch** out, purify_ctx* const* ctxs,
                        purify_sdmm_state* const* states, int32_t count);
int purify_batch_step(purify_batch* batch, int32_t iters, purify_stream_t stream);
/* Number of problems and of kernels in one batch iteration (0 before the
 * first step). */
int purify_batch_size(const purify_batch* batch, int32_t* count,
                      int32_t* kernels_per_iteration);
void purify_batch_destroy(purify_batch* batch);

/* ------------------------------------------------------------------------
 * Differentiation of the SDMM iteration (reverse mode, hand-written).
 *
 * One iteration of Algorithm 1 (§4.3-§4.4 with S = 3) for the weighted
 * problem min ||W Psi^H x||_1 s.t. ||y_w - Phi_w x||_2 <= eps, x >= 0, where
 * Phi_w = diag(w) Phi and y_w = w o y fold per-visibility weights into the
 * measurement operator (§5 notes weighting matrices fold into Phi), run
 * forward with a tape and reversed from it:
 *   step 5  x_hat' = k steps of standard CG on Q_w = Phi_w^H Phi_w + 2I from
 *           x0 = x_hat with b = x1 + x2 + x3 (stopping early if <r, r> = 0);
 *   i = 1   a1 = Psi^H x_hat' + z1, r1 = prox1(a1) (eq. prox1, lam = gamma w_j),
 *           z1' = a1 - r1, x1' = Psi (2 r1 - a1);
 *   i = 2   a2 = Phi_w x_hat' + z2, r2 = projection of a2 onto the ball of
 *           radius eps around y_w (eq. prox2, reading c1), z2' = a2 - r2,
 *           x2' = Phi_w^H (2 r2 - a2);
 *   i = 3   a3 = x_hat' + z3, r3 = max(Re a3, 0) (eq. prox3), z3' = a3 - r3,
 *           x3' = 2 r3 - a3.
 * The state is seven DEVICE complex64 arrays in this order: x_hat (N),
 * z1 (D), z2 (M), z3 (N), x1 (N), x2 (N), x3 (N); visibility-indexed arrays
 * (y, w, z2) are in the caller's order of the context's uv.  omega (D
 * float32) are the weights of f1, w (M float32) the visibility weights.
 * Complex entries are treated as real pairs (§4.1): the adjoint of an entry
 * is dL/dRe + i dL/dIm.  The calls synchronise `stream` (the CG step sizes
 * are formed on the host in FP64).  cg_iters is 0..64. */

/* gamma = beta ||Psi^H Phi_w^H y_w||_inf (§4.4's rule for the weighted
 * problem) into *gamma (host).  y, wvis: M entries (device, caller order). */
int purify_diff_penalty(purify_ctx* ctx, const float* y, const float* wvis, double beta, double* gamma,
                        purify_stream_t stream);

/* Bytes of the device tape of one iteration with cg_iters CG steps. */
int purify_diff_tape_bytes(purify_ctx* ctx, int32_t cg_iters, size_t* bytes);

/* Forward: state_out = one iteration of state_in (arrays may not alias), the
 * intermediate vectors and CG step sizes written to `tape` (device memory of
 * purify_diff_tape_bytes bytes, owned by the caller). */
int purify_diff_iteration(purify_ctx* ctx, const float* y, const float* wvis, const float* omega,
                          double gamma, double eps, int32_t cg_iters, const float* const* state_in,
                          float* const* state_out, void* tape, purify_stream_t stream);

/* Vector-Jacobian product of that iteration: given the adjoints of its
 * outputs (bar_out, seven arrays like the state) and the state_in and tape
 * of its forward, writes the adjoints of its inputs to bar_in (seven arrays,
 * distinct from bar_out) and ADDS the weights' adjoints to wvis_bar (M
 * float32) and omega_bar (D float32).  gamma is held constant. */
int purify_diff_iteration_vjp(purify_ctx* ctx, const float* y, const float* wvis, const float* omega,
                              double gamma, double eps, int32_t cg_iters, const float* const* state_in,
                              const void* tape, float* const* bar_out, float* const* bar_in,
                              float* wvis_bar, float* omega_bar, purify_stream_t stream);

/* VJP of the weighted soft threshold of §4.4 eq. prox1, r = a/|a| (|a| - gamma
 * w)^+: abar = J^T rbar, (1 - lam/|a|) rbar + lam/|a|^3 a <a, rbar> where
 * |a| > lam = gamma w, else 0; when wbar is not NULL, wbar += gamma dL/dlam
 * with dL/dlam = -<a, rbar>/|a| (0 where |a| <= lam).  count complex entries;
 * w NULL means w = 1.  All device pointers. */
int purify_vjp_soft_threshold(int64_t count, const float* a, const float* w, float gamma, const float* rbar,
                              float* abar, float* wbar, purify_stream_t stream);

/* VJP of the projection onto the ball ||r - y|| <= eps (§4.3 B, eq. prox2 read
 * as that projection): inside abar = rbar; outside, with d = a - y and c =
 * eps/||d||, abar = c (rbar - d <d, rbar>/||d||^2), and ybar = rbar - abar
 * when ybar is not NULL.  FP64 norms.  Synchronises `stream`. */
int purify_vjp_l2ball(purify_ctx* ctx, int64_t count, const float* a, const float* y, double eps,
                      const float* rbar, float* abar, float* ybar, purify_stream_t stream);

/* VJP of the positivity projection of §4.4 eq. prox3, r = max(Re a, 0) + 0i:
 * abar = (Re rbar where Re a > 0, else 0) + 0i. */
int purify_vjp_positive(int64_t count, const float* a, const float* rbar, float* abar, purify_stream_t stream);

/* Kernel timing (measurement utility; the paper has no counterpart).
 * purify_profile_enable(ctx, 1) makes every later kernel launch of this
 * context record a CUDA event before and after it on its stream;
 * purify_profile_collect synchronises the device, and for each kernel family
 * (in order of first launch) writes its name (NUL-terminated, at most 31
 * characters, into names + 32 * i), its number of launches and its total
 * event-timed milliseconds; at most max_entries entries, the count in
 * *n_entries.  Collecting clears the records; enable(ctx, 0) stops
 * recording.  Events add a little launch overhead: time throughput with
 * profiling off. */
int purify_profile_enable(purify_ctx* ctx, int on);
int purify_profile_collect(purify_ctx* ctx, int32_t max_entries, char* names,
                           int64_t* launches, double* ms, int32_t* n_entries);

/* Number of kernels the library has launched in this process (all
 * contexts), counted on the host at each launch. */
uint64_t purify_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* PURIFY_H */

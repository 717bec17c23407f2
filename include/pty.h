/*
 * pty.h -- C ABI of the GB300 (sm_103a) maximum-likelihood conjugate-gradient
 * ptychography library (libpty).
 *
 * The method is the object reconstruction of Yu et al., "Scalable and accurate multi-GPU
 * based image reconstruction of large-scale ptychography data" (arXiv 2106.07575),
 * section "Inverse problem for ptychography", run on one GPU:
 *   Eq. 1  forward model   |G psi|^2 = |F Q psi|^2 = d
 *          Q: probe p times the P x P patch of the object psi at every scan position
 *          F: 2-D far-field Fourier transform of each exit wave
 *   Eq. 2  ML objective    F(psi) = sum_j |G psi|_j^2 - 2 d_j log|G psi|_j
 *   Eq. 3  gradient        grad F = G^H (G psi - d / (G psi)^*),  G^H = Q^H F^H
 *   Eq. 5  CG update       psi_{m+1} = psi_m + gamma_m eta_m
 *   Eq. 6  Dai-Yuan        eta_m = -g_m + ||g_m||^2 / <eta_{m-1}, g_m - g_{m-1}> eta_{m-1}
 *   Eq. 7  line search     shrink gamma until F(psi + gamma eta) <= F(psi) + gamma t
 *   Algorithm 1            GRAD -> DIR -> LS -> Update per iteration, gamma^(0) = 1, tau = 0.5
 *
 * Conventions (the paper leaves these open; the library fixes them):
 *  - psi is the object transmission, [H][W] complex; positions are integer top-left
 *    corners (row, col) of the P x P patch, 0 <= row <= H-P, 0 <= col <= W-P.
 *  - F is the unitary 2-D DFT (scale 1/P per 2-D transform, kernel exp(-2 pi i k.n / P),
 *    no fftshift), so F^H = F^{-1}.  Detector arrays are in natural DFT order.
 *  - The objective is F_eps = sum |u|^2 - d log(|u|^2 + eps) (0 log(.) := 0 when d = 0),
 *    whose Wirtinger gradient is G^H(u - d u / (|u|^2 + eps)), u = G psi; Eq. 3 is used
 *    literally (derivative with respect to psi^*, no factor 2).
 *  - <a,b> in Eq. 6 is Re sum conj(a) b.  A denominator <= 0 or not finite restarts the
 *    direction with eta = -g.
 *  - Line search: gamma = gamma0; repeat { gamma *= tau; trial } until Eq. 7 holds, at
 *    most max_halvings trials; the first trial is gamma0 * tau.
 *
 * Data types.  Complex arrays are interleaved single precision (re, im) pairs, i.e.
 * `float` pointers to 2*N floats, layout-compatible with CUDA float2 / C float complex.
 * Scalars that are reductions (objective, step length, Dai-Yuan coefficient) are double.
 *
 * Memory.  Every array argument may be a host pointer or a device pointer of the device
 * the context was created on; the library detects which (unified addressing) and copies
 * host arrays through its own staging buffers.  Arguments are read or written only during
 * the call; `data` is read during pty_create only (the library keeps a compact copy of
 * the detector pixels that hold counts).
 *
 * Streams and threads.  Every call orders its device work after the work queued so far on
 * the stream given at creation (a cudaStream_t passed as void*; NULL = the legacy default
 * stream), runs it on the context's own stream, and returns after it completed.  A context must not be used from two host
 * threads at once; distinct contexts are independent.
 *
 * Errors.  Every call returns a pty_status.  No call aborts or throws; after an error
 * pty_last_error() gives a one-line description.  A context stays usable after
 * PTY_ERR_ARG / PTY_ERR_BOUNDS / PTY_STALLED; after PTY_ERR_CUDA it should be destroyed.
 */
#ifndef PTY_H_
#define PTY_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PTY_API __attribute__((visibility("default")))
#else
#define PTY_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PTY_OK = 0,
    PTY_ERR_ARG = 1,         /* bad size, null pointer, unsupported P, bad option */
    PTY_ERR_BOUNDS = 2,      /* a scan position puts the patch outside the object */
    PTY_ERR_NOMEM = 3,       /* device or host allocation failed */
    PTY_ERR_CUDA = 4,        /* a CUDA runtime call failed (message in pty_last_error) */
    PTY_ERR_NONFINITE = 5,   /* measured data holds NaN, Inf or negative values */
    PTY_STALLED = 6,         /* line search found no step within max_halvings trials */
    PTY_ERR_TIMEOUT = 7,     /* a bounded device-side wait gave up */
    PTY_ERR_UNSUPPORTED = 8  /* option or size not supported by this build */
} pty_status;

/* Solver options; pty_default_opts fills Algorithm 1's values. */
typedef struct {
    double gamma0;       /* initial step length of every line search, finite, > 0 (1.0) */
    double tau;          /* shrink factor per trial, 0 < tau < 1 (0.5) */
    double t;            /* Eq. 7 termination constant, finite (0.0) */
    int32_t max_halvings;/* trials per line search before PTY_STALLED, 1 .. 1000 (60) */
    double eps;          /* guard of log and division in the objective, in counts, finite
                            and >= 0 (0.1: with a smaller guard the gradient at dark detector
                            pixels holding counts is too ill-conditioned for single precision) */
    int32_t ls_window;   /* line-search trials evaluated per pass over the data: 4, 8, 16
                            or 32, or 0 (default) for an adaptive search: with dft = 0 the
                            leading trials that a lower bound of the objective change
                            (Jensen's inequality on the concave log, per pattern) rejects are
                            skipped, and the first pass of 6, 8, 16 or 32 trials starts at the
                            first trial the bound cannot reject, sized from the previous
                            iteration; then passes of 32.  The accepted step and the trial
                            count do not depend on it */
    int32_t flags;       /* bit 0: record per-stage GPU time (pty_stage_times); bit 1: no
                            linear form (every GRAD pass runs the forward DFT); bit 2: no
                            certified skip of leading trials (adaptive search only); bit 4:
                            scatter-add with per-thread loads instead of tensor copies; bit 5:
                            the linear GRAD pass zeroes its spectrum tile instead of reading
                            only the slots that hold counts (P <= 128; same results) */
    int32_t tile_config; /* pattern-kernel configuration: -1 (default) = autotune at
                            pty_create (the GRAD and LS passes of every configuration for P are
                            timed on the problem's own data; the choice is cached per problem
                            shape for the process); 0.. = one fixed configuration for P
                            (P=64: 0 one CTA of 256 threads; P=128: 0 one CTA of 512
                            threads, 1 cluster of 2, 2 cluster of 4, 3 one CTA of 1024
                            threads; P=256: 0 cluster of 8, 1 cluster of 4) */
    int32_t dft;         /* 2-D DFTs: 0 (default) FP32 FFT on the CUDA cores; 1 batched complex
                            GEMMs on the tensor cores with operands split into BF16 hi + lo and
                            FP32 accumulation; 2 the same with FP16 hi + lo.  1 needs
                            P = 64, 128 or 256, 2 needs P = 64 or 128; pty_adjoint needs 0. */
    int32_t estimator;   /* 0 (default): the Poisson maximum-likelihood objective of Eq. 2;
                            1: the Gaussian least-squares estimator that the paper names beside
                            it, on amplitudes: F = sum |G psi|^2 - 2 sqrt(d) sqrt(|G psi|^2 +
                            eps) + d, i.e. sum (|G psi| - sqrt d)^2 at eps = 0, gradient
                            G^H(G psi - sqrt(d) G psi / sqrt(|G psi|^2 + eps)).  1 needs dft = 0
                            and runs the line search without the certified skip */
    int32_t solver;      /* 0 (default): conjugate gradients with the Dai-Yuan direction and
                            the backtracking line search (Eq. 5-7, Algorithm 1); 1: gradient
                            descent with the constant step gd_step (Eq. 4): no line search,
                            every GRAD pass runs the forward DFT; needs dft = 0 */
    double gd_step;      /* step gamma of Eq. 4 (solver = 1), > 0 */
    int32_t ls_warm;     /* 1: warm-started line search (solver 0, dft 0): after the first
                            accepted step of the context's CG state (pty_cg_reset clears it)
                            the search starts at min(gamma0, gamma_prev / tau), so that its
                            first trial is the previous accepted step; trials stay gamma0 tau^k
                            and max_halvings counts the trials of each search.  The paper
                            leaves the initial step of Eq. 7's search free; Algorithm 1 starts
                            every search at gamma0 (0, default) */
} pty_opts;

typedef struct pty_ctx pty_ctx;

/* Per-iteration record of pty_cg_solve.  Each array pointer is host memory or NULL.
 *   F[niter+1]      F(psi_m) for m = 0..iters_done (the last entry is F of the final psi)
 *   gamma[niter]    accepted step length gamma_m
 *   halvings[niter] line-search trials used in iteration m (0 for gradient descent)
 *   alpha[niter]    Dai-Yuan coefficient of Eq. 6 (0 for the first iteration or a restart)
 * iters_done counts the iterations whose step was accepted. */
typedef struct {
    double *F;
    double *gamma;
    int32_t *halvings;
    double *alpha;
    int32_t iters_done;
} pty_cg_report;

/* Fill *o with the defaults listed in pty_opts. */
PTY_API void pty_default_opts(pty_opts *o);

/*
 * Create a context for one reconstruction problem (the inputs of Algorithm 1).
 *   out    receives the context; *out is NULL on failure.
 *   H, W   object height and width, P <= H, P <= W.
 *   P      probe / detector size; 64, 128 or 256.
 *   probe  [P][P] complex, copied.
 *   K      number of scan positions, >= 1.
 *   pos    [K][2] int32 (row, col) top-left corners, copied.
 *   data   [K][P][P] float32 measured intensities, natural DFT order, finite and >= 0;
 *          read during the call only.
 *   opts   options, or NULL for the defaults.
 *   stream cudaStream_t (as void*) on which all work of the context runs.
 * The current CUDA device at the call is the context's device.
 * Errors: PTY_ERR_ARG, PTY_ERR_BOUNDS, PTY_ERR_NONFINITE, PTY_ERR_NOMEM, PTY_ERR_CUDA.
 */
PTY_API int pty_create(pty_ctx **out, int32_t H, int32_t W, int32_t P, const float *probe, int32_t K,
               const int32_t *pos, const float *data, const pty_opts *opts, void *stream);

/*
 * Create a context whose scan positions may have a fractional part.  The paper's scan
 * positions are float32 inputs of Algorithm 1 (section "Inverse problem for ptychography");
 * how a fraction enters Q is not stated there.  The library takes position s = (row, col)
 * as the P x P window starting at floor(s) and moves the probe inside that window by the
 * fraction delta = s - floor(s) with the Fourier shift theorem:
 *   p_delta = F^H[ F[p](ky, kx) exp(-2 pi i (ky dy + kx dx) / P) ]
 * at the signed frequencies -P/2 < k < P/2, with the factor cos(pi d) at the Nyquist index
 * P/2 of each axis (a real probe stays real).  Q of Eq. 1 then multiplies patch k with its
 * own probe p_delta_k; everything else is as for pty_create.  An integer position gives
 * exactly the unshifted probe.  The shifted probe wraps around its window (a probe that has
 * decayed at the window's edge loses nothing).
 *   pos    [K][2] float32 (row, col), finite; 0 <= floor(row) <= H-P, 0 <= floor(col) <= W-P;
 *          copied.
 *   other arguments as in pty_create.
 * The context holds K probes ([K][P][P] complex, device memory).  One view only; opts.dft
 * must be 0.
 * Errors: as pty_create; PTY_ERR_BOUNDS also for a non-finite coordinate;
 * PTY_ERR_UNSUPPORTED for opts.dft != 0.
 */
PTY_API int pty_create_subpixel(pty_ctx **out, int32_t H, int32_t W, int32_t P, const float *probe, int32_t K,
                                const float *pos, const float *data, const pty_opts *opts, void *stream);

/* Release every resource of the context (NULL is ignored). */
PTY_API void pty_destroy(pty_ctx *ctx);

/* Description of the last error on this context, or with ctx NULL of the last failed call
 * without a usable context (pty_create, pty_batch_create, a NULL ctx) on the calling thread.
 * The string lives until the next call on the same context (or on the same thread). */
PTY_API const char *pty_last_error(const pty_ctx *ctx);

/*
 * Forward model, Eq. 1: out[k] = F(p * patch_k(psi)), unitary F, for every position k
 * in the caller's order.  psi [H][W] complex, out [K][P][P] complex.
 * Errors: PTY_ERR_ARG (NULL ctx or array), PTY_ERR_UNSUPPORTED (batch context),
 * PTY_ERR_NOMEM (staging of host arrays), PTY_ERR_TIMEOUT (dft = 1, 2: a bounded device
 * wait gave up), PTY_ERR_CUDA.
 */
PTY_API int pty_forward(pty_ctx *ctx, const float *psi, float *out);

/*
 * Adjoint of the forward model, the G^H of Eq. 3: x = sum_k shift_k(conj(p) * F^H y_k).
 * y [K][P][P] complex (natural DFT order), x [H][W] complex.  The scatter-add of
 * overlapping patches is summed in a fixed order: results are bitwise reproducible.
 * Errors: PTY_ERR_ARG, PTY_ERR_UNSUPPORTED (batch context, or dft != 0), PTY_ERR_NOMEM,
 * PTY_ERR_TIMEOUT (a bounded wait of the tensor-copy scatter-add gave up), PTY_ERR_CUDA.
 */
PTY_API int pty_adjoint(pty_ctx *ctx, const float *y, float *x);

/*
 * Objective and gradient, Eq. 2 and 3, at psi.  grad [H][W] complex (may be NULL to get
 * only the objective); F receives the objective (may be NULL).  Bitwise reproducible.
 * Errors: PTY_ERR_ARG (NULL ctx or psi), PTY_ERR_UNSUPPORTED (batch context),
 * PTY_ERR_NOMEM, PTY_ERR_TIMEOUT, PTY_ERR_CUDA.
 */
PTY_API int pty_gradient(pty_ctx *ctx, const float *psi, float *grad, double *F);

/*
 * niter iterations of ML-CG (Eq. 5-7, Algorithm 1 on one GPU) updating psi_inout
 * ([H][W] complex) in place.  The conjugate-gradient state (previous gradient and
 * direction) persists in the context, so consecutive calls continue one solve; the
 * first call after pty_create or pty_cg_reset starts with eta_0 = -g_0.
 * rep may be NULL.  Returns PTY_OK, or PTY_STALLED when an iteration found no step
 * (psi then holds the last accepted iterate and rep->iters_done says how many were
 * accepted).  The iteration runs without host synchronisation between its stages; it is
 * captured once as a CUDA graph and replayed (unless opts.flags bit 0 asks for per-stage
 * timing).  Needs a single-view context.
 * Errors: PTY_ERR_ARG (NULL ctx or psi, niter < 0), PTY_ERR_UNSUPPORTED (batch context),
 * PTY_ERR_NOMEM, PTY_ERR_TIMEOUT (a bounded device wait gave up), PTY_ERR_CUDA.
 * Linear form (FFT path, opts.dft = 0): Eq. 1 is linear in psi, so after an accepted step
 * G psi_{m+1} = G psi_m + gamma G eta_m; the model G psi at the detector pixels with counts
 * is then updated in place from the line search's G eta instead of by a forward DFT, and
 * the gradient's dense part conj(p) F^H G psi = |p|^2 psi is summed over positions in the
 * object domain.  A full forward pass runs at the first iteration of a call whose object
 * differs from the one the previous call returned (64-bit hash), after pty_gradient on the
 * context, and every 64th iteration (by the count since the last reset).
 */
PTY_API int pty_cg_solve(pty_ctx *ctx, float *psi_inout, int32_t niter, pty_cg_report *rep);

/*
 * Batched form: n_views independent reconstructions (for instance the views of a
 * tomographic series) of uneven object size and scan count, sharing one probe.  Every
 * stage of an iteration is one launch over all views' patterns; the views' scalars (step,
 * Dai-Yuan coefficient, objective, line-search window, stall) stay separate, so each view
 * follows exactly the iteration it would follow alone.
 *   H, W, K  [n_views] object sizes and scan counts.
 *   pos      [sum K][2] positions, view after view, in each view's own coordinates.
 *   data     [sum K][P][P] measured intensities, view after view.
 *   probe, P, opts, stream as in pty_create.
 * pty_forward, pty_adjoint, pty_gradient and pty_cg_solve need a single-view context;
 * a batch is solved with pty_batch_cg_solve.
 */
PTY_API int pty_batch_create(pty_ctx **out, int32_t n_views, const int32_t *H, const int32_t *W,
                             const int32_t *K, int32_t P, const float *probe, const int32_t *pos,
                             const float *data, const pty_opts *opts, void *stream);

/*
 * niter iterations of every view of a batch.  psi: host array of n_views pointers, each
 * to that view's [H_v][W_v] complex object (host or device memory), updated in place.
 * reps: host array of n_views reports, or NULL.  Returns PTY_STALLED if any view stalled
 * (that view keeps its last accepted iterate; the others complete their iterations).
 * Errors as pty_cg_solve (PTY_ERR_ARG also for a NULL psi[v]).
 */
PTY_API int pty_batch_cg_solve(pty_ctx *ctx, float *const *psi, int32_t niter, pty_cg_report *reps);

/* Number of views of a context (1 for pty_create). */
PTY_API int32_t pty_num_views(const pty_ctx *ctx);

/* Forget the conjugate-gradient state: the next pty_cg_solve starts with eta = -g.
 * Errors: PTY_ERR_ARG (NULL ctx), PTY_ERR_CUDA. */
PTY_API int pty_cg_reset(pty_ctx *ctx);

/*
 * Checkpoint of the conjugate-gradient state (previous gradient and direction, the
 * iteration count and the last step, and the model values kept at the detector pixels
 * with counts): pty_cg_state_size bytes of host memory.  pty_cg_state_load restores it
 * into a context of the same problem (PTY_ERR_ARG if the sizes differ); a solve resumed
 * from a checkpoint with the object the saved solve returned reproduces the uninterrupted
 * solve bit for bit.
 */
PTY_API size_t pty_cg_state_size(const pty_ctx *ctx);
PTY_API int pty_cg_state_save(pty_ctx *ctx, void *host_buf);
PTY_API int pty_cg_state_load(pty_ctx *ctx, const void *host_buf);

/*
 * The pattern-kernel plan of the context: plan[0], plan[1] = rows per CTA and threads per
 * CTA of the GRAD pass; plan[2], plan[3] = the same for the LS pass (a pattern is shared by
 * P / rows CTAs of one thread-block cluster).
 */
PTY_API int pty_get_plan(const pty_ctx *ctx, int32_t plan[4]);

/*
 * Per-stage GPU time accumulated since the last reset (needs opts.flags bit 0):
 * ms[0] GRAD pattern pass (full or linear form), ms[1] scatter-add + direction reductions,
 * ms[2] LS pattern pass (v = G eta), ms[3] small kernels (Dai-Yuan scalars, search
 * direction, line-search decisions, update), ms[4] line-search candidate windows;
 * launches[i] the matching launch counts.  Either pointer may be NULL.  reset != 0 clears
 * the counters after reading.
 */
PTY_API int pty_stage_times(pty_ctx *ctx, double ms[5], int64_t launches[5], int reset);

/*
 * Objective and gradient (as pty_gradient) without a context and without allocating any
 * memory.  The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory -- code running inside another framework's fixed memory budget,
 * a plug-in that must not grow the process's device footprint, or a path that must not
 * take the implicit device synchronisation of cudaMalloc/cudaFree.
 *   H, W, P, K   as in pty_create; P is 64 or 128; K <= 16384 and K*P*P <= 4194304.
 *   probe, pos, data, psi   device pointers, layouts as in pty_create / pty_gradient
 *                (data is the dense [K][P][P] array; positions in any order); probe, pos,
 *                psi, grad and F must be 8-byte aligned (they are read as pairs).
 *   eps          the objective's guard (pty_opts.eps), finite and >= 0.
 *   grad         device [H][W] complex output; F: device double output or NULL.
 *   stream       cudaStream_t (as void*) of the current device, on which the work runs.
 *                The call reads a status flag back and synchronises this stream, so it
 *                cannot be called while the stream is being captured into a CUDA graph.
 * The only scratch is a fixed 32.2 MiB device array inside the library, held on every
 * device where the library's code is loaded until the process exits.  Every call shares
 * it, so calls that overlap on the GPU race; calls ordered on one stream are safe.
 * Returns PTY_OK; PTY_ERR_ARG for a size beyond the limits, a NULL, host or misaligned
 * pointer, or a stream of another device;
 * PTY_ERR_BOUNDS if a position puts the patch outside the object (nothing is written);
 * PTY_ERR_CUDA if a CUDA call failed.
 */
PTY_API int pty_gradient_noalloc(int32_t H, int32_t W, int32_t P, const float *probe, int32_t K,
                                 const int32_t *pos, const float *data, double eps, const float *psi,
                                 float *grad, double *F, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PTY_H_ */

/*
 * pty_cnn.h -- learned initial guess for ML-CG ptychography (part of libpty).
 *
 * The paper starts every reconstruction from a fixed object (Algorithm 1 takes psi_0 as
 * an input); it has no learned component.  This interface adds one in front of
 * pty_cg_solve: a small convolutional network predicts, from each measured diffraction
 * pattern, the object patch under the probe; the patches are stitched into a start
 * object; the objective of Eq. 2 decides whether that start is kept or the plain start
 * (all ones) is used.  The network is trained on the GPU by the library's own kernels,
 * on (pattern, patch) pairs that the forward model of Eq. 1 generates.
 *
 * Network (L layers, C channels, P x P images; this build: C = 32, L >= 2, P = 64, 128
 * or 256):
 *   x     = log(1 + sqrt(d)) with the zero frequency moved to pixel [P/2][P/2]
 *   z_1   = conv3x3(x),  a_l = GELU(z_l) = z_l Phi(z_l),  z_{l+1} = conv3x3(a_l), l < L
 *   z_L   has 2 channels: amplitude 0.8 + 0.2 sigmoid(z_L[0]), phase (pi/2) sigmoid(z_L[1])
 *   o     = amplitude exp(i phase), the predicted patch
 * conv3x3 is a cross-correlation with zero padding:
 *   z[co][y][x] = b[co] + sum_ci sum_{dy,dx = -1..1} W[co][ci][dy+1][dx+1] a[ci][y+dy][x+dx].
 * Training loss of a batch of B pairs (d_b, t_b) with pixel weight w (normally |probe|^2):
 *   loss = sum_b sum_px w |o_b - t_b|^2 / (B sum_px w).
 * Parameters are FP32 master copies (Adam updates them); the convolutions use BF16 copies
 * of the weights (refreshed after every update) with FP32 accumulation; biases stay FP32.
 * Flat parameter layout (pty_cnn_get_params): for l = 1..L, W_l [Cout][Cin][3][3] then
 * b_l [Cout], Cin = 1 for l = 1, Cout = 2 for l = L, C otherwise.
 *
 * Memory: the arrays d, t, o, idx are DEVICE pointers (training sets live on the GPU);
 * params, w and the loss outputs may be host or device pointers where stated.
 * Streams: every call runs on the stream given at creation and returns after it
 * completed.  Errors: pty_status codes of pty.h; pty_cnn_last_error describes the last one.
 */
#ifndef PTY_CNN_H_
#define PTY_CNN_H_

#include "pty.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pty_cnn pty_cnn;

/* Adam (Kingma & Ba 2015, bias-corrected) hyper-parameters. */
typedef struct {
    double lr;    /* step size (1e-3) */
    double beta1; /* first-moment decay (0.9) */
    double beta2; /* second-moment decay (0.999) */
    double eps;   /* denominator guard (1e-8) */
} pty_adam;

/* Outcome of pty_learned_init. */
typedef struct {
    double F_learned;     /* Eq. 2 objective at the stitched network start */
    double F_ones;        /* Eq. 2 objective at the all-ones start */
    int32_t used_learned; /* 1: psi0 is the network start; 0: the ones start was kept */
    double scale;         /* factor c applied to the stitched patches (see pty_learned_init) */
    double ms;            /* wall time of the call (prediction, stitching, both objectives) */
} pty_init_report;

PTY_API void pty_default_adam(pty_adam *a);

/*
 * Create a network.  P: image size (64, 128, 256); channels: C (32); layers: L (>= 2);
 * max_batch: largest batch a call processes at once (calls with more images are run in
 * chunks; training batches must not exceed it).  Weights start at zero: load them with
 * pty_cnn_set_params or pty_cnn_init_params.  The current CUDA device is the network's.
 * Errors: PTY_ERR_ARG, PTY_ERR_UNSUPPORTED (C != 32 or P unsupported), PTY_ERR_NOMEM.
 */
PTY_API int pty_cnn_create(pty_cnn **out, int32_t P, int32_t channels, int32_t layers, int32_t max_batch,
                           void *stream);
PTY_API void pty_cnn_destroy(pty_cnn *net);
PTY_API const char *pty_cnn_last_error(const pty_cnn *net);

/* Number of FP32 parameters (weights and biases of all layers). */
PTY_API int64_t pty_cnn_num_params(const pty_cnn *net);

/* Copy all parameters in (host or device array of pty_cnn_num_params floats); resets the
 * Adam moments and step count.  pty_cnn_get_params copies the FP32 masters out. */
PTY_API int pty_cnn_set_params(pty_cnn *net, const float *params);
PTY_API int pty_cnn_get_params(pty_cnn *net, float *params);

/* He-normal initialisation (weights N(0, 2 / (9 Cin)), biases 0) from a counter-based
 * generator keyed by seed; resets Adam. */
PTY_API int pty_cnn_init_params(pty_cnn *net, uint64_t seed);

/* Pixel weight of the loss, [P][P] floats (host or device); defaults to all ones. */
PTY_API int pty_cnn_set_loss_weight(pty_cnn *net, const float *w);

/*
 * Predict patches: o[b] = network(d[b]) for b < B.  d [B][P][P] counts (natural DFT order),
 * o [B][P][P] complex (interleaved float pairs).  Device pointers.
 */
PTY_API int pty_cnn_predict(pty_cnn *net, int32_t B, const float *d, float *o);

/*
 * Loss and gradient of a batch.  Pair b is (d[idx[b]], t[idx[b]]) (idx: device int32 [B],
 * or NULL for b itself).  d [*][P][P] counts, t [*][P][P] complex target patches.
 * loss: host double or NULL; grad: host or device array of pty_cnn_num_params floats,
 * or NULL.  B <= max_batch.  Deterministic: bitwise reproducible.
 */
PTY_API int pty_cnn_loss_grad(pty_cnn *net, int32_t B, const int32_t *idx, const float *d, const float *t,
                              double *loss, float *grad);

/* One training step: loss_grad, then an Adam update of the masters (adam NULL = defaults). */
PTY_API int pty_cnn_train_step(pty_cnn *net, int32_t B, const int32_t *idx, const float *d, const float *t,
                               const pty_adam *adam, double *loss);

/*
 * Training loop over a pool of n_pairs pairs resident on the device: `steps` steps of
 * `batch` pairs each, drawn without replacement per epoch in an order shuffled by a
 * counter-based generator keyed by seed.  losses: host array of `steps` doubles (the
 * loss of each step's batch before its update) or NULL.
 */
PTY_API int pty_cnn_train(pty_cnn *net, int64_t n_pairs, const float *d, const float *t, int32_t batch,
                          int32_t steps, uint64_t seed, const pty_adam *adam, double *losses);

/*
 * Stitch patch estimates into an object by probe-weighted averaging:
 *   psi0 = sum_k |p|^2 o_k / (sum_k |p|^2 + floor * max_px sum_k |p|^2)
 * over the positions k of a single-view context, with psi0 = 1 where no position
 * reaches.  patches: device [K][P][P] complex in the caller's position order; psi0: host
 * or device [H][W] complex.  Summed over positions in a fixed order (reproducible).
 */
PTY_API int pty_stitch(pty_ctx *ctx, const float *patches, float floor, float *psi0);

/*
 * The learned start of a single-view context: predict every pattern of `d` (device
 * [K][P][P], the context's measured data in the caller's order) with `net` (P must
 * match), stitch with floor 1e-3, and scale the stitched object psi_s by the factor c at
 * which Eq. 2 is stationary along the ray {c psi_s} when eps is neglected,
 *   c^2 = sum d / sum |G psi_s|^2
 * (the denominator by Parseval from the stitch's sum of |p|^2 over positions, no extra
 * forward pass).  Then evaluate Eq. 2 at c psi_s and at the all-ones object, and write the
 * better of the two to psi0 (host or device [H][W] complex).  rep may be NULL.
 */
PTY_API int pty_learned_init(pty_ctx *ctx, pty_cnn *net, const float *d, float *psi0, pty_init_report *rep);

#ifdef __cplusplus
}
#endif

#endif /* PTY_CNN_H_ */

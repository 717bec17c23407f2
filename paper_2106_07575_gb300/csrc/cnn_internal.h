// cnn_internal.h -- kernel launchers of the learned initial guess (not part of the C ABI).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pty_internal.h"

namespace pty {
namespace cnn {

constexpr int kC = 32;  // hidden channels of this build

bool size_supported(int P);

// x[b] = log(1 + sqrt(max(d[src_b], 0))) with the zero frequency moved to [P/2][P/2];
// src_b = idx ? idx[b] : b.
cudaError_t launch_features(int P, int B, const float *d, const int *idx, float *x, cudaStream_t s);

// Hidden 3x3 convolution with kC output channels.  cin = 1 or kC (forward: z = conv + bias,
// a = GELU(z)); cin = 2 or kC (backward-data: out = conv(in; flipped transposed weights) *
// GELU'(zprev)).  w: BF16 [kC][cin][9].
// cin = kC at P = 128, 256 runs on the tensor cores (cnn_tc.cu) unless that form is switched
// off (set_conv_tc); err: device int that a timed-out tensor-core wait sets to 1.
cudaError_t launch_conv_fwd(int P, int cin, int B, const float *in, const __nv_bfloat16 *w, const float *bias,
                            float *z, float *a, int *err, cudaStream_t s);
cudaError_t launch_conv_bwd(int P, int cin, int B, const float *in, const __nv_bfloat16 *wt, const float *zprev,
                            float *out, int *err, cudaStream_t s);
// The tensor-core form of the hidden convolutions (cnn_tc.cu).
bool conv_tc_supported(int P, int cin);
cudaError_t launch_conv_tc(int P, int B, bool bwd, const float *in, const __nv_bfloat16 *w, const float *bias,
                           const float *zprev, float *z, float *a, int *err, cudaStream_t s);
// The tensor-core form of a hidden layer's weight gradient (cnn_tc.cu): the per-CTA partials
// of launch_wgrad for cin = cout = kC at P = 128, 256.
bool wgrad_tc_supported(int P, int cin, int cout);
// Number of partials launch_wgrad_tc writes.
int wgrad_tc_blocks(int P, int B);
cudaError_t launch_wgrad_tc(int P, int B, const float *a, const float *dz, float *part, int *err, cudaStream_t s);
// Process-wide switch of the tensor-core forms (tests compare both forms); on by default.
void set_conv_tc(bool on);
bool conv_tc_on();
// Output layer: z [B][2][P][P] = conv(in [B][kC][P][P]; w [2][kC][9]) + bias.
cudaError_t launch_conv_head(int P, int B, const float *in, const __nv_bfloat16 *w, const float *bias, float *z,
                             cudaStream_t s);
// Head and loss: o = (0.8 + 0.2 s0) exp(i pi/2 s1), s = sigmoid(z).  With t: part[blk] =
// block sums of w |o - t|^2 and dz = d loss / d z with loss scaled by inv_norm.  o_out,
// t may be NULL.  Returns the number of partial sums in *nparts.
cudaError_t launch_head_loss(int P, int B, const float *z, const int *idx, const float2 *t, const float *w,
                             double inv_norm, float2 *o_out, float *dz, double *part, int *nparts,
                             cudaStream_t s);
// loss[0] = inv_norm * sum of n partials (fixed order).
cudaError_t launch_loss_finalize(const double *part, int n, double inv_norm, double *loss, cudaStream_t s);
// Weight and bias gradient of one layer: partials per CTA, then a fixed-order sum into
// grad ([cout][cin][9] then [cout]).  part must hold wgrad_parts(P, B) * (cout*cin*9 + cout).
int wgrad_blocks(int P, int B);
// Partials a weight gradient of either form writes: the size (in units of cout*cin*9 + cout)
// of the part buffer.
int wgrad_part_blocks(int P, int B);
cudaError_t launch_wgrad(int P, int cin, int cout, int B, const float *a, const float *dz, float *part,
                         float *grad, int *err, cudaStream_t s);
// Adam on n masters, then the BF16 copies of every layer's weights are refreshed.
cudaError_t launch_adam(float *master, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, cudaStream_t s);
// w16 = bf16(master weights), wt16[ci][co][8 - tap] = the same (backward-data weights).
cudaError_t launch_refresh(const float *master, int cout, int cin, __nv_bfloat16 *w16, __nv_bfloat16 *wt16,
                           cudaStream_t s);

// Stitching (probe-weighted average of patches) over a single-view context's positions:
// num/den accumulated per object tile, then psi0 = num / (den + floor * max den), 1 where
// den = 0.  patches in the caller's order (perm maps sorted -> caller index).
cudaError_t launch_stitch(int P, const PatternArgs &a, const ScatterPlan &plan, const float2 *patches, float floor,
                          float2 *num, float *den, float *tile_max, float *dmax, float2 *out, cudaStream_t s);
}  // namespace cnn
}  // namespace pty

struct pty_ctx;
namespace pty {
namespace cnn {
// Stitch (as pty_stitch) into the device array out [H][W] and scale it by the factor c at
// which Eq. 2 is stationary along the ray {c psi} when eps is neglected:
// c^2 = sum d / sum |G psi|^2, with sum |G psi|^2 = sum_x |psi(x)|^2 sum_k |p(x - r_k)|^2
// (Parseval, unitary F).  sum_d: device double holding sum d.  c_out: host double (nullable).
int stitch_scaled(pty_ctx *c, const float2 *patches, float floor, const double *sum_d, float2 *out, double *c_out);
// out[0] = scale * sum_i |x_i|^2 w_i (x non-NULL) or scale * sum_i w_i (x NULL), in FP64 in a
// fixed order; part holds kPartials doubles.
constexpr int kPartials = 1024;
cudaError_t launch_sum_sq_weighted(const float2 *x, const float *w, size_t n, double *part, double *out, double scale,
                                   cudaStream_t s);
// x *= c with c = sqrt(num[0] / den[0]) (1 if den[0] <= 0); c_out[0] = c (nullable).
cudaError_t launch_scale_to(float2 *x, size_t n, const double *num, const double *den, double *c_out, cudaStream_t s);
// Fill n complex values with 1.
cudaError_t launch_fill_ones(float2 *x, size_t n, cudaStream_t s);

}  // namespace cnn
}  // namespace pty

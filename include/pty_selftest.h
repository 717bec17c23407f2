/*
 * pty_selftest.h -- device self-tests of libpty's building blocks, for the test suite.
 *
 * These entry points run one device function of the library on caller data so that tests
 * can compare it with a higher-precision reference.  They are not part of the
 * reconstruction method of the paper.
 */
#ifndef PTY_SELFTEST_H_
#define PTY_SELFTEST_H_

#include "pty.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * out[i] = log(1 + t[i]) as computed by the line-search kernels (single precision,
 * within 5 ulp of the exact value for -1 < t < 1e7).  t and out: n floats each, host or
 * device memory (copied as needed); runs on the current device and synchronises.
 * Returns PTY_OK, PTY_ERR_ARG (n < 0 or a NULL pointer with n > 0) or PTY_ERR_CUDA.
 */
PTY_API int pty_selftest_log1p(const float *t, float *out, int32_t n);

/*
 * Failure detection without a fault: every pipeline wait of the tensor-core kernels
 * (opts.dft = 1, 2) and of the tensor-copy scatter-add launched or captured into a context's
 * iteration graph from now on gives up after `polls` polls (polls <= 0 restores the
 * default, about a second per wait).  A kernel whose wait gave up lets its own copies and
 * tensor-core operations finish, frees its tensor memory and returns; the call reports
 * PTY_ERR_TIMEOUT.  Process-wide; for tests.  Returns PTY_OK.
 */
PTY_API int pty_selftest_tc_wait_limit(int64_t polls);

/*
 * *k0cert = the number of leading line-search trials of view `view` that the certificate of
 * the adaptive search (pty_opts.ls_window = 0, dft = 0) rejected without evaluating them in
 * the last iteration of the last pty_cg_solve / pty_batch_cg_solve call on ctx (0 when the
 * certificate is off).  Synchronises ctx's stream.  Returns PTY_OK, PTY_ERR_ARG (NULL ctx
 * or k0cert, view out of range) or PTY_ERR_CUDA.
 */
PTY_API int pty_selftest_ls_certified(pty_ctx *ctx, int32_t view, int32_t *k0cert);

/*
 * Switch the tensor-core form of the learned initial guess's hidden convolutions (tcgen05
 * implicit GEMMs, used at P = 128 and 256) off (enable = 0) or back on (enable != 0, the
 * default), so that tests can compare it with the CUDA-core form.  Process-wide; applies to
 * launches made after the call.  Returns the previous setting (0 or 1).
 */
PTY_API int pty_selftest_cnn_tc(int32_t enable);

#ifdef __cplusplus
}
#endif
#endif /* PTY_SELFTEST_H_ */

// cnn_api.cu -- host side of the learned initial guess (include/pty_cnn.h).
//
// A network owns its FP32 master parameters, the Adam moments, the BF16 working copies of
// the weights (forward layout [Cout][Cin][3][3] and the flipped, transposed layout
// [Cin][Cout][3][3] that the backward-data convolution reads), the loss weight, and the
// activations of one batch of up to max_batch images:
//   x [B][1][P][P], z_l and a_l = GELU(z_l) [B][C][P][P] for l < L-1 (kept for the
//   backward pass), z_{L-1} [B][2][P][P], two [B][C][P][P] buffers for dL/dz, and the
//   per-CTA partials of the weight gradient.
// A training step is one launch sequence on the network's stream: features, L
// convolutions, head+loss, then per layer (last to first) the weight gradient and the
// backward-data convolution (with GELU' fused), then Adam and the BF16 refresh.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cnn_internal.h"
#include "pty_cnn.h"
#include "pty_selftest.h"

struct pty_cnn {
    int dev = 0, P = 0, C = 0, L = 0, Bcap = 0;
    cudaStream_t s = nullptr;
    int64_t nparam = 0;
    std::vector<int> cin, cout;
    std::vector<int64_t> off;   // layer l: weights at off[l], biases at off[l] + cout*cin*9
    std::vector<int64_t> woff;  // layer l: BF16 weights at woff[l]
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16 *w16 = nullptr, *wt16 = nullptr;
    float *lw = nullptr;
    double lw_sum = 0.0;
    int64_t t = 0;
    // batch workspace
    float *x0 = nullptr, *zh = nullptr, *dzh = nullptr, *dz0 = nullptr, *dz1 = nullptr, *part = nullptr;
    std::vector<float *> z, a;
    double *lpart = nullptr, *dloss = nullptr;
    int *tc_err = nullptr;  // set by a timed-out wait of the tensor-core convolutions
    std::string err;
};

namespace {

thread_local std::string g_cnn_create_err;  // last failed call without a network, per thread

int fail(pty_cnn *n, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (n)
        n->err = buf;
    else
        g_cnn_create_err = buf;
    return code;
}

#define CKN(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return fail(n, e_ == cudaErrorMemoryAllocation ? PTY_ERR_NOMEM : PTY_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                \
    } while (0)

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
}

// splitmix64 (Steele, Lea, Flood 2014): the counter-based generator of the initialisation
// and of the training order.
uint64_t splitmix64(uint64_t x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}
double uniform01(uint64_t key) { return ((splitmix64(key) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

struct DevGuard {
    int prev = 0;
    explicit DevGuard(int dev)
    {
        cudaGetDevice(&prev);
        cudaSetDevice(dev);
    }
    ~DevGuard() { cudaSetDevice(prev); }
};

void free_all(pty_cnn *n)
{
    void *ptrs[] = {n->master, n->m, n->v, n->grad, n->w16, n->wt16, n->lw, n->x0, n->zh, n->dzh,
                    n->dz0,    n->dz1, n->part, n->lpart, n->dloss, n->tc_err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (float *p : n->z)
        if (p) cudaFree(p);
    for (float *p : n->a)
        if (p) cudaFree(p);
}

int refresh(pty_cnn *n)
{
    for (int l = 0; l < n->L; l++)
        CKN(pty::cnn::launch_refresh(n->master + n->off[l], n->cout[l], n->cin[l], n->w16 + n->woff[l],
                                     n->wt16 + n->woff[l], n->s));
    return PTY_OK;
}

const float *bias(const pty_cnn *n, int l) { return n->master + n->off[l] + (int64_t)n->cout[l] * n->cin[l] * 9; }

// Forward pass of B <= Bcap images d[idx[b]] (idx may be NULL) into the workspace.
int run_forward(pty_cnn *n, int B, const int *idx, const float *d)
{
    using namespace pty::cnn;
    CKN(launch_features(n->P, B, d, idx, n->x0, n->s));
    const float *in = n->x0;
    for (int l = 0; l < n->L - 1; l++) {
        CKN(launch_conv_fwd(n->P, n->cin[l], B, in, n->w16 + n->woff[l], bias(n, l), n->z[l], n->a[l], n->tc_err,
                            n->s));
        in = n->a[l];
    }
    const int h = n->L - 1;
    CKN(launch_conv_head(n->P, B, in, n->w16 + n->woff[h], bias(n, h), n->zh, n->s));
    return PTY_OK;
}

// Loss (into dloss[0]) and gradient (into n->grad) of a batch.
int run_loss_grad(pty_cnn *n, int B, const int *idx, const float *d, const float2 *t, double *dloss)
{
    using namespace pty::cnn;
    int st;
    if ((st = run_forward(n, B, idx, d))) return st;
    const double inv_norm = 1.0 / ((double)B * n->lw_sum);
    int nparts = 0;
    CKN(launch_head_loss(n->P, B, n->zh, idx, t, n->lw, inv_norm, nullptr, n->dzh, n->lpart, &nparts, n->s));
    CKN(launch_loss_finalize(n->lpart, nparts, 1.0 / n->lw_sum / B, dloss, n->s));
    const int P = n->P, L = n->L;
    // output layer
    CKN(launch_wgrad(P, n->cin[L - 1], 2, B, n->a[L - 2], n->dzh, n->part, n->grad + n->off[L - 1], n->tc_err,
                     n->s));
    float *cur = n->dz0, *other = n->dz1;
    CKN(launch_conv_bwd(P, 2, B, n->dzh, n->wt16 + n->woff[L - 1], n->z[L - 2], cur, n->tc_err, n->s));
    for (int l = L - 2; l >= 1; l--) {
        CKN(launch_wgrad(P, n->cin[l], n->cout[l], B, n->a[l - 1], cur, n->part, n->grad + n->off[l], n->tc_err,
                         n->s));
        CKN(launch_conv_bwd(P, n->cout[l], B, cur, n->wt16 + n->woff[l], n->z[l - 1], other, n->tc_err, n->s));
        std::swap(cur, other);
    }
    CKN(launch_wgrad(P, 1, n->cout[0], B, n->x0, cur, n->part, n->grad + n->off[0], n->tc_err, n->s));
    return PTY_OK;
}

int run_adam(pty_cnn *n, const pty_adam &ad)
{
    n->t++;
    const double bc1 = 1.0 - std::pow(ad.beta1, (double)n->t), bc2 = 1.0 - std::pow(ad.beta2, (double)n->t);
    CKN(pty::cnn::launch_adam(n->master, n->m, n->v, n->grad, n->nparam, (float)ad.lr, (float)ad.beta1,
                              (float)ad.beta2, (float)ad.eps, (float)bc1, (float)bc2, n->s));
    return refresh(n);
}

int check_adam(pty_cnn *n, const pty_adam &ad)
{
    if (!(ad.lr > 0) || !(ad.beta1 >= 0 && ad.beta1 < 1) || !(ad.beta2 >= 0 && ad.beta2 < 1) || !(ad.eps >= 0))
        return fail(n, PTY_ERR_ARG, "bad Adam hyper-parameters");
    return PTY_OK;
}

int reset_adam(pty_cnn *n)
{
    CKN(cudaMemsetAsync(n->m, 0, sizeof(float) * n->nparam, n->s));
    CKN(cudaMemsetAsync(n->v, 0, sizeof(float) * n->nparam, n->s));
    n->t = 0;
    return PTY_OK;
}

// Synchronise the network's stream; a timed-out wait of the tensor-core convolutions since the
// last check is reported (and its flag cleared).
int sync(pty_cnn *n)
{
    CKN(cudaStreamSynchronize(n->s));
    int h = 0;
    CKN(cudaMemcpy(&h, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        CKN(cudaMemset(n->tc_err, 0, sizeof(int)));
        return fail(n, PTY_ERR_TIMEOUT, "a bounded wait of the tensor-core convolutions timed out");
    }
    return PTY_OK;
}

int check_batch(pty_cnn *n, int B, const float *d, const void *t)
{
    if (B < 1 || B > n->Bcap) return fail(n, PTY_ERR_ARG, "batch %d outside [1, %d]", B, n->Bcap);
    if (!d || !t) return fail(n, PTY_ERR_ARG, "d and t must be non-NULL");
    if (!is_device_ptr(d) || !is_device_ptr(t)) return fail(n, PTY_ERR_ARG, "d and t must be device arrays");
    return PTY_OK;
}

}  // namespace

extern "C" {

int pty_selftest_cnn_tc(int32_t enable)
{
    const bool was = pty::cnn::conv_tc_on();
    pty::cnn::set_conv_tc(enable != 0);
    return was ? 1 : 0;
}

void pty_default_adam(pty_adam *a)
{
    if (!a) return;
    a->lr = 1e-3;
    a->beta1 = 0.9;
    a->beta2 = 0.999;
    a->eps = 1e-8;
}

int pty_cnn_create(pty_cnn **out, int32_t P, int32_t channels, int32_t layers, int32_t max_batch, void *stream)
{
    pty_cnn *n = nullptr;
    if (!out) return fail(nullptr, PTY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (layers < 2 || max_batch < 1) return fail(nullptr, PTY_ERR_ARG, "need layers >= 2 and max_batch >= 1");
    if (channels != pty::cnn::kC) return fail(nullptr, PTY_ERR_UNSUPPORTED, "channels must be %d", pty::cnn::kC);
    if (!pty::cnn::size_supported(P)) return fail(nullptr, PTY_ERR_UNSUPPORTED, "P must be 64, 128 or 256");
    n = new (std::nothrow) pty_cnn;
    if (!n) return fail(nullptr, PTY_ERR_NOMEM, "host allocation failed");
    cudaGetDevice(&n->dev);
    n->P = P;
    n->C = channels;
    n->L = layers;
    n->Bcap = max_batch;
    n->s = (cudaStream_t)stream;
    int64_t o = 0, wo = 0;
    for (int l = 0; l < layers; l++) {
        const int ci = l == 0 ? 1 : channels, co = l == layers - 1 ? 2 : channels;
        n->cin.push_back(ci);
        n->cout.push_back(co);
        n->off.push_back(o);
        n->woff.push_back(wo);
        o += (int64_t)co * ci * 9 + co;
        wo += (int64_t)co * ci * 9;
    }
    n->nparam = o;
    const size_t PP = (size_t)P * P, Bc = (size_t)max_batch;
    auto cleanup = [&](int code) {
        int c = fail(nullptr, code, "%s", n->err.empty() ? "device allocation failed" : n->err.c_str());
        free_all(n);
        delete n;
        return c;
    };
    if (dalloc(&n->master, o) || dalloc(&n->m, o) || dalloc(&n->v, o) || dalloc(&n->grad, o) ||
        dalloc(&n->w16, wo) || dalloc(&n->wt16, wo) || dalloc(&n->lw, PP) || dalloc(&n->x0, Bc * PP) ||
        dalloc(&n->zh, Bc * 2 * PP) || dalloc(&n->dzh, Bc * 2 * PP) || dalloc(&n->dz0, Bc * channels * PP) ||
        dalloc(&n->dz1, Bc * channels * PP) ||
        dalloc(&n->part, (size_t)pty::cnn::wgrad_part_blocks(P, max_batch) * (channels * channels * 9 + channels)) ||
        dalloc(&n->lpart, (Bc * PP + 255) / 256) || dalloc(&n->dloss, 1) || dalloc(&n->tc_err, 1)) {
        cudaGetLastError();
        return cleanup(PTY_ERR_NOMEM);
    }
    n->z.assign(layers - 1, nullptr);
    n->a.assign(layers - 1, nullptr);
    for (int l = 0; l < layers - 1; l++)
        if (dalloc(&n->z[l], Bc * channels * PP) || dalloc(&n->a[l], Bc * channels * PP)) {
            cudaGetLastError();
            return cleanup(PTY_ERR_NOMEM);
        }
    std::vector<float> ones(PP, 1.f);
    int st = PTY_OK;
    if (cudaMemcpyAsync(n->lw, ones.data(), sizeof(float) * PP, cudaMemcpyHostToDevice, n->s) != cudaSuccess ||
        cudaMemsetAsync(n->master, 0, sizeof(float) * o, n->s) != cudaSuccess ||
        cudaMemsetAsync(n->tc_err, 0, sizeof(int), n->s) != cudaSuccess)
        st = PTY_ERR_CUDA;
    n->lw_sum = (double)PP;
    if (!st) st = reset_adam(n);
    if (!st) st = refresh(n);
    if (!st) st = sync(n);
    if (st) return cleanup(st);
    *out = n;
    return PTY_OK;
}

void pty_cnn_destroy(pty_cnn *n)
{
    if (!n) return;
    DevGuard g(n->dev);
    cudaStreamSynchronize(n->s);
    free_all(n);
    delete n;
}

const char *pty_cnn_last_error(const pty_cnn *n) { return n ? n->err.c_str() : g_cnn_create_err.c_str(); }

int64_t pty_cnn_num_params(const pty_cnn *n) { return n ? n->nparam : 0; }

int pty_cnn_set_params(pty_cnn *n, const float *params)
{
    if (!n) return fail(nullptr, PTY_ERR_ARG, "net is NULL");
    if (!params) return fail(n, PTY_ERR_ARG, "params is NULL");
    DevGuard g(n->dev);
    CKN(cudaMemcpyAsync(n->master, params, sizeof(float) * n->nparam, cudaMemcpyDefault, n->s));
    int st;
    if ((st = reset_adam(n)) || (st = refresh(n))) return st;
    return sync(n);
}

int pty_cnn_get_params(pty_cnn *n, float *params)
{
    if (!n) return fail(nullptr, PTY_ERR_ARG, "net is NULL");
    if (!params) return fail(n, PTY_ERR_ARG, "params is NULL");
    DevGuard g(n->dev);
    CKN(cudaMemcpyAsync(params, n->master, sizeof(float) * n->nparam, cudaMemcpyDefault, n->s));
    return sync(n);
}

int pty_cnn_init_params(pty_cnn *n, uint64_t seed)
{
    if (!n) return fail(nullptr, PTY_ERR_ARG, "net is NULL");
    std::vector<float> h((size_t)n->nparam, 0.f);
    uint64_t ctr = 0;
    for (int l = 0; l < n->L; l++) {
        const double sd = std::sqrt(2.0 / (9.0 * n->cin[l]));
        const int64_t nw = (int64_t)n->cout[l] * n->cin[l] * 9;
        for (int64_t i = 0; i < nw; i++, ctr += 2) {
            // Box-Muller transform of two uniforms drawn at counters (seed, ctr), (seed, ctr + 1)
            const double u1 = uniform01(seed * 0x9e3779b97f4a7c15ull ^ ctr);
            const double u2 = uniform01(seed * 0x9e3779b97f4a7c15ull ^ (ctr + 1));
            h[n->off[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    return pty_cnn_set_params(n, h.data());
}

int pty_cnn_set_loss_weight(pty_cnn *n, const float *w)
{
    if (!n) return fail(nullptr, PTY_ERR_ARG, "net is NULL");
    if (!w) return fail(n, PTY_ERR_ARG, "w is NULL");
    DevGuard g(n->dev);
    const size_t PP = (size_t)n->P * n->P;
    std::vector<float> h(PP);
    CKN(cudaMemcpy(h.data(), w, sizeof(float) * PP, cudaMemcpyDefault));
    double s = 0.0;
    for (float x : h) {
        if (!(x >= 0.f) || !std::isfinite(x)) return fail(n, PTY_ERR_NONFINITE, "loss weight must be finite and >= 0");
        s += x;
    }
    if (!(s > 0.0)) return fail(n, PTY_ERR_ARG, "loss weight sums to zero");
    CKN(cudaMemcpyAsync(n->lw, h.data(), sizeof(float) * PP, cudaMemcpyHostToDevice, n->s));
    n->lw_sum = s;
    return sync(n);
}

int pty_cnn_predict(pty_cnn *n, int32_t B, const float *d, float *o)
{
    if (!n) return fail(nullptr, PTY_ERR_ARG, "net is NULL");
    if (B < 0 || (B > 0 && (!d || !o))) return fail(n, PTY_ERR_ARG, "bad arguments");
    if (B == 0) return PTY_OK;
    if (!is_device_ptr(d) || !is_device_ptr(o)) return fail(n, PTY_ERR_ARG, "d and o must be device arrays");
    DevGuard g(n->dev);
    const size_t PP = (size_t)n->P * n->P;
    for (int b0 = 0; b0 < B; b0 += n->Bcap) {
        const int nb = std::min(n->Bcap, B - b0);
        int st;
        if ((st = run_forward(n, nb, nullptr, d + (size_t)b0 * PP))) return st;
        CKN(pty::cnn::launch_head_loss(n->P, nb, n->zh, nullptr, nullptr, nullptr, 0.0,
                                       (float2 *)o + (size_t)b0 * PP, nullptr, nullptr, nullptr, n->s));
    }
    return sync(n);
}

int pty_cnn_loss_grad(pty_cnn *n, int32_t B, const int32_t *idx, const float *d, const float *t, double *loss,
                      float *grad)
{
    if (!n) return fail(nullptr, PTY_ERR_ARG, "net is NULL");
    int st;
    if ((st = check_batch(n, B, d, t))) return st;
    DevGuard g(n->dev);
    if ((st = run_loss_grad(n, B, idx, d, (const float2 *)t, n->dloss))) return st;
    double hl = 0.0;
    CKN(cudaMemcpyAsync(&hl, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->s));
    if (grad) CKN(cudaMemcpyAsync(grad, n->grad, sizeof(float) * n->nparam, cudaMemcpyDefault, n->s));
    if ((st = sync(n))) return st;
    if (loss) *loss = hl;
    return PTY_OK;
}

int pty_cnn_train_step(pty_cnn *n, int32_t B, const int32_t *idx, const float *d, const float *t,
                       const pty_adam *adam, double *loss)
{
    if (!n) return fail(nullptr, PTY_ERR_ARG, "net is NULL");
    pty_adam ad;
    pty_default_adam(&ad);
    if (adam) ad = *adam;
    int st;
    if ((st = check_adam(n, ad)) || (st = check_batch(n, B, d, t))) return st;
    DevGuard g(n->dev);
    if ((st = run_loss_grad(n, B, idx, d, (const float2 *)t, n->dloss)) || (st = run_adam(n, ad))) return st;
    double hl = 0.0;
    CKN(cudaMemcpyAsync(&hl, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->s));
    if ((st = sync(n))) return st;
    if (loss) *loss = hl;
    return PTY_OK;
}

int pty_cnn_train(pty_cnn *n, int64_t n_pairs, const float *d, const float *t, int32_t batch, int32_t steps,
                  uint64_t seed, const pty_adam *adam, double *losses)
{
    if (!n) return fail(nullptr, PTY_ERR_ARG, "net is NULL");
    pty_adam ad;
    pty_default_adam(&ad);
    if (adam) ad = *adam;
    int st;
    if ((st = check_adam(n, ad)) || (st = check_batch(n, batch, d, t))) return st;
    if (n_pairs < 1 || n_pairs > INT32_MAX || steps < 0) return fail(n, PTY_ERR_ARG, "bad n_pairs or steps");
    if (steps == 0) return PTY_OK;
    DevGuard g(n->dev);
    // training order: per epoch a Fisher-Yates shuffle driven by splitmix64(seed, epoch, i),
    // epochs concatenated
    const size_t total = (size_t)batch * steps;
    std::vector<int32_t> order;
    order.reserve(total);
    std::vector<int32_t> perm((size_t)n_pairs);
    for (uint64_t epoch = 0; order.size() < total; epoch++) {
        for (int64_t i = 0; i < n_pairs; i++) perm[i] = (int32_t)i;
        for (int64_t i = n_pairs - 1; i > 0; i--) {
            const uint64_t r = splitmix64(seed ^ splitmix64(epoch * 0x100000001b3ull + (uint64_t)i));
            const int64_t j = (int64_t)(r % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        for (int64_t i = 0; i < n_pairs && order.size() < total; i++) order.push_back(perm[i]);
    }
    int32_t *didx = nullptr;
    double *dl = nullptr;
    CKN(dalloc(&didx, total));
    if (cudaError_t e = dalloc(&dl, (size_t)steps)) {
        cudaFree(didx);
        return fail(n, PTY_ERR_NOMEM, "%s", cudaGetErrorString(e));
    }
    st = PTY_OK;
    if (cudaMemcpyAsync(didx, order.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice, n->s) != cudaSuccess)
        st = fail(n, PTY_ERR_CUDA, "index upload failed");
    for (int k = 0; k < steps && !st; k++) {
        st = run_loss_grad(n, batch, didx + (size_t)k * batch, d, (const float2 *)t, dl + k);
        if (!st) st = run_adam(n, ad);
    }
    if (!st && losses &&
        cudaMemcpyAsync(losses, dl, sizeof(double) * steps, cudaMemcpyDeviceToHost, n->s) != cudaSuccess)
        st = fail(n, PTY_ERR_CUDA, "loss download failed");
    if (!st) st = sync(n);
    cudaStreamSynchronize(n->s);
    cudaFree(didx);
    cudaFree(dl);
    return st;
}

int pty_learned_init(pty_ctx *ctx, pty_cnn *n, const float *d, float *psi0, pty_init_report *rep)
{
    if (!n) return fail(nullptr, PTY_ERR_ARG, "net is NULL");
    if (!ctx || !d || !psi0) return fail(n, PTY_ERR_ARG, "ctx, d and psi0 must be non-NULL");
    int H, W, P, K, V, dev;
    pty::ctx_info(ctx, &H, &W, &P, &K, &V, &dev);
    if (V != 1) return fail(n, PTY_ERR_UNSUPPORTED, "pty_learned_init works on single-view contexts");
    if (P != n->P) return fail(n, PTY_ERR_ARG, "network P %d differs from the context's P %d", n->P, P);
    if (dev != n->dev) return fail(n, PTY_ERR_ARG, "network and context are on different devices");
    if (!is_device_ptr(d)) return fail(n, PTY_ERR_ARG, "d must be a device array");
    DevGuard g(n->dev);
    const auto t0 = std::chrono::steady_clock::now();
    const size_t PP = (size_t)P * P, HW = (size_t)H * W;
    float2 *patches = nullptr, *pl = nullptr, *po = nullptr;
    double *red = nullptr;
    CKN(dalloc(&patches, (size_t)K * PP));
    int st = PTY_OK;
    if (dalloc(&pl, HW) || dalloc(&po, HW) || dalloc(&red, (size_t)pty::cnn::kPartials + 1))
        st = fail(n, PTY_ERR_NOMEM, "device allocation failed");
    double Fl = 0.0, Fo = 0.0, scale = 1.0;
    if (!st) st = pty_cnn_predict(n, K, d, (float *)patches);
    // sum of the measured counts, for the scale of the stitched start
    if (!st && (pty::cnn::launch_sum_sq_weighted(nullptr, d, (size_t)K * PP, red, red + pty::cnn::kPartials, 1.0,
                                                 n->s) != cudaSuccess ||
                cudaStreamSynchronize(n->s) != cudaSuccess))
        st = fail(n, PTY_ERR_CUDA, "sum of counts failed");
    if (!st && (st = pty::cnn::stitch_scaled(ctx, patches, 1e-3f, red + pty::cnn::kPartials, pl, &scale)))
        fail(n, st, "stitch: %s", pty_last_error(ctx));
    if (!st && (st = pty_gradient(ctx, (const float *)pl, nullptr, &Fl)))
        fail(n, st, "objective: %s", pty_last_error(ctx));
    if (!st) {
        if (pty::cnn::launch_fill_ones(po, HW, n->s) != cudaSuccess || cudaStreamSynchronize(n->s) != cudaSuccess)
            st = fail(n, PTY_ERR_CUDA, "fill failed");
    }
    if (!st && (st = pty_gradient(ctx, (const float *)po, nullptr, &Fo)))
        fail(n, st, "objective: %s", pty_last_error(ctx));
    const bool use = !st && std::isfinite(Fl) && Fl < Fo;
    if (!st && cudaMemcpy(psi0, use ? pl : po, sizeof(float2) * HW, cudaMemcpyDefault) != cudaSuccess)
        st = fail(n, PTY_ERR_CUDA, "copy of psi0 failed");
    cudaFree(patches);
    if (pl) cudaFree(pl);
    if (po) cudaFree(po);
    if (red) cudaFree(red);
    if (st) return st;
    if (rep) {
        rep->F_learned = Fl;
        rep->F_ones = Fo;
        rep->used_learned = use ? 1 : 0;
        rep->scale = scale;
        rep->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return PTY_OK;
}

}  // extern "C"

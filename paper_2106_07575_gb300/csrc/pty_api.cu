// pty_api.cu -- host side of libpty: the C ABI of include/pty.h.
//
// A context owns the device copies of the probe (pre-scaled by 1/P, the unitary DFT
// normalisation), the twiddle table, the position-sorted scan positions, the object
// tile -> pattern lists of the scatter-add, the conjugate-gradient state and scratch.
// One CG iteration (Algorithm 1 of the paper, single GPU) is a fixed launch sequence:
//   GRAD   k_grad (per pattern) -> k_scatter (per object tile, fused Eq. 6 reductions)
//   DIR    k_dy_finalize (Dai-Yuan coefficient, objective F(psi_m))
//   LS     windows of (k_ls per pattern -> k_ls_decide) until a step is accepted
//   Update k_update
// with every decision taken on the device, so the host only synchronises once per call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "pty.h"
#include "pty_internal.h"

using pty::DevHist;
using pty::DevState;

struct pty_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int H = 0, W = 0, P = 0, K = 0;
    const pty::PatternImpl *impl = nullptr;     // GRAD pass (and forward/adjoint) configuration
    const pty::PatternImpl *impl_ls = nullptr;  // LS pass configuration
    const pty::PatternImpl *impl_nz = nullptr;  // finest column split: the entry layout
    int CS = 1, CSl = 1, nzc = 1, CSmax = 1;
    pty_opts opts{};
    std::string err;

    // problem (device)
    float2 *probe = nullptr;  // [P][P] / P
    float2 *tw = nullptr;     // [P]
    int2 *pos = nullptr;      // [K] sorted
    int *perm = nullptr;      // [K]
    long long *nz_off = nullptr;      // [K * CS + 1]
    unsigned short *nz_slot = nullptr;  // [E]
    float *nz_d = nullptr;            // [E]
    float2 *nz_u = nullptr;           // [E]
    long long n_entries = 0;
    int *tile_start = nullptr, *tile_list = nullptr;
    int ntile_y = 0, ntile_x = 0;

    // CG state and scratch (device)
    float2 *w = nullptr;         // [K][P][P] per-pattern adjoint results
    double *fpart = nullptr;     // [K * CS]
    double *part_sc = nullptr;   // [ntiles][2]
    double *part_ls = nullptr;   // [L+2][K * CS]
    float2 *g = nullptr, *g_prev = nullptr, *eta_prev = nullptr;  // [H][W]
    DevState *st = nullptr;
    double *dscalar = nullptr;
    DevHist hist{};

    // staging for host arguments (device)
    float2 *stage_obj = nullptr, *stage_obj2 = nullptr;
    float2 *stage_pat = nullptr;  // [K][P][P]

    // stage timing
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, std::pair<size_t, size_t>>> ev_marks;
    double stage_ms[4] = {0, 0, 0, 0};
    int64_t stage_n[4] = {0, 0, 0, 0};
};

static std::string g_create_err;

namespace {

int fail(pty_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_err = buf;
    return code;
}

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            return fail(c, e_ == cudaErrorMemoryAllocation ? PTY_ERR_NOMEM : PTY_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                           \
        }                                                                                             \
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
    return cudaMalloc((void **)p, n * sizeof(T) > 0 ? n * sizeof(T) : 1);
}

void free_all(pty_ctx *c)
{
    void *ptrs[] = {c->probe,   c->tw,       c->pos,       c->perm,   c->nz_off,  c->nz_slot, c->nz_d, c->nz_u,
                    c->tile_start, c->tile_list,
                    c->w,       c->fpart,    c->part_sc,   c->part_ls, c->g,         c->g_prev,     c->eta_prev,
                    c->st,      c->dscalar,  c->hist.F,    c->hist.gamma, c->hist.halvings, c->hist.alpha,
                    c->stage_obj, c->stage_obj2, c->stage_pat};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
}

pty::PatternArgs pattern_args(const pty_ctx *c)
{
    pty::PatternArgs a;
    a.H = c->H;
    a.W = c->W;
    a.K = c->K;
    a.probe = c->probe;
    a.tw = c->tw;
    a.pos = c->pos;
    a.perm = c->perm;
    a.nz_off = c->nz_off;
    a.nzc = c->nzc;
    a.nz_slot = c->nz_slot;
    a.nz_d = c->nz_d;
    a.nz_u = c->nz_u;
    a.eps = (float)c->opts.eps;
    return a;
}

pty::ScatterPlan scatter_plan(const pty_ctx *c)
{
    pty::ScatterPlan p;
    p.TY = 32;
    p.TX = 64;
    p.ntile_y = c->ntile_y;
    p.ntile_x = c->ntile_x;
    p.tile_start = c->tile_start;
    p.tile_list = c->tile_list;
    return p;
}

pty::LsArgs ls_args(const pty_ctx *c)
{
    pty::LsArgs l;
    l.gamma0 = c->opts.gamma0;
    l.tau = c->opts.tau;
    l.t = c->opts.t;
    l.max_halvings = c->opts.max_halvings;
    l.adaptive = c->opts.ls_window == 0;
    l.L = l.adaptive ? 32 : c->opts.ls_window;  // capacity of the later windows
    return l;
}

// Device view of a caller array: the pointer itself, or a staging buffer filled from host.
int obj_in(pty_ctx *c, const float *src, float2 *stage, const float2 **out)
{
    if (is_device_ptr(src)) {
        *out = (const float2 *)src;
        return PTY_OK;
    }
    CK(cudaMemcpyAsync(stage, src, sizeof(float2) * (size_t)c->H * c->W, cudaMemcpyHostToDevice, c->stream));
    *out = stage;
    return PTY_OK;
}

int ensure_stage(pty_ctx *c)
{
    if (!c->stage_obj) CK(dalloc(&c->stage_obj, (size_t)c->H * c->W));
    if (!c->stage_obj2) CK(dalloc(&c->stage_obj2, (size_t)c->H * c->W));
    return PTY_OK;
}

int ensure_stage_pat(pty_ctx *c)
{
    if (!c->stage_pat) CK(dalloc(&c->stage_pat, (size_t)c->K * c->P * c->P));
    return PTY_OK;
}

int ensure_hist(pty_ctx *c, int n)
{
    if (c->hist.cap >= n && c->hist.F) return PTY_OK;
    int cap = std::max(n, 64);
    if (c->hist.F) {
        cudaFree(c->hist.F);
        cudaFree(c->hist.gamma);
        cudaFree(c->hist.halvings);
        cudaFree(c->hist.alpha);
        c->hist = DevHist{};
    }
    CK(dalloc(&c->hist.F, (size_t)cap + 1));
    CK(dalloc(&c->hist.gamma, (size_t)cap));
    CK(dalloc(&c->hist.halvings, (size_t)cap));
    CK(dalloc(&c->hist.alpha, (size_t)cap));
    c->hist.cap = cap;
    return PTY_OK;
}

// Stage timing: events around launches when opts.flags & 1.
size_t ev_mark(pty_ctx *c)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
        c->ev_pool.push_back(e);
    }
    size_t i = c->ev_used++;
    cudaEventRecord(c->ev_pool[i], c->stream);
    return i;
}

struct StageTimer {
    pty_ctx *c;
    int stage;
    size_t a = (size_t)-1;
    StageTimer(pty_ctx *c_, int s) : c(c_), stage(s)
    {
        if (c->opts.flags & 1) a = ev_mark(c);
    }
    ~StageTimer()
    {
        if ((c->opts.flags & 1) && a != (size_t)-1) {
            size_t b = ev_mark(c);
            if (b != (size_t)-1) c->ev_marks.push_back({stage, {a, b}});
        }
    }
};

void collect_times(pty_ctx *c)
{
    for (auto &m : c->ev_marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev_pool[m.second.first], c->ev_pool[m.second.second]) == cudaSuccess) {
            c->stage_ms[m.first] += ms;
            c->stage_n[m.first] += 1;
        }
    }
    c->ev_marks.clear();
    c->ev_used = 0;
}

int sync(pty_ctx *c)
{
    CK(cudaStreamSynchronize(c->stream));
    collect_times(c);
    return PTY_OK;
}

// The autotuner: time the GRAD and LS pattern passes of every configuration for P on the
// context's own data (psi = 1, eta = 0, a 16-candidate window) and keep the fastest of
// each.  The choice is cached per problem shape for the life of the process, so contexts of
// the same problem use the same kernels (and give the same bits).
struct PlanKey {
    int P, H, W, K;
    long long nnz;
    bool operator<(const PlanKey &o) const
    {
        return std::tie(P, H, W, K, nnz) < std::tie(o.P, o.H, o.W, o.K, o.nnz);
    }
};
std::mutex g_plan_mu;
std::map<PlanKey, std::pair<int, int>> g_plan_cache;

int autotune(pty_ctx *c)
{
    const pty::PatternImpl *impls = nullptr;
    const int n = pty::pattern_impls(c->P, &impls);
    const PlanKey key{c->P, c->H, c->W, c->K, c->n_entries};
    int best_g = 0, best_l = 0;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_plan_mu);
        auto it = g_plan_cache.find(key);
        if (it != g_plan_cache.end()) {
            best_g = it->second.first;
            best_l = it->second.second;
            cached = true;
        }
    }
    if (!cached && n > 1) {
        int st = ensure_stage(c);
        if (st) return st;
        const size_t HW = (size_t)c->H * c->W;
        std::vector<float2> ones(HW, make_float2(1.f, 0.f));
        CK(cudaMemcpyAsync(c->stage_obj, ones.data(), sizeof(float2) * HW, cudaMemcpyHostToDevice, c->stream));
        DevState hs{};
        hs.Leff = 16;
        hs.Lsel = 16;
        for (int l = 0; l < 16; l++) hs.cand[l] = std::ldexp(1.0, -(l + 1));
        CK(cudaMemcpyAsync(c->st, &hs, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        pty::PatternArgs a = pattern_args(c);
        pty::LsArgs ls = ls_args(c);
        float tg = 1e30f, tl = 1e30f;
        cudaError_t err = cudaSuccess;
        for (int j = 0; j < n && err == cudaSuccess; j++) {
            float ms = 0.f;
            for (int rep = 0; rep < 2 && err == cudaSuccess; rep++) {
                err = cudaEventRecord(e0, c->stream);
                if (err == cudaSuccess) err = impls[j].grad(a, c->stage_obj, c->w, c->fpart, nullptr, c->stream);
                if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            }
            if (err == cudaSuccess && ms < tg) {
                tg = ms;
                best_g = j;
            }
            for (int rep = 0; rep < 2 && err == cudaSuccess; rep++) {
                err = cudaEventRecord(e0, c->stream);
                if (err == cudaSuccess)
                    err = impls[j].ls(a, 16, c->stage_obj, c->g, c->eta_prev, c->part_ls, c->st, c->stream);
                if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            }
            if (err == cudaSuccess && ms < tl) {
                tl = ms;
                best_l = j;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (err != cudaSuccess) return fail(c, PTY_ERR_CUDA, "autotune: %s", cudaGetErrorString(err));
        CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
        CK(cudaStreamSynchronize(c->stream));
        std::lock_guard<std::mutex> lock(g_plan_mu);
        g_plan_cache[key] = {best_g, best_l};
    }
    c->impl = &impls[best_g];
    c->impl_ls = &impls[best_l];
    c->CS = c->P / c->impl->R;
    c->CSl = c->P / c->impl_ls->R;
    return PTY_OK;
}

}  // namespace

extern "C" {

void pty_default_opts(pty_opts *o)
{
    if (!o) return;
    o->gamma0 = 1.0;
    o->tau = 0.5;
    o->t = 0.0;
    o->max_halvings = 60;
    o->eps = 0.1;
    o->ls_window = 0;
    o->flags = 0;
    o->tile_config = -1;
}

const char *pty_last_error(const pty_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

void pty_destroy(pty_ctx *ctx)
{
    if (!ctx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ctx->dev);
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    cudaSetDevice(cur);
    delete ctx;
}

int pty_create(pty_ctx **out, int32_t H, int32_t W, int32_t P, const float *probe, int32_t K, const int32_t *pos,
               const float *data, const pty_opts *opts, void *stream)
{
    pty_ctx *c = nullptr;
    if (!out) return fail(nullptr, PTY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!probe || !pos || !data) return fail(nullptr, PTY_ERR_ARG, "probe, pos and data must be non-NULL");
    if (!pty::pattern_supported(P)) return fail(nullptr, PTY_ERR_ARG, "P=%d not supported (64, 128 or 256)", P);
    if (H < P || W < P) return fail(nullptr, PTY_ERR_ARG, "object %dx%d smaller than probe %d", H, W, P);
    if (K < 1) return fail(nullptr, PTY_ERR_ARG, "K=%d < 1", K);
    if ((int64_t)H * W > (int64_t)1 << 31) return fail(nullptr, PTY_ERR_ARG, "object too large");
    pty_opts o;
    pty_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.tau > 0.0 && o.tau < 1.0) || !(o.gamma0 > 0.0) || o.max_halvings < 1 || o.max_halvings > 1000 ||
        !(o.eps >= 0.0) || !std::isfinite(o.t) || (o.ls_window != 0 && !pty::ls_window_supported(o.ls_window)))
        return fail(nullptr, PTY_ERR_ARG, "invalid options (tau in (0,1), gamma0 > 0, 1 <= max_halvings <= 1000, "
                                          "eps >= 0, ls_window in {0,4,8,16,32})");

    // positions: host copy, bounds check, position sort
    std::vector<int32_t> hpos((size_t)2 * K);
    if (is_device_ptr(pos)) {
        if (cudaMemcpy(hpos.data(), pos, sizeof(int32_t) * 2 * K, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(nullptr, PTY_ERR_CUDA, "cannot read positions");
    } else {
        std::memcpy(hpos.data(), pos, sizeof(int32_t) * 2 * K);
    }
    for (int k = 0; k < K; k++) {
        int r = hpos[2 * k], cc = hpos[2 * k + 1];
        if (r < 0 || cc < 0 || r > H - P || cc > W - P)
            return fail(nullptr, PTY_ERR_BOUNDS, "position %d (%d,%d) puts the %dx%d patch outside %dx%d", k, r, cc, P,
                        P, H, W);
    }

    c = new (std::nothrow) pty_ctx;
    if (!c) return fail(nullptr, PTY_ERR_NOMEM, "host allocation failed");
    cudaGetDevice(&c->dev);
    c->stream = (cudaStream_t)stream;
    c->H = H;
    c->W = W;
    c->P = P;
    c->K = K;
    c->opts = o;
    {
        const pty::PatternImpl *impls = nullptr;
        const int n = pty::pattern_impls(P, &impls);
        if (n == 0 || o.tile_config >= n) {
            delete c;
            return fail(nullptr, PTY_ERR_ARG, "tile_config %d not available for P=%d (%d configurations)",
                        o.tile_config, P, n);
        }
        const int pick = o.tile_config >= 0 ? o.tile_config : 0;
        c->impl = c->impl_ls = &impls[pick];
        c->impl_nz = &impls[0];
        for (int j = 1; j < n; j++)
            if (impls[j].R < c->impl_nz->R) c->impl_nz = &impls[j];
        c->nzc = P / c->impl_nz->R;
        c->CSmax = c->nzc;
        c->CS = c->CSl = P / impls[pick].R;
    }

    auto bail = [&](int code) {
        g_create_err = c->err;
        free_all(c);
        delete c;
        return code;
    };
#define CKC(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return bail(fail(c, e_ == cudaErrorMemoryAllocation ? PTY_ERR_NOMEM : PTY_ERR_CUDA, "%s: %s", #call, \
                             cudaGetErrorString(e_)));                                                     \
    } while (0)

    std::vector<int> perm(K);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
        return hpos[2 * a] != hpos[2 * b] ? hpos[2 * a] < hpos[2 * b] : hpos[2 * a + 1] < hpos[2 * b + 1];
    });
    std::vector<int2> spos(K);
    for (int i = 0; i < K; i++) spos[i] = make_int2(hpos[2 * perm[i]], hpos[2 * perm[i] + 1]);

    // scatter plan: object tiles of 32 x 64, each with the ascending list of overlapping patterns
    const int TY = 32, TX = 64;
    c->ntile_y = (H + TY - 1) / TY;
    c->ntile_x = (W + TX - 1) / TX;
    const int ntiles = c->ntile_y * c->ntile_x;
    std::vector<int> cnt(ntiles + 1, 0);
    for (int i = 0; i < K; i++) {
        int ty0 = spos[i].x / TY, ty1 = (spos[i].x + P - 1) / TY;
        int tx0 = spos[i].y / TX, tx1 = (spos[i].y + P - 1) / TX;
        for (int ty = ty0; ty <= ty1; ty++)
            for (int tx = tx0; tx <= tx1; tx++) cnt[ty * c->ntile_x + tx + 1]++;
    }
    for (int b = 0; b < ntiles; b++) cnt[b + 1] += cnt[b];
    std::vector<int> list(cnt[ntiles]);
    std::vector<int> fillp(cnt.begin(), cnt.end() - 1);
    for (int i = 0; i < K; i++) {
        int ty0 = spos[i].x / TY, ty1 = (spos[i].x + P - 1) / TY;
        int tx0 = spos[i].y / TX, tx1 = (spos[i].y + P - 1) / TX;
        for (int ty = ty0; ty <= ty1; ty++)
            for (int tx = tx0; tx <= tx1; tx++) list[fillp[ty * c->ntile_x + tx]++] = i;
    }

    // probe / P and twiddles exp(-2 pi i m / P), from double precision
    std::vector<float2> hprobe((size_t)P * P), htw(P);
    {
        std::vector<float> raw((size_t)2 * P * P);
        if (is_device_ptr(probe)) {
            if (cudaMemcpy(raw.data(), probe, sizeof(float) * 2 * P * P, cudaMemcpyDeviceToHost) != cudaSuccess)
                return bail(fail(c, PTY_ERR_CUDA, "cannot read probe"));
        } else {
            std::memcpy(raw.data(), probe, sizeof(float) * 2 * P * P);
        }
        for (size_t e = 0; e < (size_t)P * P; e++) {
            if (!std::isfinite(raw[2 * e]) || !std::isfinite(raw[2 * e + 1]))
                return bail(fail(c, PTY_ERR_NONFINITE, "probe holds a non-finite value"));
            hprobe[e] = make_float2(raw[2 * e] / (float)P, raw[2 * e + 1] / (float)P);
        }
        const double pi = 3.14159265358979323846;
        for (int m = 0; m < P; m++) {
            double a = -2.0 * pi * (double)m / (double)P;
            htw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    }

    const size_t PP = (size_t)P * P, HW = (size_t)H * W;
    CKC(dalloc(&c->probe, PP));
    CKC(dalloc(&c->tw, (size_t)P));
    CKC(dalloc(&c->pos, (size_t)K));
    CKC(dalloc(&c->perm, (size_t)K));
    CKC(dalloc(&c->tile_start, (size_t)ntiles + 1));
    CKC(dalloc(&c->tile_list, std::max<size_t>(list.size(), 1)));
    CKC(dalloc(&c->w, (size_t)K * PP));
    CKC(dalloc(&c->fpart, (size_t)K * c->CSmax));
    CKC(dalloc(&c->part_sc, (size_t)ntiles * 2));
    CKC(dalloc(&c->part_ls, (size_t)K * c->CSmax * (32 + 2)));
    CKC(dalloc(&c->g, HW));
    CKC(dalloc(&c->g_prev, HW));
    CKC(dalloc(&c->eta_prev, HW));
    CKC(dalloc(&c->st, (size_t)1));
    CKC(dalloc(&c->dscalar, (size_t)4));
    CKC(cudaMemcpyAsync(c->probe, hprobe.data(), sizeof(float2) * PP, cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemcpyAsync(c->tw, htw.data(), sizeof(float2) * P, cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemcpyAsync(c->pos, spos.data(), sizeof(int2) * K, cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemcpyAsync(c->perm, perm.data(), sizeof(int) * K, cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemcpyAsync(c->tile_start, cnt.data(), sizeof(int) * (ntiles + 1), cudaMemcpyHostToDevice, c->stream));
    if (!list.empty())
        CKC(cudaMemcpyAsync(c->tile_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemsetAsync(c->g_prev, 0, sizeof(float2) * HW, c->stream));
    CKC(cudaMemsetAsync(c->eta_prev, 0, sizeof(float2) * HW, c->stream));
    CKC(cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));

    // measured data: read here only (a host array goes through a temporary device copy)
    // and kept as the compact list of pixels with counts, in tile slot order
    const float *dd = data;
    float *dtmp = nullptr;
    if (!is_device_ptr(data)) {
        CKC(dalloc(&dtmp, (size_t)K * PP));
        CKC(cudaMemcpyAsync(dtmp, data, sizeof(float) * K * PP, cudaMemcpyHostToDevice, c->stream));
        dd = dtmp;
    }
    auto free_tmp = [&]() {
        if (dtmp) cudaFree(dtmp);
        dtmp = nullptr;
    };
    int *flag = (int *)c->dscalar;
    int *dcnt = nullptr;
    const int KC = K * c->nzc;
    std::vector<int> hcnt(KC);
    int hflag = 0;
    cudaError_t ce = cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
    if (ce == cudaSuccess) ce = pty::launch_check_data(dd, (size_t)K * PP, flag, c->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = dalloc(&dcnt, (size_t)KC);
    if (ce == cudaSuccess) ce = c->impl_nz->nz_count(dd, c->perm, K, dcnt, c->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hcnt.data(), dcnt, sizeof(int) * KC, cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (dcnt) cudaFree(dcnt);
    if (ce != cudaSuccess) {
        free_tmp();
        return bail(fail(c, PTY_ERR_CUDA, "data check: %s", cudaGetErrorString(ce)));
    }
    if (hflag) {
        free_tmp();
        return bail(fail(c, PTY_ERR_NONFINITE, "measured data holds NaN, Inf or negative values"));
    }
    std::vector<long long> hoff(KC + 1, 0);
    for (int i = 0; i < KC; i++) hoff[i + 1] = hoff[i] + hcnt[i];
    c->n_entries = hoff[KC];
    const size_t E = (size_t)std::max<long long>(c->n_entries, 1);
    ce = dalloc(&c->nz_off, (size_t)KC + 1);
    if (ce == cudaSuccess) ce = dalloc(&c->nz_slot, E);
    if (ce == cudaSuccess) ce = dalloc(&c->nz_d, E);
    if (ce == cudaSuccess) ce = dalloc(&c->nz_u, E);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(c->nz_off, hoff.data(), sizeof(long long) * (KC + 1), cudaMemcpyHostToDevice, c->stream);
    if (ce == cudaSuccess) ce = c->impl_nz->nz_fill(dd, c->perm, K, c->nz_off, c->nz_slot, c->nz_d, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    free_tmp();
    if (ce != cudaSuccess)
        return bail(fail(c, ce == cudaErrorMemoryAllocation ? PTY_ERR_NOMEM : PTY_ERR_CUDA, "data compaction: %s",
                         cudaGetErrorString(ce)));
#undef CKC
    if (o.tile_config < 0) {
        const int at = autotune(c);
        if (at != PTY_OK) {
            g_create_err = c->err;
            free_all(c);
            delete c;
            return at;
        }
    }
    *out = c;
    return PTY_OK;
}

int pty_forward(pty_ctx *c, const float *psi, float *out)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!psi || !out) return fail(c, PTY_ERR_ARG, "psi and out must be non-NULL");
    int st = ensure_stage(c);
    if (st) return st;
    const float2 *dpsi;
    if ((st = obj_in(c, psi, c->stage_obj, &dpsi))) return st;
    const bool dev_out = is_device_ptr(out);
    if (!dev_out && (st = ensure_stage_pat(c))) return st;
    float2 *dout = dev_out ? (float2 *)out : c->stage_pat;
    CK(c->impl->forward(pattern_args(c), dpsi, dout, c->stream));
    if (!dev_out)
        CK(cudaMemcpyAsync(out, dout, sizeof(float2) * (size_t)c->K * c->P * c->P, cudaMemcpyDeviceToHost,
                           c->stream));
    return sync(c);
}

int pty_adjoint(pty_ctx *c, const float *y, float *x)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!y || !x) return fail(c, PTY_ERR_ARG, "y and x must be non-NULL");
    int st = ensure_stage(c);
    if (st) return st;
    const size_t n = (size_t)c->K * c->P * c->P;
    const float2 *dy = (const float2 *)y;
    if (!is_device_ptr(y)) {
        if ((st = ensure_stage_pat(c))) return st;
        CK(cudaMemcpyAsync(c->stage_pat, y, sizeof(float2) * n, cudaMemcpyHostToDevice, c->stream));
        dy = c->stage_pat;
    }
    const bool dev_x = is_device_ptr(x);
    float2 *dx = dev_x ? (float2 *)x : c->stage_obj;
    pty::PatternArgs a = pattern_args(c);
    CK(c->impl->adjoint(a, dy, c->w, c->stream));
    CK(pty::launch_scatter(c->P, a, scatter_plan(c), c->w, dx, 0, nullptr, nullptr, nullptr, nullptr, c->stream));
    if (!dev_x) CK(cudaMemcpyAsync(x, dx, sizeof(float2) * (size_t)c->H * c->W, cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

int pty_gradient(pty_ctx *c, const float *psi, float *grad, double *F)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!psi) return fail(c, PTY_ERR_ARG, "psi must be non-NULL");
    int st = ensure_stage(c);
    if (st) return st;
    const float2 *dpsi;
    if ((st = obj_in(c, psi, c->stage_obj, &dpsi))) return st;
    pty::PatternArgs a = pattern_args(c);
    CK(c->impl->grad(a, dpsi, c->w, c->fpart, nullptr, c->stream));
    const bool dev_g = grad && is_device_ptr(grad);
    float2 *dg = dev_g ? (float2 *)grad : c->stage_obj2;
    CK(pty::launch_scatter(c->P, a, scatter_plan(c), c->w, dg, 0, nullptr, nullptr, nullptr, nullptr, c->stream));
    CK(pty::launch_sum(c->fpart, c->K * c->CS, c->dscalar, c->stream));
    if (grad && !dev_g)
        CK(cudaMemcpyAsync(grad, dg, sizeof(float2) * (size_t)c->H * c->W, cudaMemcpyDeviceToHost, c->stream));
    double hF = 0.0;
    CK(cudaMemcpyAsync(&hF, c->dscalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((st = sync(c))) return st;
    if (F) *F = hF;
    return PTY_OK;
}

int pty_cg_reset(pty_ctx *c)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    const size_t HW = (size_t)c->H * c->W;
    CK(cudaMemsetAsync(c->g_prev, 0, sizeof(float2) * HW, c->stream));
    CK(cudaMemsetAsync(c->eta_prev, 0, sizeof(float2) * HW, c->stream));
    CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
    return sync(c);
}

int pty_cg_solve(pty_ctx *c, float *psi_inout, int32_t niter, pty_cg_report *rep)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!psi_inout || niter < 0) return fail(c, PTY_ERR_ARG, "psi must be non-NULL and niter >= 0");
    int st = ensure_stage(c);
    if (st) return st;
    if ((st = ensure_hist(c, niter))) return st;
    const size_t HW = (size_t)c->H * c->W;
    const bool dev_psi = is_device_ptr(psi_inout);
    float2 *psi = dev_psi ? (float2 *)psi_inout : c->stage_obj;
    if (!dev_psi) CK(cudaMemcpyAsync(psi, psi_inout, sizeof(float2) * HW, cudaMemcpyHostToDevice, c->stream));

    const pty::PatternArgs a = pattern_args(c);
    const pty::ScatterPlan plan = scatter_plan(c);
    const pty::LsArgs ls = ls_args(c);
    // first window >= 4 candidates when adaptive (then full windows of L), else L each
    const int first = ls.adaptive ? 4 : ls.L;
    const int rest = std::max(0, c->opts.max_halvings - first);
    const int nwin = 1 + (rest + ls.L - 1) / ls.L;
    const int ntiles = c->ntile_x * c->ntile_y;
    CK(pty::launch_begin_solve(c->st, c->stream));
    for (int it = 0; it < niter; it++) {
        {
            StageTimer t(c, 0);
            CK(c->impl->grad(a, psi, c->w, c->fpart, c->st, c->stream));
        }
        {
            StageTimer t(c, 1);
            CK(pty::launch_scatter(c->P, a, plan, c->w, c->g, 1, c->eta_prev, c->g_prev, c->part_sc, c->st,
                                   c->stream));
        }
        {
            StageTimer t(c, 3);
            CK(pty::launch_dy_finalize(c->fpart, c->K * c->CS, c->part_sc, ntiles, c->st, c->hist, ls, c->stream));
        }
        for (int wdx = 0; wdx < nwin; wdx++) {
            {
                StageTimer t(c, 2);
                // the first window of an adaptive search runs on the 16- or the 32-candidate
                // kernel as the device chose; the other one returns at once
                if (wdx == 0 && ls.adaptive)
                    CK(c->impl_ls->ls(a, 16, psi, c->g, c->eta_prev, c->part_ls, c->st, c->stream));
                CK(c->impl_ls->ls(a, ls.L, psi, c->g, c->eta_prev, c->part_ls, c->st, c->stream));
            }
            StageTimer t(c, 3);
            CK(pty::launch_ls_decide(c->part_ls, c->K * c->CSl, ls, c->st, c->hist, c->stream));
        }
        StageTimer t(c, 3);
        CK(pty::launch_update((int)HW, psi, c->g, c->eta_prev, c->g_prev, c->st, c->stream));
    }
    DevState hs;
    CK(cudaMemcpyAsync(&hs, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    if (!dev_psi) CK(cudaMemcpyAsync(psi_inout, psi, sizeof(float2) * HW, cudaMemcpyDeviceToHost, c->stream));
    std::vector<double> hF(niter + 1), hg(std::max(niter, 1)), ha(std::max(niter, 1));
    std::vector<int> hh(std::max(niter, 1));
    if (rep && niter > 0) {
        CK(cudaMemcpyAsync(hF.data(), c->hist.F, sizeof(double) * (niter + 1), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(hg.data(), c->hist.gamma, sizeof(double) * niter, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(ha.data(), c->hist.alpha, sizeof(double) * niter, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(hh.data(), c->hist.halvings, sizeof(int) * niter, cudaMemcpyDeviceToHost, c->stream));
    }
    if ((st = sync(c))) return st;
    if (rep) {
        const int done = hs.m;
        rep->iters_done = done;
        const int nrec = std::min(niter, done + (hs.stalled ? 1 : 0));
        if (rep->F)
            for (int i = 0; i <= std::min(done, niter); i++) rep->F[i] = hF[i];
        for (int i = 0; i < nrec; i++) {
            if (rep->gamma) rep->gamma[i] = hg[i];
            if (rep->alpha) rep->alpha[i] = ha[i];
            if (rep->halvings) rep->halvings[i] = hh[i];
        }
    }
    if (hs.stalled) return fail(c, PTY_STALLED, "line search found no step within %d trials at iteration %d",
                                c->opts.max_halvings, hs.m);
    return PTY_OK;
}

size_t pty_cg_state_size(const pty_ctx *c)
{
    if (!c) return 0;
    return 2 * sizeof(float2) * (size_t)c->H * c->W + sizeof(DevState);
}

int pty_cg_state_save(pty_ctx *c, void *host_buf)
{
    if (!c || !host_buf) return fail(c, PTY_ERR_ARG, "ctx and buffer must be non-NULL");
    const size_t HW = (size_t)c->H * c->W;
    char *b = (char *)host_buf;
    CK(cudaMemcpyAsync(b, c->g_prev, sizeof(float2) * HW, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(b + sizeof(float2) * HW, c->eta_prev, sizeof(float2) * HW, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(b + 2 * sizeof(float2) * HW, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

int pty_cg_state_load(pty_ctx *c, const void *host_buf)
{
    if (!c || !host_buf) return fail(c, PTY_ERR_ARG, "ctx and buffer must be non-NULL");
    const size_t HW = (size_t)c->H * c->W;
    const char *b = (const char *)host_buf;
    DevState hs;
    std::memcpy(&hs, b + 2 * sizeof(float2) * HW, sizeof(DevState));
    hs.m = 0;
    hs.decided = 0;
    hs.stalled = 0;
    CK(cudaMemcpyAsync(c->g_prev, b, sizeof(float2) * HW, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->eta_prev, b + sizeof(float2) * HW, sizeof(float2) * HW, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->st, &hs, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
    return sync(c);
}

int pty_get_plan(const pty_ctx *c, int32_t plan[4])
{
    if (!c || !plan) return fail(nullptr, PTY_ERR_ARG, "ctx and plan must be non-NULL");
    plan[0] = c->impl->R;
    plan[1] = c->impl->NT;
    plan[2] = c->impl_ls->R;
    plan[3] = c->impl_ls->NT;
    return PTY_OK;
}

int pty_stage_times(pty_ctx *c, double ms[4], int64_t launches[4], int reset)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    for (int i = 0; i < 4; i++) {
        if (ms) ms[i] = c->stage_ms[i];
        if (launches) launches[i] = c->stage_n[i];
    }
    if (reset)
        for (int i = 0; i < 4; i++) {
            c->stage_ms[i] = 0;
            c->stage_n[i] = 0;
        }
    return PTY_OK;
}

}  // extern "C"

#include "pty_selftest.h"

extern "C" int pty_selftest_log1p(const float *t, float *out, int32_t n)
{
    pty_ctx *c = nullptr;
    if (n < 0 || (n > 0 && (!t || !out))) return fail(nullptr, PTY_ERR_ARG, "bad arguments");
    if (n == 0) return PTY_OK;
    float *dt = nullptr, *dout = nullptr;
    const bool dev_t = is_device_ptr(t), dev_o = is_device_ptr(out);
    cudaError_t e = cudaSuccess;
    if (!dev_t) e = cudaMalloc(&dt, sizeof(float) * n);
    if (e == cudaSuccess && !dev_o) e = cudaMalloc(&dout, sizeof(float) * n);
    if (e == cudaSuccess && !dev_t) e = cudaMemcpy(dt, t, sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = pty::launch_selftest_log1p(dev_t ? t : dt, dev_o ? out : dout, n, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && !dev_o) e = cudaMemcpy(out, dout, sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (dt) cudaFree(dt);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return fail(c, PTY_ERR_CUDA, "selftest: %s", cudaGetErrorString(e));
    return PTY_OK;
}

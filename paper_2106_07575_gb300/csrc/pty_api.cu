// pty_api.cu -- host side of libpty: the C ABI of include/pty.h.
//
// A context owns the device copies of the probe (pre-scaled by 1/P, the unitary DFT
// normalisation), the twiddle table, the position-sorted scan positions, the compact
// measured data, the object tile -> pattern lists of the scatter-add, the conjugate-
// gradient state and scratch, for one view or for a batch of independent views.  A batch
// is packed into one "atlas" object: view v occupies rows [R0_v, R0_v + H_v) (R0_v a
// multiple of the 32-row scatter tile) and columns [0, W_v) of an array of width max W_v,
// so patterns, scatter tiles and rows of different views never mix and every stage runs
// as one launch over all views.  Scalars of the method (alpha, gamma, F, the line-search
// window, the stall flag) are per view.
//
// One CG iteration (Algorithm 1 of the paper, single GPU) is a fixed launch sequence:
//   GRAD   k_grad (full form) or k_grad_lin (linear form) per pattern -> k_scatter_tma (per
//          object tile, by tensor copies, fused Eq. 6 reductions)
//   DIR    k_dy_finalize (per view: Dai-Yuan coefficient, objective F(psi_m)) -> k_eta
//   LS     k_ls_fft per pattern (G eta at the pixels with counts, certificate rows) ->
//          k_ls_certify -> windows of (k_ls_entries -> k_ls_decide) until a step is accepted
//   Update k_update, k_update_counters
// with every decision taken on the device.  The sequence is captured once as a CUDA graph
// and replayed per iteration; the host synchronises once per call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "cnn_internal.h"
#include "pty.h"
#include "pty_cnn.h"
#include "pty_internal.h"

using pty::DevHist;
using pty::DevState;

struct pty_ctx {
    int dev = 0;
    cudaStream_t user = nullptr;  // the caller's stream
    cudaStream_t s = nullptr;     // the context's own stream (captured into graphs)
    cudaEvent_t join = nullptr;
    int V = 1, P = 0, K = 0;
    int HA = 0, WA = 0;  // atlas rows and width
    std::vector<int> Hv, Wv, Kv, R0, Koff;
    const pty::PatternImpl *impl = nullptr;     // GRAD pass (and forward/adjoint) configuration
    const pty::PatternImpl *impl_ls = nullptr;  // LS pass configuration
    const pty::PatternImpl *impl_nz = nullptr;  // finest column split: the entry layout
    int CS = 1, CSl = 1, nzc = 1, CSmax = 1;
    pty_opts opts{};
    std::string err;

    // problem (device)
    float2 *probe = nullptr;  // [P][P] / P, or [K][P][P] / P with fractional positions
    long long probe_stride = 0;  // 0: one probe; P * P: one per sorted pattern
    float2 *tw = nullptr;     // [P]
    int2 *pos = nullptr;      // [K] sorted, atlas coordinates
    int *perm = nullptr;      // [K] caller index of sorted pattern i
    int *pat_view = nullptr;  // [K]
    int *view_pat_off = nullptr, *view_tile_off = nullptr, *row_view = nullptr, *tile_view = nullptr;
    long long *nz_off = nullptr;        // [K * nzc + 1]
    unsigned short *nz_slot = nullptr;  // [E]
    float *nz_d = nullptr;              // [E]
    float2 *nz_u = nullptr;             // [E]
    float2 *nz_v = nullptr;             // [E]
    long long n_entries = 0;
    unsigned *nz_mask = nullptr;  // entry slots per pattern (PatternArgs::nz_mask), P <= 128
    int *tile_start = nullptr, *tile_list = nullptr;
    int ntile_y = 0, ntile_x = 0;

    // CG state and scratch (device)
    float2 *w = nullptr;        // [K][P][P] per-pattern adjoint results
    alignas(64) unsigned char wmap[128] = {};  // tensor map of w for the tensor-copy scatter-add
    bool wmap_ok = false;
    float2 *fpart = nullptr;    // [K * CS] float-float partial sums
    float2 *part_sc = nullptr;  // [ntiles][3]
    float2 *part_ls = nullptr;  // [L+2][K * CS]
    float2 *psi = nullptr, *g = nullptr, *g_prev = nullptr, *eta_prev = nullptr;  // atlas
    float2 *eta = nullptr;       // atlas: the current search direction (LS stage)
    float *illum = nullptr;      // atlas: sum over positions of |probe / P|^2 (Parseval totals)
    float2 *part_eta = nullptr;  // [ntiles][2] object-tile sums of the LS stage
    float *dsum = nullptr;       // [K * CSl] counts per (pattern, LS chunk): certificate weights
    bool cert = false;           // certified skip of leading line-search trials
    unsigned long long *hash = nullptr;  // [V] object hashes (solve entry / exit)
    bool cache_dirty = false;  // the entries' u no longer belong to the last solve's object
    DevState *st = nullptr;     // [V]
    double *dscalar = nullptr;
    DevHist hist{};
    // pinned host staging of a solve call's results (device state, history, error flag), so
    // that the call copies them back asynchronously and synchronises once
    unsigned char *hpin = nullptr;
    size_t hpin_bytes = 0;

    // staging for host arguments (device)
    float2 *stage_obj = nullptr, *stage_obj2 = nullptr;
    float2 *stage_pat = nullptr;  // [K][P][P]

    // tensor-core DFT form (opts.dft != 0)
    uint8_t *tc_img_fwd = nullptr, *tc_img_inv = nullptr;
    int *tc_err = nullptr;  // a bounded device wait gave up (tensor-core DFT, tensor-copy scatter)
    float2 *tc_x = nullptr, *tc_t = nullptr, *tc_u = nullptr;  // [K][P][P] work buffers
    float2 *tc_pars = nullptr;                                  // [2][K] Parseval sums

    // stitching of patch estimates (pty_stitch)
    float *st_den = nullptr;   // [HA][WA] sum of |p|^2
    float *st_tmax = nullptr;  // [ntiles + 1] per-tile maxima, then the maximum
    double *st_red = nullptr;  // [kPartials + 2] reduction scratch of the scaled stitch

    // one CG iteration as a CUDA graph
    cudaGraphExec_t iter_exec = nullptr;
    bool graph_failed = false;

    // stage timing
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, std::pair<size_t, size_t>>> ev_marks;
    double stage_ms[5] = {0, 0, 0, 0, 0};
    int64_t stage_n[5] = {0, 0, 0, 0, 0};
};

// message of the last failed call without a context, per calling thread
static thread_local std::string g_create_err;

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
    void *ptrs[] = {c->probe,      c->tw,         c->pos,        c->perm,      c->pat_view,     c->view_pat_off,
                    c->view_tile_off, c->row_view, c->tile_view,  c->nz_off,    c->nz_slot,      c->nz_d, c->nz_mask,
                    c->nz_u,       c->nz_v,       c->tile_start, c->tile_list,  c->w,         c->fpart,        c->part_sc,
                    c->part_ls,    c->psi,        c->g,          c->g_prev,    c->eta_prev,     c->st,
                    c->dscalar,    c->hist.F,     c->hist.gamma, c->hist.halvings, c->hist.alpha, c->stage_obj,
                    c->stage_obj2, c->stage_pat, c->tc_img_fwd, c->tc_img_inv, c->tc_err, c->tc_x, c->tc_t,
                    c->tc_u, c->tc_pars, c->st_den, c->st_tmax, c->st_red,
                    c->eta, c->illum, c->part_eta, c->hash, c->dsum};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->hpin) cudaFreeHost(c->hpin);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->iter_exec) cudaGraphExecDestroy(c->iter_exec);
    if (c->join) cudaEventDestroy(c->join);
    if (c->s) cudaStreamDestroy(c->s);
}

pty::PatternArgs pattern_args(const pty_ctx *c)
{
    pty::PatternArgs a;
    a.H = c->HA;
    a.W = c->WA;
    a.K = c->K;
    a.probe = c->probe;
    a.probe_stride = c->probe_stride;
    a.tw = c->tw;
    a.pos = c->pos;
    a.perm = c->perm;
    a.nz_off = c->nz_off;
    a.nz_mask = c->nz_mask;
    a.nzc = c->nzc;
    a.nz_slot = c->nz_slot;
    a.nz_d = c->nz_d;
    a.nz_u = c->nz_u;
    a.nz_v = c->nz_v;
    a.pat_view = c->pat_view;
    a.V = c->V;
    a.eps = (float)c->opts.eps;
    a.est = c->opts.estimator;
    a.dsum = c->cert ? c->dsum : nullptr;
    return a;
}

pty::ScatterPlan scatter_plan(const pty_ctx *c)
{
    pty::ScatterPlan p;
    p.TY = pty::kTileY;
    p.TX = pty::kTileX;
    p.ntile_y = c->ntile_y;
    p.ntile_x = c->ntile_x;
    p.tile_start = c->tile_start;
    p.tile_list = c->tile_list;
    p.tile_view = c->tile_view;
    return p;
}

// A device wait of the call gave up (flag read after the call's synchronisation): clear the
// flag and report it.
int check_wait_error(pty_ctx *c, int herr)
{
    if (!herr) return PTY_OK;
    cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->s);
    return fail(c, PTY_ERR_TIMEOUT, "a bounded device wait timed out (tensor-core DFT or tensor-copy scatter-add)");
}

// The scatter-add of c->w: by tensor copies when the context has the tensor map of w.
cudaError_t scatter(pty_ctx *c, const pty::PatternArgs &a, const pty::ScatterPlan &plan, float2 *out, int dy,
                    float2 *part, const DevState *st, const float2 *psi = nullptr, const float *D = nullptr)
{
    if (c->wmap_ok)
        return pty::launch_scatter_tma(c->P, c->wmap, a, plan, out, dy, c->eta_prev, c->g_prev, part, st, c->s, psi, D,
                                       c->tc_err, pty::tc_wait_limit());
    return pty::launch_scatter(c->P, a, plan, c->w, out, dy, c->eta_prev, c->g_prev, part, st, c->s, psi, D);
}

pty::ViewMap view_map(const pty_ctx *c)
{
    pty::ViewMap m;
    m.V = c->V;
    m.pat_off = c->view_pat_off;
    m.tile_off = c->view_tile_off;
    m.row_view = c->row_view;
    return m;
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
    l.warm = c->opts.ls_warm != 0;
    l.gd = c->opts.solver == 1;
    l.gd_step = c->opts.gd_step;
    return l;
}

// Order the context's stream after the caller's (the caller may have just written inputs).
int enter(pty_ctx *c)
{
    CK(cudaEventRecord(c->join, c->user));
    CK(cudaStreamWaitEvent(c->s, c->join, 0));
    return PTY_OK;
}

int ensure_stage(pty_ctx *c)
{
    const size_t n = (size_t)c->HA * c->WA;
    if (!c->stage_obj) CK(dalloc(&c->stage_obj, n));
    if (!c->stage_obj2) CK(dalloc(&c->stage_obj2, n));
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
    const int cap = std::max(n, 64);
    if (c->hist.F) {
        cudaFree(c->hist.F);
        cudaFree(c->hist.gamma);
        cudaFree(c->hist.halvings);
        cudaFree(c->hist.alpha);
        c->hist = DevHist{};
    }
    CK(dalloc(&c->hist.F, (size_t)c->V * (cap + 1)));
    CK(dalloc(&c->hist.gamma, (size_t)c->V * cap));
    CK(dalloc(&c->hist.halvings, (size_t)c->V * cap));
    CK(dalloc(&c->hist.alpha, (size_t)c->V * cap));
    c->hist.cap = cap;
    // the captured iteration refers to the history arrays: capture again
    if (c->iter_exec) {
        cudaGraphExecDestroy(c->iter_exec);
        c->iter_exec = nullptr;
    }
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
    cudaEventRecord(c->ev_pool[i], c->s);
    return i;
}

struct StageTimer {
    pty_ctx *c;
    int stage;
    bool on;
    size_t a = (size_t)-1;
    StageTimer(pty_ctx *c_, int s, bool on_) : c(c_), stage(s), on(on_)
    {
        if (on) a = ev_mark(c);
    }
    ~StageTimer()
    {
        if (on && a != (size_t)-1) {
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
    CK(cudaStreamSynchronize(c->s));
    collect_times(c);
    return PTY_OK;
}

// Copy the caller's objects (one per view, [H_v][W_v], host or device) into an atlas buffer.
int views_in(pty_ctx *c, const float *const *psi, float2 *atlas)
{
    for (int v = 0; v < c->V; v++) {
        const size_t pitch = sizeof(float2) * c->WA, width = sizeof(float2) * c->Wv[v];
        CK(cudaMemcpy2DAsync(atlas + (size_t)c->R0[v] * c->WA, pitch, psi[v], width, width, c->Hv[v],
                             cudaMemcpyDefault, c->s));
    }
    return PTY_OK;
}

int views_out(pty_ctx *c, float *const *psi, const float2 *atlas)
{
    for (int v = 0; v < c->V; v++) {
        const size_t pitch = sizeof(float2) * c->WA, width = sizeof(float2) * c->Wv[v];
        CK(cudaMemcpy2DAsync(psi[v], width, atlas + (size_t)c->R0[v] * c->WA, pitch, width, c->Hv[v],
                             cudaMemcpyDefault, c->s));
    }
    return PTY_OK;
}

// GRAD pattern pass of the tensor-core form: psi -> w (sorted order) and fpart.
int tc_grad(pty_ctx *c, const float2 *psi, const DevState *st)
{
    const pty::PatternArgs a = pattern_args(c);
    const bool bf16 = c->opts.dft == 1;
    const int rows = c->K * c->P;
    CK(pty::launch_gather_patches(a, c->P, psi, c->tc_x, c->s));
    CK(pty::tc_dft_rows(c->P, bf16, c->tc_x, c->tc_t, c->tc_img_fwd, rows, nullptr, nullptr, c->tc_err, c->s));
    CK(pty::tc_dft_rows(c->P, bf16, c->tc_t, c->tc_u, c->tc_img_fwd, rows, nullptr, nullptr, c->tc_err, c->s));
    CK(pty::launch_tc_residual(a, c->P, c->tc_u, c->fpart, st, c->s));
    CK(pty::tc_dft_rows(c->P, bf16, c->tc_u, c->tc_t, c->tc_img_inv, rows, nullptr, nullptr, c->tc_err, c->s));
    CK(pty::tc_dft_rows(c->P, bf16, c->tc_t, c->w, c->tc_img_inv, rows, nullptr, c->probe, c->tc_err, c->s));
    return PTY_OK;
}

// The launches of one CG iteration on the context's stream (plain, timed or captured).
// GRAD passes in the linear form between full passes: every kLinPeriod-th iteration (by the
// total count since the last reset) recomputes u at the entries with the forward DFT.  Over
// 128 iterations of the 1024^2 workload the objective of the linear form stays within 2.6e-7
// of the full form's with identical trial counts for periods 16 to 128 alike: the FP32 drift
// of the carried u is below CG's own amplification of rounding.
#ifndef PTY_LIN_PERIOD
#define PTY_LIN_PERIOD 64  // iterations between full forward passes of the GRAD stage
#endif
constexpr int kLinPeriod = PTY_LIN_PERIOD;

int launch_iteration(pty_ctx *c, bool timed)
{
    if (c->opts.dft != 0) {
        const pty::PatternArgs a = pattern_args(c);
        const pty::ScatterPlan plan = scatter_plan(c);
        const pty::ViewMap vm = view_map(c);
        const pty::LsArgs ls = ls_args(c);
        const bool bf16 = c->opts.dft == 1;
        const int rows = c->K * c->P;
        const int first = ls.adaptive ? 4 : ls.L;
        const int nwin = 1 + (std::max(0, c->opts.max_halvings - first) + ls.L - 1) / ls.L;
        int st;
        {
            StageTimer t(c, 0, timed);
            if ((st = tc_grad(c, c->psi, c->st))) return st;
        }
        {
            StageTimer t(c, 1, timed);
            CK(scatter(c, a, plan, c->g, 1, c->part_sc, c->st));
        }
        {
            StageTimer t(c, 3, timed);
            CK(pty::launch_dy_finalize(c->fpart, 1, 0, c->part_sc, 0.0, vm, c->st, c->hist, ls, c->s));
        }
        {
            StageTimer t(c, 2, timed);  // v = G eta once per iteration; windows reuse it
            CK(pty::launch_tc_gather_eta(a, c->P, c->psi, c->g, c->eta_prev, c->tc_x, c->tc_pars, c->st, c->s));
            CK(pty::tc_dft_rows(c->P, bf16, c->tc_x, c->tc_t, c->tc_img_fwd, rows, nullptr, nullptr, c->tc_err, c->s));
            CK(pty::tc_dft_rows(c->P, bf16, c->tc_t, c->tc_u, c->tc_img_fwd, rows, nullptr, nullptr, c->tc_err, c->s));
        }
        for (int wdx = 0; wdx < nwin; wdx++) {
            {
                StageTimer t(c, 4, timed);
                if (wdx == 0 && ls.adaptive)
                    CK(pty::launch_tc_ls_entries(a, c->P, 16, c->tc_u, c->tc_pars, c->part_ls, c->st, c->s));
                CK(pty::launch_tc_ls_entries(a, c->P, ls.L, c->tc_u, c->tc_pars, c->part_ls, c->st, c->s));
            }
            StageTimer t(c, 3, timed);
            CK(pty::launch_ls_decide(c->part_ls, c->K, 1, 0, 0, vm, nullptr, 0.0, ls, c->st, c->hist, c->s));
        }
        StageTimer t(c, 3, timed);
        CK(pty::launch_update(c->HA, c->WA, vm, c->psi, c->g, c->eta_prev, c->g_prev, c->st, 0, c->s));
        return PTY_OK;
    }
    const pty::PatternArgs a = pattern_args(c);
    const pty::ScatterPlan plan = scatter_plan(c);
    const pty::ViewMap vm = view_map(c);
    const pty::LsArgs ls = ls_args(c);
    if (ls.gd) {
        // gradient descent (Eq. 4): GRAD (full form), scatter, F(psi_m), psi -= gamma g
        {
            StageTimer t(c, 0, timed);
            CK(c->impl->grad(a, c->psi, c->w, c->fpart, c->st, c->s));
        }
        {
            StageTimer t(c, 1, timed);
            CK(scatter(c, a, plan, c->g, 1, c->part_sc, c->st, c->psi, c->illum));
        }
        StageTimer t(c, 3, timed);
        CK(pty::launch_dy_finalize(c->fpart, c->CS, c->impl->grad_cols(a), c->part_sc, (double)c->P * c->P, vm, c->st,
                                   c->hist, ls, c->s));
        CK(pty::launch_gd_step(vm, ls, c->st, c->hist, c->s));
        CK(pty::launch_update(c->HA, c->WA, vm, c->psi, c->g, c->eta_prev, c->g_prev, c->st, 0, c->s));
        return PTY_OK;
    }
    // first window >= 4 candidates when adaptive (then full windows of L), else L each
    const int first = ls.adaptive ? 4 : ls.L;
    const int rest = std::max(0, c->opts.max_halvings - first);
    const int nwin = 1 + (rest + ls.L - 1) / ls.L;
    {
        StageTimer t(c, 0, timed);  // full pass, or the linear form (each returns at once if not chosen)
        CK(c->impl->grad(a, c->psi, c->w, c->fpart, c->st, c->s));
        CK(c->impl->grad_lin(a, c->w, c->fpart, c->st, c->s));
    }
    {
        StageTimer t(c, 1, timed);
        CK(scatter(c, a, plan, c->g, 1, c->part_sc, c->st, c->psi, c->illum));
    }
    {
        StageTimer t(c, 3, timed);
        CK(pty::launch_dy_finalize(c->fpart, c->CS, c->impl->grad_cols(a), c->part_sc, (double)c->P * c->P, vm, c->st,
                                   c->hist, ls, c->s));
    }
    {
        StageTimer t(c, 3, timed);  // the search direction and its object sums
        CK(pty::launch_eta(c->HA, c->WA, plan, c->psi, c->g, c->eta_prev, c->illum, c->eta, c->part_eta, c->st, c->s));
    }
    {
        StageTimer t(c, 2, timed);  // v = G eta once per iteration; the windows reuse it
        CK(c->impl_ls->ls(a, c->eta, c->part_ls, c->st, c->s));
    }
    // with one view the LS pass and the windows write one column per CTA
    const int ls_cols = c->impl_ls->ls_cols(a), en_cols = pty::ls_entries_cols(a, c->CSl, c->V);
    if (c->cert) {
        StageTimer t(c, 4, timed);
        CK(pty::launch_ls_certify(c->part_ls, c->K * c->CSl, c->CSl, ls_cols, vm, c->part_eta, (double)c->P * c->P, ls,
                                  c->st, c->s));
    }
    for (int wdx = 0; wdx < nwin; wdx++) {
        {
            StageTimer t(c, 4, timed);
            // the first window of an adaptive search runs on the 4- or 8- (warm start), 8-
            // (certified start), 16- or 32-candidate kernel as the device chose; the others
            // return at once
            if (wdx == 0 && ls.adaptive && ls.warm) {
                CK(pty::launch_ls_entries(a, c->CSl, c->V, 4, c->part_ls, c->st, c->s));
                CK(pty::launch_ls_entries(a, c->CSl, c->V, 8, c->part_ls, c->st, c->s));
            }
            if (wdx == 0 && ls.adaptive && c->cert) {
                CK(pty::launch_ls_entries(a, c->CSl, c->V, 6, c->part_ls, c->st, c->s));
                CK(pty::launch_ls_entries(a, c->CSl, c->V, 8, c->part_ls, c->st, c->s));
            }
            if (wdx == 0 && ls.adaptive) CK(pty::launch_ls_entries(a, c->CSl, c->V, 16, c->part_ls, c->st, c->s));
            CK(pty::launch_ls_entries(a, c->CSl, c->V, ls.L, c->part_ls, c->st, c->s));
        }
        StageTimer t(c, 3, timed);
        CK(pty::launch_ls_decide(c->part_ls, c->K * c->CSl, c->CSl, ls_cols, en_cols, vm, c->part_eta,
                                 (double)c->P * c->P, ls, c->st,
                                 c->hist, c->s));
    }
    StageTimer t(c, 3, timed);
    const int lin_period = (c->opts.flags & 2) ? 0 : kLinPeriod;
    CK(pty::launch_update(c->HA, c->WA, vm, c->psi, c->g, c->eta_prev, c->g_prev, c->st, lin_period, c->s));
    return PTY_OK;
}

// Capture one iteration into a graph (once per context and configuration).
void build_graph(pty_ctx *c)
{
    if (c->iter_exec || c->graph_failed) return;
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        const int st = launch_iteration(c, false);
        ok = cudaStreamEndCapture(c->s, &g) == cudaSuccess && st == PTY_OK;
    }
    if (ok) ok = cudaGraphInstantiate(&c->iter_exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();
        c->iter_exec = nullptr;
        c->graph_failed = true;  // plain launches of the same kernels from now on
    }
}

// The autotuner: time the GRAD pass in its linear form (the form of all but every 64th
// iteration) and the LS pattern pass of every configuration for P on the context's own data
// (entries' u = v = 0, eta = 0, a 16-candidate window; the minimum of three runs each) and
// keep the fastest of each.  The first iteration of every solve runs the full form, which
// recomputes u at the entries.  The choice is cached per problem shape for the life of the process, so contexts of
// the same problem use the same kernels (and give the same bits).
struct PlanKey {
    int P, H, W, K, V;
    long long nnz;
    bool operator<(const PlanKey &o) const
    {
        return std::tie(P, H, W, K, V, nnz) < std::tie(o.P, o.H, o.W, o.K, o.V, o.nnz);
    }
};
std::mutex g_plan_mu;
std::map<PlanKey, std::pair<int, int>> g_plan_cache;

int autotune(pty_ctx *c)
{
    const pty::PatternImpl *impls = nullptr;
    const int n = pty::pattern_impls(c->P, &impls);
    const PlanKey key{c->P, c->HA, c->WA, c->K, c->V, c->n_entries};
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
        const size_t HW = (size_t)c->HA * c->WA;
        std::vector<float2> ones(HW, make_float2(1.f, 0.f));
        CK(cudaMemcpyAsync(c->psi, ones.data(), sizeof(float2) * HW, cudaMemcpyHostToDevice, c->s));
        CK(cudaMemsetAsync(c->nz_u, 0, sizeof(float2) * (size_t)std::max<long long>(c->n_entries, 1), c->s));
        CK(cudaMemsetAsync(c->nz_v, 0, sizeof(float2) * (size_t)std::max<long long>(c->n_entries, 1), c->s));
        std::vector<DevState> hs(c->V);
        for (auto &h : hs) {
            h.lin = 1;  // the linear form runs
            h.last_gamma = 0.5;
            h.Leff = 16;
            h.Lsel = 16;
            for (int l = 0; l < 16; l++) {
                h.cand[l] = std::ldexp(1.0, -(l + 1));
                h.cand_f[l] = (float)h.cand[l];
            }
        }
        CK(cudaMemcpyAsync(c->st, hs.data(), sizeof(DevState) * c->V, cudaMemcpyHostToDevice, c->s));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        const pty::PatternArgs a = pattern_args(c);
        float tg = 1e30f, tl = 1e30f;
        cudaError_t err = cudaSuccess;
        for (int j = 0; j < n && err == cudaSuccess; j++) {
            float mg = 1e30f, ml = 1e30f, ms = 0.f;
            for (int rep = 0; rep < 3 && err == cudaSuccess; rep++) {
                err = cudaEventRecord(e0, c->s);
                if (err == cudaSuccess) err = impls[j].grad_lin(a, c->w, c->fpart, c->st, c->s);
                if (err == cudaSuccess) err = cudaEventRecord(e1, c->s);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                if (err == cudaSuccess) mg = std::min(mg, ms);
            }
            if (err == cudaSuccess && mg < tg) {
                tg = mg;
                best_g = j;
            }
            for (int rep = 0; rep < 3 && err == cudaSuccess; rep++) {
                err = cudaEventRecord(e0, c->s);
                if (err == cudaSuccess) err = impls[j].ls(a, c->eta, c->part_ls, c->st, c->s);
                if (err == cudaSuccess) err = cudaEventRecord(e1, c->s);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                if (err == cudaSuccess) ml = std::min(ml, ms);
            }
            if (err == cudaSuccess && ml < tl) {
                tl = ml;
                best_l = j;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (err != cudaSuccess) return fail(c, PTY_ERR_CUDA, "autotune: %s", cudaGetErrorString(err));
        CK(cudaMemsetAsync(c->st, 0, sizeof(DevState) * c->V, c->s));
        CK(cudaStreamSynchronize(c->s));
        std::lock_guard<std::mutex> lock(g_plan_mu);
        g_plan_cache[key] = {best_g, best_l};
    }
    c->impl = &impls[best_g];
    c->impl_ls = &impls[best_l];
    c->CS = c->P / c->impl->R;
    c->CSl = c->P / c->impl_ls->R;
    return PTY_OK;
}

// fpos (optional, one view): float positions [K][2]; the window starts at floor(fpos) and
// each position gets its own probe, moved by the fraction (subpixel.cu).  pos is then unused.
int create_views(pty_ctx **out, int32_t V, const int32_t *Hs, const int32_t *Ws, const int32_t *Ks, int32_t P,
                 const float *probe, const int32_t *pos, const float *data, const pty_opts *opts, void *stream,
                 const float *fpos = nullptr)
{
    if (!out) return fail(nullptr, PTY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (V < 1 || !Hs || !Ws || !Ks) return fail(nullptr, PTY_ERR_ARG, "bad view description");
    if (!probe || !(pos || fpos) || !data) return fail(nullptr, PTY_ERR_ARG, "probe, pos and data must be non-NULL");
    if (!pty::pattern_supported(P)) return fail(nullptr, PTY_ERR_ARG, "P=%d not supported (64, 128 or 256)", P);
    long long K = 0, rows = 0;
    int WA = 0;
    for (int v = 0; v < V; v++) {
        if (Hs[v] < P || Ws[v] < P)
            return fail(nullptr, PTY_ERR_ARG, "view %d: object %dx%d smaller than probe %d", v, Hs[v], Ws[v], P);
        if (Ks[v] < 1) return fail(nullptr, PTY_ERR_ARG, "view %d: K=%d < 1", v, Ks[v]);
        K += Ks[v];
        rows = (v + 1 < V) ? (rows + Hs[v] + 31) / 32 * 32 : rows + Hs[v];
        WA = std::max(WA, (int)Ws[v]);
    }
    if (K > (1LL << 30) || rows * WA > (1LL << 31)) return fail(nullptr, PTY_ERR_ARG, "problem too large");
    pty_opts o;
    pty_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.tau > 0.0 && o.tau < 1.0) || !(o.gamma0 > 0.0 && std::isfinite(o.gamma0)) || o.max_halvings < 1 ||
        o.max_halvings > 1000 || !(o.eps >= 0.0 && std::isfinite(o.eps)) || !std::isfinite(o.t) || (o.ls_window != 0 && !pty::ls_window_supported(o.ls_window)) ||
        o.dft < 0 || o.dft > 2 || (o.estimator != 0 && o.estimator != 1) || (o.solver != 0 && o.solver != 1) ||
        (o.ls_warm != 0 && o.ls_warm != 1) || (o.solver == 1 && !(o.gd_step > 0.0 && std::isfinite(o.gd_step))) ||
        (o.solver == 1 && o.ls_warm))
        return fail(nullptr, PTY_ERR_ARG, "invalid options (tau in (0,1), finite gamma0 > 0, 1 <= max_halvings <= "
                                          "1000, finite eps >= 0, finite t, ls_window in {0,4,8,16,32}, dft in {0,1,2}, estimator and "
                                          "solver in {0,1}, gd_step > 0 with solver 1, ls_warm 0 or 1 with solver 0)");
    if (o.dft != 0 && !pty::tc_dft_supported(P, o.dft == 1))
        return fail(nullptr, PTY_ERR_UNSUPPORTED,
                    "the tensor-core DFT supports P = 64, 128 and 256 (split BF16) or P = 64, 128 (split FP16)");
    if (o.dft != 0 && (o.estimator != 0 || o.solver != 0 || o.ls_warm))
        return fail(nullptr, PTY_ERR_UNSUPPORTED,
                    "the least-squares estimator, gradient descent and the warm-started search need dft = 0");
    if (fpos && (V != 1 || o.dft != 0))
        return fail(nullptr, PTY_ERR_UNSUPPORTED, "fractional positions need one view and dft = 0");

    // positions: host copy, bounds check per view, atlas coordinates, position sort
    std::vector<int32_t> hpos((size_t)2 * K);
    std::vector<float> hfrac;  // fractional parts (row, col) per caller index, with fpos
    if (fpos) {
        std::vector<float> hf((size_t)2 * K);
        if (is_device_ptr(fpos)) {
            if (cudaMemcpy(hf.data(), fpos, sizeof(float) * 2 * K, cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(nullptr, PTY_ERR_CUDA, "cannot read positions");
        } else {
            std::memcpy(hf.data(), fpos, sizeof(float) * 2 * K);
        }
        hfrac.resize((size_t)2 * K);
        for (size_t e = 0; e < hf.size(); e++) {
            if (!std::isfinite(hf[e]) || std::fabs(hf[e]) > 1e9f)
                return fail(nullptr, PTY_ERR_BOUNDS, "position %d holds a non-finite or huge coordinate",
                            (int)(e / 2));
            const double fl = std::floor((double)hf[e]);
            hpos[e] = (int32_t)fl;
            hfrac[e] = (float)((double)hf[e] - fl);  // exact: a float minus its floor
        }
    } else if (is_device_ptr(pos)) {
        if (cudaMemcpy(hpos.data(), pos, sizeof(int32_t) * 2 * K, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(nullptr, PTY_ERR_CUDA, "cannot read positions");
    } else {
        std::memcpy(hpos.data(), pos, sizeof(int32_t) * 2 * K);
    }
    std::vector<int> R0(V), Koff(V + 1, 0), view_of(K);
    for (int v = 0, r = 0; v < V; v++) {
        R0[v] = r;
        r = (r + Hs[v] + 31) / 32 * 32;
        Koff[v + 1] = Koff[v] + Ks[v];
    }
    for (int v = 0; v < V; v++)
        for (int k = Koff[v]; k < Koff[v + 1]; k++) {
            const int r = hpos[2 * k], cc = hpos[2 * k + 1];
            if (r < 0 || cc < 0 || r > Hs[v] - P || cc > Ws[v] - P)
                return fail(nullptr, PTY_ERR_BOUNDS, "view %d position %d (%d,%d) puts the %dx%d patch outside %dx%d",
                            v, k - Koff[v], r, cc, P, P, Hs[v], Ws[v]);
            hpos[2 * k] = r + R0[v];
            view_of[k] = v;
        }

    pty_ctx *c = new (std::nothrow) pty_ctx;
    if (!c) return fail(nullptr, PTY_ERR_NOMEM, "host allocation failed");
    cudaGetDevice(&c->dev);
    c->user = (cudaStream_t)stream;
    c->V = V;
    c->P = P;
    c->K = (int)K;
    c->HA = (int)rows;
    c->WA = WA;
    c->Hv.assign(Hs, Hs + V);
    c->Wv.assign(Ws, Ws + V);
    c->Kv.assign(Ks, Ks + V);
    c->R0 = R0;
    c->Koff = Koff;
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
    CKC(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
    CKC(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming));
    if (enter(c) != PTY_OK) return bail(PTY_ERR_CUDA);

    std::vector<int> perm(K);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
        return hpos[2 * a] != hpos[2 * b] ? hpos[2 * a] < hpos[2 * b] : hpos[2 * a + 1] < hpos[2 * b + 1];
    });
    std::vector<int2> spos(K);
    std::vector<int> pview(K), vpoff(V + 1, 0);
    for (int i = 0; i < K; i++) {
        spos[i] = make_int2(hpos[2 * perm[i]], hpos[2 * perm[i] + 1]);
        pview[i] = view_of[perm[i]];
    }
    for (int v = 0; v < V; v++) vpoff[v + 1] = vpoff[v] + Ks[v];  // views are contiguous after the sort

    // scatter plan: object tiles of kTileY x kTileX, each with the ascending list of
    // overlapping patterns
    const int TY = pty::kTileY, TX = pty::kTileX;
    c->ntile_y = (c->HA + TY - 1) / TY;
    c->ntile_x = (c->WA + TX - 1) / TX;
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
    std::vector<int> rview(c->HA, V - 1), tview(ntiles), vtoff(V + 1, 0);
    for (int v = 0; v < V; v++)
        for (int y = R0[v]; y < std::min(c->HA, v + 1 < V ? R0[v + 1] : c->HA); y++) rview[y] = v;
    for (int b = 0; b < ntiles; b++) tview[b] = rview[(b / c->ntile_x) * TY];
    for (int v = 0; v < V; v++) vtoff[v] = (R0[v] / TY) * c->ntile_x;
    vtoff[V] = ntiles;

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

    const size_t PP = (size_t)P * P, HW = (size_t)c->HA * c->WA;
    CKC(dalloc(&c->probe, fpos ? (size_t)K * PP : PP));
    CKC(dalloc(&c->tw, (size_t)P));
    CKC(dalloc(&c->pos, (size_t)K));
    CKC(dalloc(&c->perm, (size_t)K));
    CKC(dalloc(&c->pat_view, (size_t)K));
    CKC(dalloc(&c->view_pat_off, (size_t)V + 1));
    CKC(dalloc(&c->view_tile_off, (size_t)V + 1));
    CKC(dalloc(&c->row_view, (size_t)c->HA));
    CKC(dalloc(&c->tile_view, (size_t)ntiles));
    CKC(dalloc(&c->tile_start, (size_t)ntiles + 1));
    CKC(dalloc(&c->tile_list, std::max<size_t>(list.size(), 1)));
    CKC(dalloc(&c->w, (size_t)K * PP));
    CKC(dalloc(&c->tc_err, (size_t)1));
    CKC(cudaMemset(c->tc_err, 0, sizeof(int)));
    // scatter-add by tensor copies unless the driver cannot describe w (or opts.flags bit 4)
    c->wmap_ok = !(o.flags & 16) && pty::scatter_tma_map_bytes() <= sizeof(c->wmap) &&
                 pty::make_scatter_tma_map(c->wmap, c->w, P, (int)K);
    CKC(dalloc(&c->fpart, (size_t)K * c->CSmax));
    CKC(dalloc(&c->part_sc, (size_t)ntiles * 3));
    CKC(dalloc(&c->hash, (size_t)V));
    CKC(dalloc(&c->part_ls, (size_t)K * c->CSmax * (32 + 2)));
    CKC(dalloc(&c->psi, HW));
    CKC(dalloc(&c->g, HW));
    CKC(dalloc(&c->g_prev, HW));
    CKC(dalloc(&c->eta_prev, HW));
    CKC(dalloc(&c->eta, HW));
    CKC(dalloc(&c->illum, HW));
    CKC(dalloc(&c->part_eta, (size_t)ntiles * 2));
    CKC(dalloc(&c->st, (size_t)V));
    CKC(dalloc(&c->dscalar, (size_t)4));
    if (fpos) {
        // one probe per sorted pattern, moved by its position's fraction
        std::vector<float2> sfrac(K);
        for (int i = 0; i < K; i++) sfrac[i] = make_float2(hfrac[2 * perm[i]], hfrac[2 * perm[i] + 1]);
        float2 *dp = nullptr, *df = nullptr;
        cudaError_t e = dalloc(&dp, PP);
        if (e == cudaSuccess) e = dalloc(&df, (size_t)K);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dp, hprobe.data(), sizeof(float2) * PP, cudaMemcpyHostToDevice, c->s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(df, sfrac.data(), sizeof(float2) * K, cudaMemcpyHostToDevice, c->s);
        if (e == cudaSuccess) e = pty::launch_shift_probes(P, (int)K, dp, df, c->probe, c->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
        if (dp) cudaFree(dp);
        if (df) cudaFree(df);
        CKC(e);
        c->probe_stride = (long long)PP;
    } else {
        CKC(cudaMemcpyAsync(c->probe, hprobe.data(), sizeof(float2) * PP, cudaMemcpyHostToDevice, c->s));
    }
    CKC(cudaMemcpyAsync(c->tw, htw.data(), sizeof(float2) * P, cudaMemcpyHostToDevice, c->s));
    CKC(cudaMemcpyAsync(c->pos, spos.data(), sizeof(int2) * K, cudaMemcpyHostToDevice, c->s));
    CKC(cudaMemcpyAsync(c->perm, perm.data(), sizeof(int) * K, cudaMemcpyHostToDevice, c->s));
    CKC(cudaMemcpyAsync(c->pat_view, pview.data(), sizeof(int) * K, cudaMemcpyHostToDevice, c->s));
    CKC(cudaMemcpyAsync(c->view_pat_off, vpoff.data(), sizeof(int) * (V + 1), cudaMemcpyHostToDevice, c->s));
    CKC(cudaMemcpyAsync(c->view_tile_off, vtoff.data(), sizeof(int) * (V + 1), cudaMemcpyHostToDevice, c->s));
    CKC(cudaMemcpyAsync(c->row_view, rview.data(), sizeof(int) * c->HA, cudaMemcpyHostToDevice, c->s));
    CKC(cudaMemcpyAsync(c->tile_view, tview.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice, c->s));
    CKC(cudaMemcpyAsync(c->tile_start, cnt.data(), sizeof(int) * (ntiles + 1), cudaMemcpyHostToDevice, c->s));
    if (!list.empty())
        CKC(cudaMemcpyAsync(c->tile_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, c->s));
    CKC(cudaMemsetAsync(c->g_prev, 0, sizeof(float2) * HW, c->s));
    CKC(cudaMemsetAsync(c->eta_prev, 0, sizeof(float2) * HW, c->s));
    CKC(cudaMemsetAsync(c->eta, 0, sizeof(float2) * HW, c->s));
    CKC(cudaMemsetAsync(c->psi, 0, sizeof(float2) * HW, c->s));
    CKC(pty::launch_illumination(P, pattern_args(c), scatter_plan(c), c->illum, c->s));
    CKC(cudaMemsetAsync(c->st, 0, sizeof(DevState) * V, c->s));

    // measured data: read here only (a host array goes through a temporary device copy)
    // and kept as the compact list of pixels with counts, in tile slot order
    const float *dd = data;
    float *dtmp = nullptr;
    if (!is_device_ptr(data)) {
        CKC(dalloc(&dtmp, (size_t)K * PP));
        CKC(cudaMemcpyAsync(dtmp, data, sizeof(float) * K * PP, cudaMemcpyHostToDevice, c->s));
        dd = dtmp;
    }
    auto free_tmp = [&]() {
        if (dtmp) cudaFree(dtmp);
        dtmp = nullptr;
    };
    int *flag = (int *)c->dscalar;
    int *dcnt = nullptr;
    const int KC = (int)K * c->nzc;
    std::vector<int> hcnt(KC);
    int hflag = 0;
    cudaError_t ce = cudaMemsetAsync(flag, 0, sizeof(int), c->s);
    if (ce == cudaSuccess) ce = pty::launch_check_data(dd, (size_t)K * PP, flag, c->s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    if (ce == cudaSuccess) ce = dalloc(&dcnt, (size_t)KC);
    if (ce == cudaSuccess) ce = c->impl_nz->nz_count(dd, c->perm, (int)K, dcnt, c->s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hcnt.data(), dcnt, sizeof(int) * KC, cudaMemcpyDeviceToHost, c->s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->s);
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
    if (ce == cudaSuccess) ce = dalloc(&c->nz_v, E);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(c->nz_off, hoff.data(), sizeof(long long) * (KC + 1), cudaMemcpyHostToDevice, c->s);
    if (ce == cudaSuccess) ce = c->impl_nz->nz_fill(dd, c->perm, (int)K, c->nz_off, c->nz_slot, c->nz_d, c->s);
    // the entry slots as bit masks for the linear GRAD pass (unless opts.flags bit 5)
    if (ce == cudaSuccess && P <= 128 && !(o.flags & 32)) {
        const size_t words = (size_t)K * P * P / 32;
        ce = dalloc(&c->nz_mask, words);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(c->nz_mask, 0, sizeof(unsigned) * words, c->s);
        if (ce == cudaSuccess) ce = pty::launch_nz_mask(pattern_args(c), P, c->nz_mask, c->s);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->s);
    free_tmp();
    if (ce != cudaSuccess)
        return bail(fail(c, ce == cudaErrorMemoryAllocation ? PTY_ERR_NOMEM : PTY_ERR_CUDA, "data compaction: %s",
                         cudaGetErrorString(ce)));
    if (o.dft != 0) {
        std::vector<uint8_t> img;
        const bool bf16 = o.dft == 1;
        CKC(pty::tc_dft_images(P, bf16, -1, img));
        CKC(dalloc(&c->tc_img_fwd, img.size()));
        CKC(cudaMemcpy(c->tc_img_fwd, img.data(), img.size(), cudaMemcpyHostToDevice));
        CKC(pty::tc_dft_images(P, bf16, +1, img));
        CKC(dalloc(&c->tc_img_inv, img.size()));
        CKC(cudaMemcpy(c->tc_img_inv, img.data(), img.size(), cudaMemcpyHostToDevice));
        CKC(dalloc(&c->tc_x, (size_t)K * PP));
        CKC(dalloc(&c->tc_t, (size_t)K * PP));
        CKC(dalloc(&c->tc_u, (size_t)K * PP));
        CKC(dalloc(&c->tc_pars, (size_t)2 * K));
        c->CS = c->CSl = 1;  // one partial per pattern in this form
    }
#undef CKC
    if (o.tile_config < 0 && o.dft == 0) {
        const int at = autotune(c);
        if (at != PTY_OK) return bail(at);
    }
    // certified skip of leading line-search trials: adaptive windows of the FFT form
    if (o.dft == 0 && o.ls_window == 0 && !(o.flags & 4) && o.estimator == 0 && o.solver == 0 && !o.ls_warm) {
        cudaError_t ce2 = dalloc(&c->dsum, (size_t)K * c->CSl);
        if (ce2 == cudaSuccess) ce2 = pty::launch_chunk_dsum(pattern_args(c), c->CSl, c->dsum, c->s);
        if (ce2 == cudaSuccess) ce2 = cudaStreamSynchronize(c->s);
        if (ce2 != cudaSuccess)
            return bail(fail(c, ce2 == cudaErrorMemoryAllocation ? PTY_ERR_NOMEM : PTY_ERR_CUDA, "certificate weights: %s",
                             cudaGetErrorString(ce2)));
        c->cert = true;
    }
    *out = c;
    return PTY_OK;
}

// Layout of the pinned staging area: [V] DevState, then the history arrays F [V][cap+1],
// gamma, alpha [V][cap] (double), halvings [V][cap] (int), then the tensor-core error flag.
struct HostStage {
    DevState *st;
    double *F, *gamma, *alpha;
    int *halvings, *err;
};

int ensure_pinned(pty_ctx *c, HostStage &h)
{
    const size_t V = c->V, cap = c->hist.cap;
    const size_t n = sizeof(DevState) * V + sizeof(double) * V * (3 * cap + 1) + sizeof(int) * (V * cap + 1);
    if (c->hpin_bytes < n) {
        if (c->hpin) cudaFreeHost(c->hpin);
        c->hpin = nullptr;
        c->hpin_bytes = 0;
        CK(cudaMallocHost((void **)&c->hpin, n));
        c->hpin_bytes = n;
    }
    unsigned char *q = c->hpin;
    h.st = (DevState *)q;
    q += sizeof(DevState) * V;
    h.F = (double *)q;
    h.gamma = h.F + V * (cap + 1);
    h.alpha = h.gamma + V * cap;
    h.halvings = (int *)(h.alpha + V * cap);
    h.err = h.halvings + V * cap;
    return PTY_OK;
}

// Fill a host report per view from the staged history.
void read_reports(const pty_ctx *c, int niter, pty_cg_report *rep, const HostStage &h)
{
    if (!rep) return;
    const int cap = c->hist.cap;
    for (int v = 0; v < c->V; v++) {
        const int done = h.st[v].m;
        rep[v].iters_done = done;
        if (niter <= 0) continue;
        const int nrec = std::min(niter, done + (h.st[v].stalled ? 1 : 0));
        if (rep[v].F)
            for (int i = 0; i <= std::min(done, niter); i++) rep[v].F[i] = h.F[(size_t)v * (cap + 1) + i];
        for (int i = 0; i < nrec; i++) {
            if (rep[v].gamma) rep[v].gamma[i] = h.gamma[(size_t)v * cap + i];
            if (rep[v].alpha) rep[v].alpha[i] = h.alpha[(size_t)v * cap + i];
            if (rep[v].halvings) rep[v].halvings[i] = h.halvings[(size_t)v * cap + i];
        }
    }
}

int solve(pty_ctx *c, float *const *psi, int32_t niter, pty_cg_report *rep)
{
    int st;
    if ((st = enter(c))) return st;
    if ((st = ensure_hist(c, niter))) return st;
    if ((st = views_in(c, (const float *const *)psi, c->psi))) return st;
    // the entries' u and v carry over only to the object the previous call returned
    CK(pty::launch_hash(c->HA, c->WA, c->row_view, c->psi, c->hash, c->V, c->s));
    CK(pty::launch_check_hash(c->st, c->V, c->hash, c->cache_dirty ? 1 : 0, c->s));
    c->cache_dirty = false;
    CK(pty::launch_begin_solve(c->st, c->V, c->s));
    const bool timed = (c->opts.flags & 1) != 0;
    if (!timed && niter > 0) build_graph(c);
    for (int it = 0; it < niter; it++) {
        if (!timed && c->iter_exec) {
            CK(cudaGraphLaunch(c->iter_exec, c->s));
        } else if ((st = launch_iteration(c, timed))) {
            return st;
        }
    }
    if (c->opts.solver == 1 && niter > 0) {
        // gradient descent: F of the final object, the last entry of the history
        const pty::PatternArgs a = pattern_args(c);
        CK(c->impl->grad(a, c->psi, c->w, c->fpart, c->st, c->s));
        CK(pty::launch_objective_to_hist(c->fpart, c->CS, c->impl->grad_cols(a), view_map(c), c->st, c->hist, c->s));
    }
    CK(pty::launch_hash(c->HA, c->WA, c->row_view, c->psi, c->hash, c->V, c->s));
    CK(pty::launch_store_hash(c->st, c->V, c->hash, c->s));
    // the call's results: asynchronous copies into pinned staging, one synchronisation
    HostStage hs;
    if ((st = ensure_pinned(c, hs))) return st;
    *hs.err = 0;
    CK(cudaMemcpyAsync(hs.st, c->st, sizeof(DevState) * c->V, cudaMemcpyDeviceToHost, c->s));
    if (rep && niter > 0) {
        const size_t V = c->V, cap = c->hist.cap;
        CK(cudaMemcpyAsync(hs.F, c->hist.F, sizeof(double) * V * (cap + 1), cudaMemcpyDeviceToHost, c->s));
        CK(cudaMemcpyAsync(hs.gamma, c->hist.gamma, sizeof(double) * V * cap, cudaMemcpyDeviceToHost, c->s));
        CK(cudaMemcpyAsync(hs.alpha, c->hist.alpha, sizeof(double) * V * cap, cudaMemcpyDeviceToHost, c->s));
        CK(cudaMemcpyAsync(hs.halvings, c->hist.halvings, sizeof(int) * V * cap, cudaMemcpyDeviceToHost, c->s));
    }
    if (c->tc_err) CK(cudaMemcpyAsync(hs.err, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    if ((st = views_out(c, psi, c->psi))) return st;
    if ((st = sync(c))) return st;
    if ((st = check_wait_error(c, *hs.err))) return st;
    read_reports(c, niter, rep, hs);
    for (int v = 0; v < c->V; v++)
        if (hs.st[v].stalled)
            return fail(c, PTY_STALLED, "view %d: line search found no step within %d trials at iteration %d", v,
                        c->opts.max_halvings, hs.st[v].m);
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
    o->dft = 0;
    o->estimator = 0;
    o->solver = 0;
    o->gd_step = 0.0;
    o->ls_warm = 0;
}

const char *pty_last_error(const pty_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

void pty_destroy(pty_ctx *ctx)
{
    if (!ctx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ctx->dev);
    if (ctx->s) cudaStreamSynchronize(ctx->s);
    free_all(ctx);
    cudaSetDevice(cur);
    delete ctx;
}

int pty_create(pty_ctx **out, int32_t H, int32_t W, int32_t P, const float *probe, int32_t K, const int32_t *pos,
               const float *data, const pty_opts *opts, void *stream)
{
    return create_views(out, 1, &H, &W, &K, P, probe, pos, data, opts, stream);
}

int pty_create_subpixel(pty_ctx **out, int32_t H, int32_t W, int32_t P, const float *probe, int32_t K,
                        const float *pos, const float *data, const pty_opts *opts, void *stream)
{
    if (!pos) {
        if (out) *out = nullptr;
        return fail(nullptr, PTY_ERR_ARG, "probe, pos and data must be non-NULL");
    }
    return create_views(out, 1, &H, &W, &K, P, probe, nullptr, data, opts, stream, pos);
}

int pty_batch_create(pty_ctx **out, int32_t n_views, const int32_t *H, const int32_t *W, const int32_t *K,
                     int32_t P, const float *probe, const int32_t *pos, const float *data, const pty_opts *opts,
                     void *stream)
{
    return create_views(out, n_views, H, W, K, P, probe, pos, data, opts, stream);
}

int pty_forward(pty_ctx *c, const float *psi, float *out)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!psi || !out) return fail(c, PTY_ERR_ARG, "psi and out must be non-NULL");
    if (c->V != 1) return fail(c, PTY_ERR_UNSUPPORTED, "pty_forward works on single-view contexts");
    int st;
    if ((st = enter(c)) || (st = ensure_stage(c))) return st;
    if ((st = views_in(c, &psi, c->stage_obj))) return st;
    const bool dev_out = is_device_ptr(out);
    if (!dev_out && (st = ensure_stage_pat(c))) return st;
    float2 *dout = dev_out ? (float2 *)out : c->stage_pat;
    if (c->opts.dft == 0) {
        CK(c->impl->forward(pattern_args(c), c->stage_obj, dout, c->s));
    } else {
        // tensor-core form: gather, row DFT (transposed store), row DFT into caller order
        const bool bf16 = c->opts.dft == 1;
        CK(pty::launch_gather_patches(pattern_args(c), c->P, c->stage_obj, c->tc_x, c->s));
        CK(pty::tc_dft_rows(c->P, bf16, c->tc_x, c->tc_t, c->tc_img_fwd, c->K * c->P, nullptr, nullptr, c->tc_err,
                            c->s));
        CK(pty::tc_dft_rows(c->P, bf16, c->tc_t, dout, c->tc_img_fwd, c->K * c->P, c->perm, nullptr, c->tc_err,
                            c->s));
        int herr = 0;
        CK(cudaMemcpyAsync(&herr, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        if (herr) return fail(c, PTY_ERR_TIMEOUT, "tensor-core DFT: a device wait timed out");
    }
    if (!dev_out)
        CK(cudaMemcpyAsync(out, dout, sizeof(float2) * (size_t)c->K * c->P * c->P, cudaMemcpyDeviceToHost, c->s));
    return sync(c);
}

int pty_adjoint(pty_ctx *c, const float *y, float *x)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!y || !x) return fail(c, PTY_ERR_ARG, "y and x must be non-NULL");
    if (c->V != 1) return fail(c, PTY_ERR_UNSUPPORTED, "pty_adjoint works on single-view contexts");
    if (c->opts.dft != 0) return fail(c, PTY_ERR_UNSUPPORTED, "pty_adjoint uses the FFT form (dft = 0)");
    int st;
    if ((st = enter(c)) || (st = ensure_stage(c))) return st;
    const size_t n = (size_t)c->K * c->P * c->P;
    const float2 *dy = (const float2 *)y;
    if (!is_device_ptr(y)) {
        if ((st = ensure_stage_pat(c))) return st;
        CK(cudaMemcpyAsync(c->stage_pat, y, sizeof(float2) * n, cudaMemcpyHostToDevice, c->s));
        dy = c->stage_pat;
    }
    pty::PatternArgs a = pattern_args(c);
    CK(c->impl->adjoint(a, dy, c->w, c->s));
    CK(scatter(c, a, scatter_plan(c), c->stage_obj, 0, nullptr, nullptr));
    float *xo[1] = {x};
    if ((st = views_out(c, xo, c->stage_obj))) return st;
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    if ((st = sync(c))) return st;
    return check_wait_error(c, herr);
}

int pty_gradient(pty_ctx *c, const float *psi, float *grad, double *F)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!psi) return fail(c, PTY_ERR_ARG, "psi must be non-NULL");
    if (c->V != 1) return fail(c, PTY_ERR_UNSUPPORTED, "pty_gradient works on single-view contexts");
    int st;
    if ((st = enter(c)) || (st = ensure_stage(c))) return st;
    if ((st = views_in(c, &psi, c->stage_obj))) return st;
    pty::PatternArgs a = pattern_args(c);
    c->cache_dirty = true;  // the pass below overwrites u at the entries
    if (c->opts.dft != 0) {
        if ((st = tc_grad(c, c->stage_obj, nullptr))) return st;
    } else {
        CK(c->impl->grad(a, c->stage_obj, c->w, c->fpart, nullptr, c->s));
    }
    CK(scatter(c, a, scatter_plan(c), c->stage_obj2, 0, nullptr, nullptr));
    const int fcols = c->opts.dft != 0 ? 0 : c->impl->grad_cols(a);
    CK(pty::launch_sum(c->fpart, fcols > 0 ? fcols : c->K * c->CS, c->dscalar, c->s));
    if (grad) {
        float *go[1] = {grad};
        if ((st = views_out(c, go, c->stage_obj2))) return st;
    }
    double hF = 0.0;
    int herr = 0;
    CK(cudaMemcpyAsync(&hF, c->dscalar, sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(&herr, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    if ((st = sync(c))) return st;
    if ((st = check_wait_error(c, herr))) return st;
    if (F) *F = hF;
    return PTY_OK;
}

int pty_cg_reset(pty_ctx *c)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    int st;
    if ((st = enter(c))) return st;
    const size_t HW = (size_t)c->HA * c->WA;
    CK(cudaMemsetAsync(c->g_prev, 0, sizeof(float2) * HW, c->s));
    CK(cudaMemsetAsync(c->eta_prev, 0, sizeof(float2) * HW, c->s));
    CK(cudaMemsetAsync(c->st, 0, sizeof(DevState) * c->V, c->s));
    return sync(c);
}

int pty_cg_solve(pty_ctx *c, float *psi_inout, int32_t niter, pty_cg_report *rep)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!psi_inout || niter < 0) return fail(c, PTY_ERR_ARG, "psi must be non-NULL and niter >= 0");
    if (c->V != 1) return fail(c, PTY_ERR_UNSUPPORTED, "use pty_batch_cg_solve for a batch of views");
    float *p[1] = {psi_inout};
    return solve(c, p, niter, rep);
}

int pty_batch_cg_solve(pty_ctx *c, float *const *psi, int32_t niter, pty_cg_report *reps)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!psi || niter < 0) return fail(c, PTY_ERR_ARG, "psi must be non-NULL and niter >= 0");
    for (int v = 0; v < c->V; v++)
        if (!psi[v]) return fail(c, PTY_ERR_ARG, "psi[%d] is NULL", v);
    return solve(c, psi, niter, reps);
}

int32_t pty_num_views(const pty_ctx *c) { return c ? c->V : 0; }

// Checkpoint layout: header {magic, H*W of the atlas, views, entries} (4 x int64), g_prev,
// eta_prev, the per-view DevState, then u and v at the entries (the linear form's cache).
namespace {
constexpr long long kStateMagic = 0x5054594347310003LL;
size_t state_bytes(const pty_ctx *c)
{
    const size_t HW = (size_t)c->HA * c->WA, E = (size_t)std::max<long long>(c->n_entries, 0);
    return 4 * sizeof(long long) + 2 * sizeof(float2) * HW + sizeof(DevState) * c->V + 2 * sizeof(float2) * E;
}
}  // namespace

size_t pty_cg_state_size(const pty_ctx *c)
{
    if (!c) return 0;
    return state_bytes(c);
}

int pty_cg_state_save(pty_ctx *c, void *host_buf)
{
    if (!c || !host_buf) return fail(c, PTY_ERR_ARG, "ctx and buffer must be non-NULL");
    int st;
    if ((st = enter(c))) return st;
    const size_t HW = (size_t)c->HA * c->WA, E = (size_t)std::max<long long>(c->n_entries, 0);
    char *b = (char *)host_buf;
    const long long hdr[4] = {kStateMagic, (long long)HW, (long long)c->V, (long long)E};
    std::memcpy(b, hdr, sizeof hdr);
    b += sizeof hdr;
    CK(cudaMemcpyAsync(b, c->g_prev, sizeof(float2) * HW, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(b + sizeof(float2) * HW, c->eta_prev, sizeof(float2) * HW, cudaMemcpyDeviceToHost, c->s));
    char *bs = b + 2 * sizeof(float2) * HW;
    CK(cudaMemcpyAsync(bs, c->st, sizeof(DevState) * c->V, cudaMemcpyDeviceToHost, c->s));
    char *be = bs + sizeof(DevState) * c->V;
    if (E) {
        CK(cudaMemcpyAsync(be, c->nz_u, sizeof(float2) * E, cudaMemcpyDeviceToHost, c->s));
        CK(cudaMemcpyAsync(be + sizeof(float2) * E, c->nz_v, sizeof(float2) * E, cudaMemcpyDeviceToHost, c->s));
    }
    if ((st = sync(c))) return st;
    if (c->cache_dirty) {  // the entries were overwritten since the last solve: no linear carry-over
        std::vector<DevState> hs(c->V);
        std::memcpy(hs.data(), bs, sizeof(DevState) * c->V);
        for (auto &h : hs) h.lin = 0;
        std::memcpy(bs, hs.data(), sizeof(DevState) * c->V);
    }
    return PTY_OK;
}

int pty_cg_state_load(pty_ctx *c, const void *host_buf)
{
    if (!c || !host_buf) return fail(c, PTY_ERR_ARG, "ctx and buffer must be non-NULL");
    int st;
    if ((st = enter(c))) return st;
    const size_t HW = (size_t)c->HA * c->WA, E = (size_t)std::max<long long>(c->n_entries, 0);
    const char *b = (const char *)host_buf;
    long long hdr[4];
    std::memcpy(hdr, b, sizeof hdr);
    if (hdr[0] != kStateMagic || hdr[1] != (long long)HW || hdr[2] != (long long)c->V || hdr[3] != (long long)E)
        return fail(c, PTY_ERR_ARG, "checkpoint does not belong to a problem of this context's sizes");
    b += sizeof hdr;
    std::vector<DevState> hs(c->V);
    std::memcpy(hs.data(), b + 2 * sizeof(float2) * HW, sizeof(DevState) * c->V);
    for (auto &h : hs) {
        h.m = 0;
        h.decided = 0;
        h.stalled = 0;
    }
    const char *be = b + 2 * sizeof(float2) * HW + sizeof(DevState) * c->V;
    CK(cudaMemcpyAsync(c->g_prev, b, sizeof(float2) * HW, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->eta_prev, b + sizeof(float2) * HW, sizeof(float2) * HW, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->st, hs.data(), sizeof(DevState) * c->V, cudaMemcpyHostToDevice, c->s));
    if (E) {
        CK(cudaMemcpyAsync(c->nz_u, be, sizeof(float2) * E, cudaMemcpyHostToDevice, c->s));
        CK(cudaMemcpyAsync(c->nz_v, be + sizeof(float2) * E, sizeof(float2) * E, cudaMemcpyHostToDevice, c->s));
    }
    c->cache_dirty = false;
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

int pty_stage_times(pty_ctx *c, double ms[5], int64_t launches[5], int reset)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    for (int i = 0; i < 5; i++) {
        if (ms) ms[i] = c->stage_ms[i];
        if (launches) launches[i] = c->stage_n[i];
    }
    if (reset)
        for (int i = 0; i < 5; i++) {
            c->stage_ms[i] = 0;
            c->stage_n[i] = 0;
        }
    return PTY_OK;
}

}  // extern "C"

namespace {
// Probe-weighted stitching into c->stage_obj (atlas layout); c->st_den keeps sum_k |p/P|^2.
int stitch_into_stage(pty_ctx *c, const float2 *patches, float floor_)
{
    int st;
    if ((st = enter(c)) || (st = ensure_stage(c))) return st;
    const int ntiles = c->ntile_x * c->ntile_y;
    if (!c->st_den) CK(dalloc(&c->st_den, (size_t)c->HA * c->WA));
    if (!c->st_tmax) CK(dalloc(&c->st_tmax, (size_t)ntiles + 1));
    CK(pty::cnn::launch_stitch(c->P, pattern_args(c), scatter_plan(c), patches, floor_, c->stage_obj2, c->st_den,
                               c->st_tmax, c->st_tmax + ntiles, c->stage_obj, c->s));
    return PTY_OK;
}
}  // namespace

int pty::cnn::stitch_scaled(pty_ctx *c, const float2 *patches, float floor_, const double *sum_d, float2 *out,
                            double *c_out)
{
    int st;
    if ((st = stitch_into_stage(c, patches, floor_))) return st;
    if (!c->st_red) CK(dalloc(&c->st_red, (size_t)pty::cnn::kPartials + 2));
    const size_t n = (size_t)c->HA * c->WA;
    double *A = c->st_red + pty::cnn::kPartials;
    // sum |G psi|^2 = P^2 sum_x |psi(x)|^2 sum_k |p(x - r_k) / P|^2 (the stored probe is p / P)
    CK(pty::cnn::launch_sum_sq_weighted(c->stage_obj, c->st_den, n, c->st_red, A, (double)c->P * c->P, c->s));
    CK(pty::cnn::launch_scale_to(c->stage_obj, n, sum_d, A, A + 1, c->s));
    float *po[1] = {(float *)out};
    if ((st = views_out(c, po, c->stage_obj))) return st;
    double hc = 1.0;
    CK(cudaMemcpyAsync(&hc, A + 1, sizeof(double), cudaMemcpyDeviceToHost, c->s));
    if ((st = sync(c))) return st;
    if (c_out) *c_out = hc;
    return PTY_OK;
}

extern "C" {

int pty_stitch(pty_ctx *c, const float *patches, float floor_, float *psi0)
{
    if (!c) return fail(nullptr, PTY_ERR_ARG, "ctx is NULL");
    if (!patches || !psi0) return fail(c, PTY_ERR_ARG, "patches and psi0 must be non-NULL");
    if (!(floor_ >= 0.f) || !std::isfinite(floor_)) return fail(c, PTY_ERR_ARG, "floor must be finite and >= 0");
    if (c->V != 1) return fail(c, PTY_ERR_UNSUPPORTED, "pty_stitch works on single-view contexts");
    if (!is_device_ptr(patches)) return fail(c, PTY_ERR_ARG, "patches must be a device array");
    int st;
    if ((st = stitch_into_stage(c, (const float2 *)patches, floor_))) return st;
    float *po[1] = {psi0};
    if ((st = views_out(c, po, c->stage_obj))) return st;
    return sync(c);
}

}  // extern "C"

namespace pty {
int ctx_info(const pty_ctx *c, int *H, int *W, int *P, int *K, int *V, int *dev)
{
    if (!c) return PTY_ERR_ARG;
    *H = c->Hv.empty() ? 0 : c->Hv[0];
    *W = c->Wv.empty() ? 0 : c->Wv[0];
    *P = c->P;
    *K = c->K;
    *V = c->V;
    *dev = c->dev;
    return PTY_OK;
}
}  // namespace pty

#include "pty_selftest.h"

extern "C" int pty_selftest_tc_wait_limit(int64_t polls)
{
    pty::tc_set_wait_limit((long long)polls);
    return PTY_OK;
}

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

extern "C" int pty_selftest_ls_certified(pty_ctx *c, int32_t view, int32_t *k0cert)
{
    if (!c || !k0cert || view < 0 || view >= c->V) return fail(c, PTY_ERR_ARG, "bad arguments");
    if (enter(c) != PTY_OK) return PTY_ERR_CUDA;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, (const char *)(c->st + view) + offsetof(pty::DevState, k0cert), sizeof(int),
                                    cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return fail(c, PTY_ERR_CUDA, "selftest: %s", cudaGetErrorString(e));
    *k0cert = c->cert ? v : 0;
    return PTY_OK;
}

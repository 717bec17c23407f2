// object_kernels.cu -- object-sized steps of ML-CG and the small scalar kernels.
//
//   k_scatter     Q^H of Eq. 3: the patch-sized results of all positions are summed into
//                 the object.  One thread block owns one object tile and walks the
//                 position-sorted list of patterns that overlap it (built once on the
//                 host), accumulating in registers in that fixed order: no atomics, and
//                 bitwise reproducible.  Optionally fuses the two reductions of the
//                 Dai-Yuan coefficient (Eq. 6): ||g||^2 and Re <eta_prev, g - g_prev>.
//   k_dy_finalize DIR stage scalars (Eq. 6, with the restart rule) and F(psi_m) (Eq. 2).
//   k_ls_certify  LS stage: leading trials rejected by the Jensen lower bound of the
//                 objective change, then the first exact window.
//   k_ls_decide   LS stage decision (Eq. 7): the first candidate of the window that does
//                 not increase the objective, else open the next window or stall.
//   k_update      Update stage (Eq. 5): psi += gamma eta, keeping eta and g for Eq. 6.
// All sums of partials run in float-float (reduce.cuh) in a fixed order; the scalar
// decisions are taken in FP64 from them.
#include <cmath>

#include "pty_internal.h"
#include "reduce.cuh"
#include "scatter_tail.cuh"

namespace pty {

#ifndef PTY_SCATTER_LD
#define PTY_SCATTER_LD __ldcs  // load of the per-pattern results: read once, evict first
#endif

namespace {
constexpr int kScTY = kTileY, kScTX = kTileX, kScNT = 256, kScNJ = kScTY * kScTX / kScNT;
constexpr int kSumNT = 256;
}  // namespace

template <int P>
__global__ void __launch_bounds__(kScNT) k_scatter(PatternArgs a, ScatterPlan plan, const float2 *__restrict__ w,
                                                   float2 *__restrict__ out, int dy, const float2 *__restrict__ ep,
                                                   const float2 *__restrict__ gp, float2 *__restrict__ part,
                                                   const DevState *__restrict__ st, const float2 *__restrict__ psi,
                                                   const float *__restrict__ D, float p2)
{
    const int b = blockIdx.x;
    if (st && st[plan.tile_view[b]].stalled) return;
    const bool lin = st && st[plan.tile_view[b]].lin;
    __shared__ float2 red[(kScNT / 32) * 3];
    __shared__ float2 tot[3];
    const int ty = b / plan.ntile_x, tx = b % plan.ntile_x;
    const int x = tx * kScTX + (threadIdx.x % kScTX);
    const int y0 = ty * kScTY + threadIdx.x / kScTX;
    float2 acc[kScNJ];
#pragma unroll
    for (int j = 0; j < kScNJ; j++) acc[j] = make_float2(0.f, 0.f);
    const int q0 = plan.tile_start[b], q1 = plan.tile_start[b + 1];
    for (int q = q0; q < q1; q++) {
        const int i = __ldg(plan.tile_list + q);
        const int2 rc = __ldg(a.pos + i);
        const int dx = x - rc.y;
        if (dx < 0 || dx >= P) continue;
        const float2 *wi = w + (size_t)i * P * P + dx;
#pragma unroll
        for (int j = 0; j < kScNJ; j++) {
            const int yy = y0 + (kScNT / kScTX) * j - rc.x;
            if (yy >= 0 && yy < P) {
                const float2 v = PTY_SCATTER_LD(wi + yy * P);
                acc[j].x += v.x;
                acc[j].y += v.y;
            }
        }
    }
    scatter_tail<kScNT, kScNJ, kScNT / kScTX>(a, acc, x, y0, b, lin, out, dy, ep, gp, part, psi, D, p2, red, tot);
}

// Illumination map D(x) = sum over positions k covering x of |p_k(x - r_k)|^2 (p_k the
// stored probe of position k, i.e. the probe / P), per object tile from the same
// position-sorted lists.
template <int P>
__global__ void __launch_bounds__(kScNT) k_illum(PatternArgs a, ScatterPlan plan, float *__restrict__ D)
{
    const int b = blockIdx.x;
    const int ty = b / plan.ntile_x, tx = b % plan.ntile_x;
    const int x = tx * kScTX + (threadIdx.x % kScTX);
    const int y0 = ty * kScTY + threadIdx.x / kScTX;
    float acc[kScNJ];
#pragma unroll
    for (int j = 0; j < kScNJ; j++) acc[j] = 0.f;
    for (int q = plan.tile_start[b]; q < plan.tile_start[b + 1]; q++) {
        const int i = __ldg(plan.tile_list + q);
        const int2 rc = __ldg(a.pos + i);
        const int dx = x - rc.y;
        if (dx < 0 || dx >= P) continue;
        const float2 *pk = probe_of(a, i);
#pragma unroll
        for (int j = 0; j < kScNJ; j++) {
            const int yy = y0 + (kScNT / kScTX) * j - rc.x;
            if (yy >= 0 && yy < P) {
                const float2 p = __ldg(pk + yy * P + dx);
                acc[j] += p.x * p.x + p.y * p.y;
            }
        }
    }
    if (x >= a.W) return;
#pragma unroll
    for (int j = 0; j < kScNJ; j++) {
        const int y = y0 + (kScNT / kScTX) * j;
        if (y < a.H) D[(size_t)y * a.W + x] = acc[j];
    }
}

// Search direction of Eq. 6, eta = -g + alpha eta_prev (alpha of the tile's view), and the
// view's real-space sums that Parseval's identity turns into the line search's totals over
// all detector pixels: part[b] = (sum D Re conj(psi) eta, sum D |eta|^2) over tile b.
__global__ void __launch_bounds__(kScNT) k_eta(int H, int W, ScatterPlan plan, const float2 *__restrict__ psi,
                                               const float2 *__restrict__ g, const float2 *__restrict__ ep,
                                               const float *__restrict__ D, float2 *__restrict__ eta,
                                               float2 *__restrict__ part, const DevState *__restrict__ sts)
{
    const int b = blockIdx.x;
    const DevState *st = sts + plan.tile_view[b];
    if (st->stalled) return;
    __shared__ float2 red[(kScNT / 32) * 2];
    __shared__ float2 tot[2];
    const int ty = b / plan.ntile_x, tx = b % plan.ntile_x;
    const int x = tx * kScTX + (threadIdx.x % kScTX);
    const int y0 = ty * kScTY + threadIdx.x / kScTX;
    const float alpha = st->alpha_f;
    float s0 = 0.f, s1 = 0.f;
    if (x < W) {
#pragma unroll
        for (int j = 0; j < kScNJ; j++) {
            const int y = y0 + (kScNT / kScTX) * j;
            if (y < H) {
                const size_t o = (size_t)y * W + x;
                const float2 gv = __ldg(g + o), ev = __ldg(ep + o), pv = __ldg(psi + o);
                const float2 e = make_float2(fmaf(alpha, ev.x, -gv.x), fmaf(alpha, ev.y, -gv.y));
                eta[o] = e;
                const float dd = __ldg(D + o);
                s0 = fmaf(dd, fmaf(pv.x, e.x, pv.y * e.y), s0);
                s1 = fmaf(dd, fmaf(e.x, e.x, e.y * e.y), s1);
            }
        }
    }
    float v[2] = {s0, s1};
    block_sum_ff<kScNT, 2>(v, red, tot);
    if (threadIdx.x < 2) part[2 * b + threadIdx.x] = tot[threadIdx.x];
}

// Each thread sums a fixed strided subset, then the block combines: fixed order.
__device__ __forceinline__ float2 strided_sum(const float2 *v, int n, int stride, int off)
{
    float2 s = make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < n; i += kSumNT) s = ff_add(s, v[(size_t)i * stride + off]);
    return s;
}

__global__ void __launch_bounds__(kSumNT) k_sum(const float2 *__restrict__ v, int n, double *__restrict__ out)
{
    __shared__ float2 red[kSumNT / 32];
    __shared__ float2 tot[1];
    float2 x[1] = {strided_sum(v, n, 1, 0)};
    block_sum_ff<kSumNT, 1>(x, red, tot);
    if (threadIdx.x == 0) *out = ff_value(tot[0]);
}

__device__ __forceinline__ void open_window(DevState *st, double gamma0, double tau)
{
    // candidates gamma0 tau^(k0 + l + 1), l < Leff
    double g = gamma0;
    for (int k = 0; k < st->k0; k++) g *= tau;
    for (int l = 0; l < st->Leff; l++) {
        g *= tau;
        st->cand[l] = g;
        st->cand_f[l] = (float)g;
    }
}

__global__ void __launch_bounds__(kSumNT) k_dy_finalize(const float2 *__restrict__ fpart, int cs, int fcols,
                                                        const float2 *__restrict__ part, double p2, ViewMap vm,
                                                        DevState *sts, DevHist h, LsArgs ls)
{
    const int v = blockIdx.x;
    DevState *st = sts + v;
    if (st->stalled) return;
    __shared__ float2 red[(kSumNT / 32) * 4];
    __shared__ float2 tot[4];
    const int f0 = fcols > 0 ? 0 : vm.pat_off[v] * cs, f1 = fcols > 0 ? fcols : vm.pat_off[v + 1] * cs;
    const int t0 = vm.tile_off[v], t1 = vm.tile_off[v + 1];
    float2 v4[4] = {strided_sum(fpart + f0, f1 - f0, 1, 0), strided_sum(part + 3 * (size_t)t0, t1 - t0, 3, 0),
                    strided_sum(part + 3 * (size_t)t0, t1 - t0, 3, 1), strided_sum(part + 3 * (size_t)t0, t1 - t0, 3, 2)};
    block_sum_ff<kSumNT, 4>(v4, red, tot);
    if (threadIdx.x == 0) {
        // linear form: sum |u|^2 over all pixels = P^2 sum D |psi|^2 (0 from the tiles otherwise)
        const double Fm = ff_value(tot[0]) + p2 * ff_value(tot[3]), gg = ff_value(tot[1]), den = ff_value(tot[2]);
        double alpha = 0.0;
        if (ls.gd) {
            // Eq. 4: the step follows -grad F alone
        } else if (den > 0.0 && isfinite(den) && isfinite(gg)) {
            alpha = gg / den;
        } else if (st->total > 0) {
            st->restarts += 1;
        }
        st->alpha = alpha;
        st->alpha_f = (float)alpha;
        st->Fm = Fm;
        st->k0 = 0;
        st->decided = 0;
        // first window: the previous iteration's trial count plus one (adaptive), or L
        int Le = ls.L;
        if (ls.adaptive) {
            Le = st->last_halvings > 0 ? st->last_halvings + 1 : 16;
            Le = Le < 4 ? 4 : (Le > ls.L ? ls.L : Le);
        }
        st->Leff = Le;
        st->Lsel = ls.adaptive ? (Le <= 16 ? 16 : 32) : ls.L;
        st->k0cert = 0;
        st->kwarm = 0;
        if (ls.warm && st->total > 0 && st->last_halvings > 0) {
            // warm start: the search begins at gamma0 tau^(last - 1) = gamma_prev / tau, so
            // its first trial is the previous accepted step gamma0 tau^last; the first window
            // holds the previous search's distance to its accepted trial plus two candidates
            const int kw = st->last_halvings - 1;
            st->k0 = kw;
            st->kwarm = kw;
            if (ls.adaptive) {
                const int Lw = st->last_excess + 2;
                const int Ls = Lw <= 4 ? 4 : (Lw <= 8 ? 8 : (Lw <= 16 ? 16 : 32));
                st->Leff = Ls < ls.L ? Ls : ls.L;
                st->Lsel = st->Leff;
            }
        }
        open_window(st, ls.gamma0, ls.tau);
        double gj = ls.gamma0;  // the leading trials for the certificate rows of the LS pass
        for (int j = 0; j < kCertN; j++) {
            gj *= ls.tau;
            st->cert_f[j] = (float)gj;
        }
        const int m = st->m;
        if (m < h.cap) {
            h.F[(size_t)v * (h.cap + 1) + m] = Fm;
            h.alpha[(size_t)v * h.cap + m] = alpha;
        }
    }
}

// Rows of partials have length kc; view v's entries are [pat_off[v] cs, pat_off[v+1] cs).
// The open window of view v has st->Leff <= 32 candidates.
// Sum of n doubles v[0], v[stride], ... by one warp in a fixed order: each lane keeps four
// accumulators over a fixed strided subset, then a butterfly across the warp.
__device__ __forceinline__ float2 warp_strided_sum(const float2 *__restrict__ v, int n, int lane)
{
    float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
    int i = lane;
    for (; i + 96 < n; i += 128) {
        s0 = ff_add(s0, v[i]);
        s1 = ff_add(s1, v[i + 32]);
        s2 = ff_add(s2, v[i + 64]);
        s3 = ff_add(s3, v[i + 96]);
    }
    for (; i < n; i += 32) s0 = ff_add(s0, v[i]);
    return warp_sum_ff(ff_add(ff_add(s0, s1), ff_add(s2, s3)));
}

constexpr int kDecNT = 1024;

__global__ void __launch_bounds__(kDecNT) k_ls_decide(const float2 *__restrict__ part, int kc, int cs, int ls_cols,
                                                      int en_cols, ViewMap vm, const float2 *__restrict__ vpart,
                                                      double vscale, DevState *sts, DevHist h, LsArgs ls)
{
    const int v = blockIdx.x;
    DevState *st = sts + v;
    if (st->stalled || st->decided) return;
    __shared__ double tot[32 + 2];
    __shared__ double vtot[2];
    // warp w sums rows j = w, w + 32, ... of the view's partials (fixed order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Leff = st->Leff;
    const int p0 = vm.pat_off[v] * cs, p1 = vm.pat_off[v + 1] * cs;
    for (int j = warp; j < Leff + 2; j += kDecNT / 32) {
        const int nc = j < 2 ? ls_cols : en_cols;  // per-CTA columns (one view) or the view's range
        const float2 s = nc > 0 ? warp_strided_sum(part + (size_t)j * kc, nc, lane)
                                : warp_strided_sum(part + (size_t)j * kc + p0, p1 - p0, lane);
        if (lane == 0) tot[j] = ff_value(s);
    }
    // the view's object-tile sums of the all-pixel totals of rows 0 and 1 (Parseval)
    if (vpart && warp >= 30) {
        const int j = warp - 30, t0 = vm.tile_off[v], n = vm.tile_off[v + 1] - t0;
        float2 t0s = make_float2(0.f, 0.f);
        for (int b = lane; b < n; b += 32) t0s = ff_add(t0s, vpart[2 * (t0 + b) + j]);
        t0s = warp_sum_ff(t0s);
        if (lane == 0) vtot[j] = vscale * ff_value(t0s);
    }
    __syncthreads();
    if (vpart && threadIdx.x < 2) tot[threadIdx.x] += vtot[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        // trials are counted from the start of this search (kwarm trials skipped by a warm start)
        const int m = st->m, k0 = st->k0, kw = st->kwarm;
        const size_t hf = (size_t)v * (h.cap + 1) + m, hi = (size_t)v * h.cap + m;
        for (int l = 0; l < Leff && k0 + l + 1 - kw <= ls.max_halvings; l++) {
            const double gam = st->cand[l];
            // F(psi + gam eta) - F(psi): quadratic part of the d = 0 pixels plus the rest
            const double dF = gam * (2.0 * tot[0] + gam * tot[1]) + tot[2 + l];
            if (dF <= gam * ls.t) {
                st->gamma = gam;
                st->gamma_f = (float)gam;
                st->Fnext = st->Fm + dF;
                st->decided = 1;
                st->last_halvings = k0 + l + 1;  // gamma = gamma0 tau^last_halvings
                st->last_excess = k0 + l - st->k0cert - kw;
                if (m < h.cap) {
                    h.gamma[hi] = gam;
                    h.halvings[hi] = k0 + l + 1 - kw;
                    h.F[hf + 1] = st->Fm + dF;
                }
                return;
            }
        }
        const int k1 = k0 + Leff;
        if (k1 - kw >= ls.max_halvings) {
            st->stalled = 1;
            if (m < h.cap) {
                h.gamma[hi] = st->cand[ls.max_halvings - 1 - (k0 - kw)];
                h.halvings[hi] = ls.max_halvings;
                h.F[hf + 1] = st->Fm;
            }
        } else {
            st->k0 = k1;
            st->Leff = ls.L;  // later windows use the full capacity
            st->Lsel = ls.L;
            open_window(st, ls.gamma0, ls.tau);
        }
    }
}

// Certified rejection of the leading trials of Algorithm 1's backtracking (Eq. 7).  The LS
// pass wrote, per (pattern, chunk), a lower bound of the entries' share of the objective change
// at each of the first kCertN trials (Jensen's inequality on the concave log1p, see
// ls_cert_rows) and its magnitude; with the pixels without counts (rows 0, 1 plus the object
// sums, exact) the view's bound is LB_j <= F(psi + gamma_j eta) - F(psi).  Every leading trial
// with LB_j above the acceptance threshold gamma_j t by more than a rounding margin would be
// rejected by the plain search, so the first window opens at the first trial the bound cannot
// reject; its size (6, 8, 16 or 32 trials) follows the previous iteration's distance between that
// trial and the accepted one.  Accepted step and trial count are those of the plain search.
__global__ void __launch_bounds__(kDecNT) k_ls_certify(const float2 *__restrict__ part, int kc, int cs, int ls_cols,
                                                       ViewMap vm, const float2 *__restrict__ vpart, double vscale,
                                                       DevState *sts, LsArgs ls)
{
    const int v = blockIdx.x;
    DevState *st = sts + v;
    if (st->stalled) return;
    constexpr int NR = 2 + 2 * kCertN;
    __shared__ double tot[NR];
    __shared__ double vtot[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p0 = ls_cols > 0 ? 0 : vm.pat_off[v] * cs, p1 = ls_cols > 0 ? ls_cols : vm.pat_off[v + 1] * cs;
    for (int j = warp; j < NR; j += kDecNT / 32) {
        const float2 s = warp_strided_sum(part + (size_t)j * kc + p0, p1 - p0, lane);
        if (lane == 0) tot[j] = ff_value(s);
    }
    if (vpart && warp >= 30) {
        const int j = warp - 30, t0 = vm.tile_off[v], n = vm.tile_off[v + 1] - t0;
        float2 t0s = make_float2(0.f, 0.f);
        for (int b = lane; b < n; b += 32) t0s = ff_add(t0s, vpart[2 * (t0 + b) + j]);
        t0s = warp_sum_ff(t0s);
        if (lane == 0) vtot[j] = vscale * ff_value(t0s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (vpart) {
            tot[0] += vtot[0];
            tot[1] += vtot[1];
        }
        int k0 = 0;
        double g = ls.gamma0;
        for (; k0 < kCertN && k0 + 1 < ls.max_halvings; k0++) {
            g *= ls.tau;
            const double quad = g * (2.0 * tot[0] + g * tot[1]);  // pixels without counts
            const double lb = quad + tot[2 + k0];
            const double margin = 1e-4 * (fabs(quad) + tot[2 + kCertN + k0]);
            if (!(lb > g * ls.t + margin)) break;  // NaN rows give no certificate
        }
        st->k0 = k0;
        st->k0cert = k0;
        const int Le = st->last_halvings > 0 ? st->last_excess + 2 : 16;
        const int Ls = Le <= 6 ? 6 : (Le <= 8 ? 8 : (Le <= 16 ? 16 : 32));
        st->Leff = Ls;
        st->Lsel = Ls;
        open_window(st, ls.gamma0, ls.tau);
    }
}

// Sum of the counts of each (pattern, chunk): one block per chunk, FP64 (once per problem).
__global__ void __launch_bounds__(kSumNT) k_chunk_dsum(PatternArgs a, int cs, float *__restrict__ dsum)
{
    __shared__ double red[kSumNT / 32];
    __shared__ double tot[1];
    const int i = blockIdx.x / cs, c = blockIdx.x % cs, per = a.nzc / cs;
    const long long e0 = a.nz_off[(size_t)i * a.nzc + c * per], e1 = a.nz_off[(size_t)i * a.nzc + (c + 1) * per];
    double sum = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += kSumNT) sum += a.nz_d[e];
    double v[1] = {sum};
    block_sum<kSumNT, 1>(v, red, tot);
    if (threadIdx.x == 0) dsum[blockIdx.x] = (float)tot[0];
}

__global__ void k_update(int H, int W, ViewMap vm, float2 *__restrict__ psi, const float2 *__restrict__ g,
                         float2 *__restrict__ ep, float2 *__restrict__ gp, const DevState *sts)
{
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const DevState *st = sts + vm.row_view[i / W];
        if (st->stalled || !st->decided) continue;
        const float gam = st->gamma_f, alpha = st->alpha_f;
        const float2 gv = g[i], ev = ep[i];
        const float2 eta = make_float2(fmaf(alpha, ev.x, -gv.x), fmaf(alpha, ev.y, -gv.y));
        float2 p = psi[i];
        p.x = fmaf(gam, eta.x, p.x);
        p.y = fmaf(gam, eta.y, p.y);
        psi[i] = p;
        ep[i] = eta;
        gp[i] = gv;
    }
}

// Gradient descent (Eq. 4): psi_{m+1} = psi_m - gamma grad F(psi_m) with the constant step
// gamma; k_update then applies it with alpha = 0 (eta = -g).
__global__ void k_gd_step(ViewMap vm, DevState *sts, DevHist h, LsArgs ls)
{
    for (int v = threadIdx.x; v < vm.V; v += blockDim.x) {
        DevState *st = sts + v;
        if (st->stalled) continue;
        st->gamma = ls.gd_step;
        st->gamma_f = (float)ls.gd_step;
        st->decided = 1;
        st->last_halvings = 0;
        const int m = st->m;
        if (m < h.cap) {
            h.gamma[(size_t)v * h.cap + m] = ls.gd_step;
            h.halvings[(size_t)v * h.cap + m] = 0;
        }
    }
}

// F(psi) of each view (full-form GRAD partials) into the history slot of the current count.
__global__ void __launch_bounds__(kSumNT) k_objective_to_hist(const float2 *__restrict__ fpart, int cs, int fcols,
                                                              ViewMap vm, const DevState *__restrict__ sts, DevHist h)
{
    const int v = blockIdx.x;
    const DevState *st = sts + v;
    __shared__ float2 red[kSumNT / 32];
    __shared__ float2 tot[1];
    const int f0 = fcols > 0 ? 0 : vm.pat_off[v] * cs, f1 = fcols > 0 ? fcols : vm.pat_off[v + 1] * cs;
    float2 x[1] = {strided_sum(fpart + f0, f1 - f0, 1, 0)};
    block_sum_ff<kSumNT, 1>(x, red, tot);
    if (threadIdx.x == 0 && !st->stalled && st->m <= h.cap) h.F[(size_t)v * (h.cap + 1) + st->m] = ff_value(tot[0]);
}

// lin_period > 0: the next GRAD pass runs in the linear form unless the total iteration
// count is a multiple of lin_period (a full forward DFT then bounds the drift of u).
__global__ void k_update_counters(DevState *sts, int V, int lin_period)
{
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        DevState *st = sts + v;
        if (st->stalled || !st->decided) continue;
        st->m += 1;
        st->total += 1;
        st->last_gamma = st->gamma;
        st->lin = lin_period > 0 && (st->total % lin_period) != 0;
    }
}

// Order-independent 64-bit hash of each view's object: the sum modulo 2^64 of a mixed
// (index, value bits) key per pixel (splitmix64 finaliser, Steele, Lea, Flood 2014).
__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__global__ void __launch_bounds__(256) k_hash(int W, const int *__restrict__ row_view, const float2 *__restrict__ psi,
                                              unsigned long long *__restrict__ out)
{
    // one block per object row: a row belongs to one view; one atomic add per row
    __shared__ unsigned long long red[8];
    const int y = blockIdx.x;
    unsigned long long h = 0;
    for (int x = threadIdx.x; x < W; x += 256) {
        const size_t i = (size_t)y * W + x;
        const float2 v = psi[i];
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(v.x) << 32 | __float_as_uint(v.y)) ^ mix64(i);
        h += mix64(key);  // integer sum: exact in any order
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = h;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < 8; k++) t += red[k];
        atomicAdd(out + row_view[y], t);
    }
}

// Start of a solve call: the entries' u and v stay usable only if every view's object is
// the one the previous call ended with (and nothing else overwrote them: force == 0).
__global__ void k_check_hash(DevState *sts, int V, const unsigned long long *__restrict__ h, int force)
{
    for (int v = threadIdx.x; v < V; v += blockDim.x)
        if (force || h[v] != sts[v].psi_hash) sts[v].lin = 0;
}

__global__ void k_store_hash(DevState *sts, int V, const unsigned long long *__restrict__ h)
{
    for (int v = threadIdx.x; v < V; v += blockDim.x) sts[v].psi_hash = h[v];
}

__global__ void k_check_data(const float *__restrict__ d, size_t n, int *flag)
{
    int bad = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = d[i];
        bad |= !(v >= 0.0f) || isinf(v);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void k_begin_solve(DevState *sts, int V)
{
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        sts[v].m = 0;
        sts[v].stalled = 0;
        sts[v].decided = 0;
    }
}

// ------------------------------------------------------------------------------------
cudaError_t launch_scatter(int P, const PatternArgs &a, const ScatterPlan &plan, const float2 *w, float2 *out,
                           int dy, const float2 *eta_prev, const float2 *g_prev, float2 *part, const DevState *st,
                           cudaStream_t s, const float2 *psi, const float *D)
{
    const float p2 = (float)P * (float)P;
    const int nb = plan.ntile_x * plan.ntile_y;
    switch (P) {
    case 64: k_scatter<64><<<nb, kScNT, 0, s>>>(a, plan, w, out, dy, eta_prev, g_prev, part, st, psi, D, p2); break;
    case 128: k_scatter<128><<<nb, kScNT, 0, s>>>(a, plan, w, out, dy, eta_prev, g_prev, part, st, psi, D, p2); break;
    case 256: k_scatter<256><<<nb, kScNT, 0, s>>>(a, plan, w, out, dy, eta_prev, g_prev, part, st, psi, D, p2); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_illumination(int P, const PatternArgs &a, const ScatterPlan &plan, float *D, cudaStream_t s)
{
    const int nb = plan.ntile_x * plan.ntile_y;
    switch (P) {
    case 64: k_illum<64><<<nb, kScNT, 0, s>>>(a, plan, D); break;
    case 128: k_illum<128><<<nb, kScNT, 0, s>>>(a, plan, D); break;
    case 256: k_illum<256><<<nb, kScNT, 0, s>>>(a, plan, D); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_eta(int H, int W, const ScatterPlan &plan, const float2 *psi, const float2 *g, const float2 *ep,
                       const float *D, float2 *eta, float2 *part, const DevState *st, cudaStream_t s)
{
    k_eta<<<plan.ntile_x * plan.ntile_y, kScNT, 0, s>>>(H, W, plan, psi, g, ep, D, eta, part, st);
    return cudaGetLastError();
}

cudaError_t launch_sum(const float2 *v, int n, double *out, cudaStream_t s)
{
    k_sum<<<1, kSumNT, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t launch_dy_finalize(const float2 *fpart, int cs, int fcols, const float2 *part, double p2, const ViewMap &vm,
                               DevState *st, DevHist h, const LsArgs &ls, cudaStream_t s)
{
    k_dy_finalize<<<vm.V, kSumNT, 0, s>>>(fpart, cs, fcols, part, p2, vm, st, h, ls);
    return cudaGetLastError();
}

cudaError_t launch_ls_certify(const float2 *part, int kc, int cs, int ls_cols, const ViewMap &vm, const float2 *vpart,
                              double vscale, const LsArgs &ls, DevState *st, cudaStream_t s)
{
    k_ls_certify<<<vm.V, kDecNT, 0, s>>>(part, kc, cs, ls_cols, vm, vpart, vscale, st, ls);
    return cudaGetLastError();
}

// One block per pattern: the bits of its entry slots (PatternArgs::nz_mask).
__global__ void __launch_bounds__(256) k_nz_mask(const long long *__restrict__ off, int nzc,
                                                 const unsigned short *__restrict__ slot, int P,
                                                 unsigned *__restrict__ mask)
{
    const int i = blockIdx.x;
    const long long e0 = off[(size_t)i * nzc], e1 = off[(size_t)(i + 1) * nzc];
    unsigned *m = mask + (size_t)i * (P * P / 32);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int sl = slot[e], qy = sl / P, qx = sl % P;
        atomicOr(m + qx * (P / 32) + qy / 32, 1u << (qy % 32));
    }
}

cudaError_t launch_nz_mask(const PatternArgs &a, int P, unsigned *mask, cudaStream_t s)
{
    if (P % 32 != 0 || a.K < 1) return cudaErrorInvalidValue;
    k_nz_mask<<<a.K, 256, 0, s>>>(a.nz_off, a.nzc, a.nz_slot, P, mask);
    return cudaGetLastError();
}

cudaError_t launch_chunk_dsum(const PatternArgs &a, int cs, float *dsum, cudaStream_t s)
{
    k_chunk_dsum<<<a.K * cs, kSumNT, 0, s>>>(a, cs, dsum);
    return cudaGetLastError();
}

cudaError_t launch_ls_decide(const float2 *part, int kc, int cs, int ls_cols, int en_cols, const ViewMap &vm,
                             const float2 *vpart, double vscale, const LsArgs &ls, DevState *st, DevHist h,
                             cudaStream_t s)
{
    k_ls_decide<<<vm.V, kDecNT, 0, s>>>(part, kc, cs, ls_cols, en_cols, vm, vpart, vscale, st, h, ls);
    return cudaGetLastError();
}

cudaError_t launch_update(int H, int W, const ViewMap &vm, float2 *psi, const float2 *g, float2 *eta_prev,
                          float2 *g_prev, DevState *st, int lin_period, cudaStream_t s)
{
    size_t nb = ((size_t)H * W + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    k_update<<<(unsigned)nb, 256, 0, s>>>(H, W, vm, psi, g, eta_prev, g_prev, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_update_counters<<<1, 32, 0, s>>>(st, vm.V, lin_period);
    return cudaGetLastError();
}

cudaError_t launch_gd_step(const ViewMap &vm, const LsArgs &ls, DevState *st, DevHist h, cudaStream_t s)
{
    k_gd_step<<<1, 32, 0, s>>>(vm, st, h, ls);
    return cudaGetLastError();
}

cudaError_t launch_objective_to_hist(const float2 *fpart, int cs, int fcols, const ViewMap &vm, const DevState *st,
                                     DevHist h, cudaStream_t s)
{
    k_objective_to_hist<<<vm.V, kSumNT, 0, s>>>(fpart, cs, fcols, vm, st, h);
    return cudaGetLastError();
}

cudaError_t launch_check_data(const float *d, size_t n, int *flag, cudaStream_t s)
{
    size_t nb = (n + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    if (nb < 1) nb = 1;
    k_check_data<<<(unsigned)nb, 256, 0, s>>>(d, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_begin_solve(DevState *st, int V, cudaStream_t s)
{
    k_begin_solve<<<1, 32, 0, s>>>(st, V);
    return cudaGetLastError();
}

cudaError_t launch_hash(int H, int W, const int *row_view, const float2 *psi, unsigned long long *h, int V,
                        cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(h, 0, sizeof(unsigned long long) * V, s);
    if (e != cudaSuccess) return e;
    k_hash<<<H, 256, 0, s>>>(W, row_view, psi, h);
    return cudaGetLastError();
}

cudaError_t launch_check_hash(DevState *st, int V, const unsigned long long *h, int force, cudaStream_t s)
{
    k_check_hash<<<1, 32, 0, s>>>(st, V, h, force);
    return cudaGetLastError();
}

cudaError_t launch_store_hash(DevState *st, int V, const unsigned long long *h, cudaStream_t s)
{
    k_store_hash<<<1, 32, 0, s>>>(st, V, h);
    return cudaGetLastError();
}

}  // namespace pty

// pty_internal.h -- declarations shared by the translation units of libpty (not part of
// the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

namespace pty {

// Solver state that lives in device memory so that one CG iteration runs without host
// synchronisation: the line-search decision, the Dai-Yuan coefficient and the stall flag
// are produced and consumed by kernels.
// Leading trials of a line search that the Jensen lower bound of the objective change can
// reject without evaluating them (ls_fft epilogue, k_ls_certify).
constexpr int kCertN = 16;

struct DevState {
    int m;         // iterations accepted in the current pty_cg_solve call
    int k0;        // line-search trials already rejected in the current iteration
    int decided;   // the current iteration's step has been chosen
    int stalled;   // no step within max_halvings: the solve is over
    int total;     // iterations accepted since the last reset (checkpointed)
    int restarts;  // Dai-Yuan restarts (denominator <= 0 or not finite)
    int Leff;      // candidates in the open line-search window
    int last_halvings;  // trials of the last accepted step (sizes the next first window)
    int Lsel;      // capacity of the LS kernel that runs the open window (16 or 32 when adaptive)
    int lin;       // the entries hold u and v of the last accepted step: the next GRAD pass
                   // updates u = u + gamma v in place instead of running the forward DFT
    double alpha;  // Dai-Yuan coefficient of the current iteration (Eq. 6)
    double gamma;  // accepted step of the current iteration
    double Fm;     // F(psi_m)
    double Fnext;  // F(psi_m + gamma eta_m) of the accepted trial
    double last_gamma;
    unsigned long long psi_hash;  // hash of the view's object when the last solve call ended
    double cand[32];  // candidate steps gamma0 tau^(k0+l+1) of the open line-search window
    // FP32 roundings of alpha, gamma and cand for the per-pixel kernels (a double-to-float
    // conversion per thread would run on the slow FP64 pipe)
    float alpha_f, gamma_f;
    float cand_f[32];
    // certified skip of the first line-search trials (ls_fft epilogue + k_ls_certify):
    float cert_f[kCertN];  // gamma0 tau^(j+1), j < kCertN, rounded to FP32
    int k0cert;            // trials of the current iteration rejected by the certificate
    int last_excess;       // accepted trial index minus k0cert, last iteration (window size)
    int kwarm;             // trials the warm-started search skipped this iteration: its first
                           // trial is gamma0 tau^(kwarm + 1), the previous accepted step
};

// Per-call history arrays (device), one block of `cap` iterations per view, indexed by
// DevState::m: F[v * (cap + 1) + m], gamma / halvings / alpha [v * cap + m].
struct DevHist {
    double *F;
    double *gamma;
    int *halvings;
    double *alpha;
    int cap;
};

// Everything a per-pattern kernel needs about the problem.  The measured intensities are
// held as a compact list of the detector pixels with counts ("entries"), per pattern in
// ascending slot order (the permuted order the forward DFT leaves the spectrum in): pixels
// with d = 0 enter the objective, the gradient and the line search only through |u|^2,
// u and sums that Parseval's identity turns into real-space sums.
struct PatternArgs {
    int H, W, K;
    const float2 *probe;        // [P][P], scaled by 1/P (the unitary normalisation); with
                                // probe_stride = P * P one probe per sorted pattern [K][P][P]
    long long probe_stride = 0; // elements between the probes of consecutive patterns
    const float2 *tw;           // [P] exp(-2 pi i m / P)
    const int2 *pos;            // [K] (row, col), position-sorted order
    const int *perm;            // [K] caller index of sorted pattern i
    const long long *nz_off;    // [K * nzc + 1] first entry of (sorted pattern i, column chunk c)
    int nzc;                    // column chunks per pattern in the entry layout (P / R_min)
    const unsigned short *nz_slot;  // [E] global slot qy * P + qx of each entry
    const float *nz_d;          // [E] measured counts (> 0) of each entry
    float2 *nz_u;               // [E] u = G psi_m at each entry (GRAD pass -> LS pass)
    float2 *nz_v;               // [E] v = G eta_m at each entry (LS pass -> candidate windows)
    const int *pat_view;        // [K] view of sorted pattern i (all 0 for one view)
    int V;                      // views
    float eps;
    int est;  // 0: Poisson likelihood (Eq. 2); 1: least squares on amplitudes
    // [K * CS] sum of the counts of each (pattern, CTA) chunk of the LS configuration; set
    // when the LS pass also writes the certificate rows (else nullptr)
    const float *dsum;
    // [K][P * P / 32] (P <= 128, else nullptr): bit qx * P + qy of pattern i's mask is set when
    // the spectrum slot (qy, qx) of the tile holds an entry (word qx * P / 32 + qy / 32, bit
    // qy % 32), so that the linear GRAD pass reads only those slots instead of zeroing the tile
    const unsigned *nz_mask = nullptr;
};

// Line-search window description (device scalars come from DevState).
struct LsArgs {
    double gamma0, tau, t;
    int max_halvings;
    int L;         // candidates per pass (the kernel's capacity)
    int adaptive;  // first window of an iteration sized from the previous trial count
    int warm;      // warm-started search: the first trial is the previous accepted step
    int gd;        // gradient descent (Eq. 4): no direction coefficient, no line search
    double gd_step;
};

// Probe of sorted pattern i (the shared probe when probe_stride is 0).
__host__ __device__ __forceinline__ const float2 *probe_of(const PatternArgs &a, int i)
{
    return a.probe + (size_t)i * (size_t)a.probe_stride;
}

// ---- pattern kernels (pattern_kernels.cuh, instantiated per P in pattern_p*.cu) ----
// One configuration: patterns of P x P held by clusters of P / R CTAs of NT threads.
// Per-pattern sums are written per CTA: fpart[K * CS], LS partials [L + 2][K * CS].  All
// partial sums are float-float pairs (float2: hi, lo; reduce.cuh).
struct PatternImpl {
    int P, R, NT;
    // out[perm[i]] = F(p * patch_i(psi))   (unitary)
    cudaError_t (*forward)(const PatternArgs &, const float2 *psi, float2 *out, cudaStream_t);
    // w[i] = conj(p) * F^H y[perm[i]]
    cudaError_t (*adjoint)(const PatternArgs &, const float2 *y, float2 *w, cudaStream_t);
    // GRAD pattern pass: w[i] = conj(p) F^H r_i, r the likelihood residual of u = G psi;
    // fpart = objective terms; u kept at the entries.  Exits early when st->stalled.
    cudaError_t (*grad)(const PatternArgs &, const float2 *psi, float2 *w, float2 *fpart, const DevState *st,
                        cudaStream_t);
    // GRAD pattern pass in the linear form (views with st->lin set; k_grad skips them):
    // u = u + gamma_last v at the entries, fpart = entry terms of the objective,
    // w[i] = conj(p) F^H Delta_i with Delta the residual's difference from u.
    cudaError_t (*grad_lin)(const PatternArgs &, float2 *w, float2 *fpart, const DevState *st, cudaStream_t);
    // LS pattern pass, once per iteration: v = G eta (eta the object-sized search direction)
    // is kept at the entries (nz_v) and part[0][.], part[1][.] = -(sum Re conj(u) v, sum
    // |v|^2) over the entries (per CTA, rows of length K * CS): the all-pixel totals come from
    // object sums (launch_eta).  Exits when st->stalled.
    cudaError_t (*ls)(const PatternArgs &, const float2 *eta, float2 *part, const DevState *st, cudaStream_t);
    // Columns the LS pass writes per row: with one view a persistent single-CTA configuration
    // sums its patterns per CTA and writes gridDim columns (returned); otherwise 0: one
    // column per (pattern, CTA) chunk.
    int (*ls_cols)(const PatternArgs &);
    // Columns of fpart the GRAD passes write: with one view a single-CTA configuration sums
    // per CTA (both GRAD kernels on the same grid, returned); otherwise 0 (one per chunk).
    int (*grad_cols)(const PatternArgs &);
    // Entries of the measured data: counts per (pattern, CTA) chunk, then the compact list.
    cudaError_t (*nz_count)(const float *d, const int *perm, int K, int *cnt, cudaStream_t);
    cudaError_t (*nz_fill)(const float *d, const int *perm, int K, const long long *off, unsigned short *slot,
                           float *dval, cudaStream_t);
};
// Configurations available for P (table of n entries; n = 0 if P is not supported).
int pattern_impls(int P, const PatternImpl **out);
bool pattern_supported(int P);
int ls_window_supported(int L);  // 1 if L is an instantiated window size
// out[i] = log1p_fast(t[i]) (device self-test of the line-search logarithm)
cudaError_t launch_selftest_log1p(const float *t, float *out, int n, cudaStream_t s);

// ---- line-search candidate windows (ls_entries.cu) ----
// part[2 + l][i * cs + c] = sum over the entries of chunk c of pattern i of the objective
// change at candidate l (gamma0 tau^(k0+l+1)), from u (nz_u), v (nz_v) and d: the window
// of the L-candidate kernel; returns at once unless st->Lsel == L and a window is open.
// Columns launch_ls_entries writes per row with one view (one per CTA), else 0 (one per unit).
int ls_entries_cols(const PatternArgs &a, int cs, int V);
cudaError_t launch_ls_entries(const PatternArgs &a, int cs, int V, int L, float2 *part, const DevState *st,
                              cudaStream_t s);
// PatternArgs::nz_mask of the K patterns from the entries (mask zeroed by the caller).
cudaError_t launch_nz_mask(const PatternArgs &a, int P, unsigned *mask, cudaStream_t s);

// ---- tensor-core DFT (tc_dft.cu) ----
// One application: Y[b][k][y] = sum_n X[b][y][n] exp(sign 2 pi i n k / P) for the nrows =
// B * P rows of X (output block b goes to out_index[b] when out_index is non-NULL); two
// applications give the unnormalised 2-D DFT.  img: the split DFT matrix images built by
// tc_dft_images (device copy).  err |= 1 on a timed-out device wait.
bool tc_dft_supported(int P, bool bf16);
// Polls every pipeline wait of the tensor-core kernels allows before it gives up (the kernel
// then records err |= 1); tc_set_wait_limit(polls <= 0) restores the default.
long long tc_wait_limit();
void tc_set_wait_limit(long long polls);
cudaError_t tc_dft_images(int P, bool bf16, int sign, std::vector<uint8_t> &out);
// conj_mul (nullable): the stored element (k, y) of block b is multiplied by conj(conj_mul[k*P + y]).
cudaError_t tc_dft_rows(int P, bool bf16, const float2 *X, float2 *Y, const void *img, int nrows,
                        const int *out_index, const float2 *conj_mul, int *err, cudaStream_t s);
cudaError_t launch_gather_patches(const PatternArgs &a, int P, const float2 *psi, float2 *X, cudaStream_t s);
// The BF16 split form as a persistent warp-specialised kernel (tc_ws.cu): its B images
// (interleaved real/imaginary K) and the row DFT with the semantics of tc_dft_rows.
cudaError_t tc_ws_images(int P, int sign, std::vector<uint8_t> &out);
cudaError_t tc_ws_rows(int P, const float2 *X, float2 *Y, const void *img, int nrows, const int *out_index,
                       const float2 *conj_mul, int *err, cudaStream_t s);
// CG pieces of the tensor-core form (tc_cg.cu); spectra U, V are [K][P][P] in natural order.
// Residual of Eq. 3 in place in U at the entries, objective terms fpart[i], u kept in nz_u.
cudaError_t launch_tc_residual(const PatternArgs &a, int P, float2 *U, float2 *fpart, const DevState *st,
                               cudaStream_t s);
// X[i] = (probe / P) * eta patch with eta = -g + alpha_v eta_prev; pars[0][i], pars[1][i] =
// P^2 sum conj(p psi / P) (p eta / P) and P^2 sum |p eta / P|^2 (real parts, Parseval sums).
cudaError_t launch_tc_gather_eta(const PatternArgs &a, int P, const float2 *psi, const float2 *g, const float2 *ep,
                                 float2 *X, float2 *pars, const DevState *st, cudaStream_t s);
// Candidate sums of one line-search window from V at the entries (layout [L+2][K]).
cudaError_t launch_tc_ls_entries(const PatternArgs &a, int P, int L, const float2 *V, const float2 *pars,
                                 float2 *part, const DevState *st, cudaStream_t s);

// ---- object kernels (object_kernels.cu) ----
// Object tile of the scatter-add and of the other object-tile kernels (rows x columns);
// views of a batch start on multiples of 32 rows, a multiple of kTileY.
#ifndef PTY_TILE_Y
#define PTY_TILE_Y 16
#endif
#ifndef PTY_TILE_X
#define PTY_TILE_X 64
#endif
constexpr int kTileY = PTY_TILE_Y, kTileX = PTY_TILE_X;
static_assert(32 % kTileY == 0 && 256 % kTileX == 0 && (kTileY * kTileX) % 256 == 0, "object tile shape");
struct ScatterPlan {
    int TY, TX;       // object tile
    int ntile_y, ntile_x;
    const int *tile_start;  // [ntiles + 1] CSR offsets
    const int *tile_list;   // sorted pattern indices overlapping each tile, ascending
    const int *tile_view;   // [ntiles] view of each tile (views start on tile rows)
};

// Per-view ranges of the batched layout (device arrays).
struct ViewMap {
    int V;
    const int *pat_off;   // [V + 1] sorted pattern range of each view
    const int *tile_off;  // [V + 1] scatter-tile range of each view
    const int *row_view;  // [H] view of each object row
};
// out[y][x] = sum over patterns i covering (y, x), in ascending i, of w[i][y-r_i][x-c_i],
// plus P^2 D psi for views in the linear form (st->lin; psi, D the object and illumination).
// With dy != 0 also part[b] = (sum |out|^2, sum Re conj(eta_prev) (out - g_prev),
// linear form ? sum D |psi|^2 : 0) per tile b ([ntiles][3]).
// Scatter-add with the per-pattern results fetched by tensor copies (scatter_tma.cu): map is
// a tensor map of w [K][P][P] (scatter_tma_map_bytes() bytes, 64-byte aligned, made by
// make_scatter_tma_map, false if the driver cannot); same sums in the same order as
// launch_scatter.  A bounded wait that gives up sets *err.
size_t scatter_tma_map_bytes();
bool make_scatter_tma_map(void *map, const float2 *w, int P, int K);
cudaError_t launch_scatter_tma(int P, const void *map, const PatternArgs &a, const ScatterPlan &plan, float2 *out,
                               int dy, const float2 *eta_prev, const float2 *g_prev, float2 *part,
                               const DevState *st, cudaStream_t s, const float2 *psi, const float *D, int *err,
                               long long spin_limit);
cudaError_t launch_scatter(int P, const PatternArgs &a, const ScatterPlan &plan, const float2 *w,
                           float2 *out, int dy, const float2 *eta_prev, const float2 *g_prev,
                           float2 *part, const DevState *st, cudaStream_t s, const float2 *psi = nullptr,
                           const float *D = nullptr);
// Fixed-order sum of n float-float values into *out (one block).
cudaError_t launch_sum(const float2 *v, int n, double *out, cudaStream_t s);
// DIR stage scalars per view (one block each): F_m = sum of the view's fpart (CS per
// pattern) plus p2 times the tiles' third partial (linear form); alpha from the view's tile
// partials (restart rule); opens the first line-search window; writes the history of
// iteration m.
// fcols > 0: fpart holds fcols per-CTA columns (one view), else one per pattern chunk.
cudaError_t launch_dy_finalize(const float2 *fpart, int cs, int fcols, const float2 *part, double p2, const ViewMap &vm,
                               DevState *st, DevHist h, const LsArgs &ls, cudaStream_t s);
// LS stage decision per view over the open window; part rows have length kc (K * CS), the
// view's partials are [pat_off[v] * cs, pat_off[v + 1] * cs).  vpart (nullable): object-tile
// partials [ntiles][2] added, times vscale, to rows 0 and 1 over the view's tiles.
// Certified skip of leading trials (Jensen bound rows of the LS pass), then the first window.
// ls_cols: columns of the LS pass's rows when it sums per CTA (one view), else 0.
cudaError_t launch_ls_certify(const float2 *part, int kc, int cs, int ls_cols, const ViewMap &vm, const float2 *vpart,
                              double vscale, const LsArgs &ls, DevState *st, cudaStream_t s);
// dsum[i * cs + c] = sum of the counts of chunk c of sorted pattern i (cs chunks per pattern).
cudaError_t launch_chunk_dsum(const PatternArgs &a, int cs, float *dsum, cudaStream_t s);
// ls_cols / en_cols: columns of rows 0-1 (LS pass) / rows 2.. (windows) when summed per CTA
// (one view), else 0 (one column per pattern chunk, the view's range).
cudaError_t launch_ls_decide(const float2 *part, int kc, int cs, int ls_cols, int en_cols, const ViewMap &vm,
                             const float2 *vpart, double vscale, const LsArgs &ls, DevState *st, DevHist h,
                             cudaStream_t s);
// D[y][x] = sum over the positions covering (y, x) of |probe / P|^2 at the covered pixel.
cudaError_t launch_illumination(int P, const PatternArgs &a, const ScatterPlan &plan, float *D, cudaStream_t s);
// subpixel.cu: out[k] = probe moved by frac[k] = (dy, dx) pixels (Fourier shift theorem,
// Nyquist factor cos(pi d)) for k < K; probe [P][P], out [K][P][P] (create time only).
cudaError_t launch_shift_probes(int P, int K, const float2 *probe, const float2 *frac, float2 *out, cudaStream_t s);
// eta = -g + alpha_v eta_prev over the object (H x W, scatter tiles) and the per-tile sums
// part[b] = (sum D Re conj(psi) eta, sum D |eta|^2).
cudaError_t launch_eta(int H, int W, const ScatterPlan &plan, const float2 *psi, const float2 *g, const float2 *ep,
                       const float *D, float2 *eta, float2 *part, const DevState *st, cudaStream_t s);
// Update stage for every object pixel (W columns per row): psi += gamma eta,
// eta_prev <- eta = -g + alpha eta_prev, g_prev <- g, with the scalars of the row's view.
// lin_period > 0 enables the linear form of the next GRAD pass (a full pass every
// lin_period iterations).
cudaError_t launch_update(int H, int W, const ViewMap &vm, float2 *psi, const float2 *g, float2 *eta_prev,
                          float2 *g_prev, DevState *st, int lin_period, cudaStream_t s);
// Gradient descent (Eq. 4): the step of every view is ls.gd_step, taken without a search
// (history: gamma = gd_step, trials 0, F(psi_{m+1}) written by the next GRAD stage).
cudaError_t launch_gd_step(const ViewMap &vm, const LsArgs &ls, DevState *st, DevHist h, cudaStream_t s);
// F(psi) of each view from the GRAD pass's objective partials into the history slot of the
// current iteration count (the final objective of a gradient-descent call).
cudaError_t launch_objective_to_hist(const float2 *fpart, int cs, int fcols, const ViewMap &vm, const DevState *st,
                                     DevHist h, cudaStream_t s);
// flag |= 1 if any of the n floats is NaN, Inf or negative.
cudaError_t launch_check_data(const float *d, size_t n, int *flag, cudaStream_t s);
cudaError_t launch_begin_solve(DevState *st, int V, cudaStream_t s);
// h[v] = order-independent 64-bit hash of view v's rows of psi (H x W atlas).
cudaError_t launch_hash(int H, int W, const int *row_view, const float2 *psi, unsigned long long *h, int V,
                        cudaStream_t s);
// st[v].lin = 0 where force or h[v] differs from st[v].psi_hash; store h into psi_hash.
cudaError_t launch_check_hash(DevState *st, int V, const unsigned long long *h, int force, cudaStream_t s);
cudaError_t launch_store_hash(DevState *st, int V, const unsigned long long *h, cudaStream_t s);

}  // namespace pty

struct pty_ctx;
namespace pty {
// Sizes of a context: view 0's object H x W, P, K, the number of views and the device.
int ctx_info(const pty_ctx *c, int *H, int *W, int *P, int *K, int *V, int *dev);

}  // namespace pty

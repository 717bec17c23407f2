/*
 * ORACLE for maximum-likelihood conjugate-gradient (ML-CG) ptychography.
 * TEST INFRASTRUCTURE ONLY: this file is compiled into liborc.so, which only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load.  The product
 * (the CUDA library under paper_2106_07575_gb300/csrc) never includes, links or calls
 * it, and the two share no code, header, table or constant generator.
 *
 * Plain, slow, FP64 code written from the paper (Yu et al., "Scalable and accurate
 * multi-GPU based image reconstruction of large-scale ptychography data", PtyGer,
 * arXiv 2106.07575), section "Inverse problem for ptychography":
 *   Eq. 1  forward model        |G psi|^2 = |F Q psi|^2 = d
 *   Eq. 2  ML objective         F(psi) = sum_j |G psi|_j^2 - 2 d_j log|G psi|_j
 *   Eq. 3  gradient             grad F = G^H (G psi - d / (G psi)^*)
 *   Eq. 5  CG update            psi_{m+1} = psi_m + gamma_m eta_m
 *   Eq. 6  Dai-Yuan direction   eta_m = -g_m + ||g_m||^2 / <eta_{m-1}, g_m - g_{m-1}> eta_{m-1}
 *   Eq. 7  line search          shrink gamma until F(psi + gamma eta) <= F(psi) + gamma t
 *   Algorithm 1                 GRAD -> DIR -> LS -> Update, gamma^(0)=1, tau=0.5
 * The multi-GPU parts of Algorithm 1 (gather/scatter, all-reduce, border exchange)
 * are not part of this single-device method and are absent here.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *  - psi is the object transmission (H x W); the exit wave of position k is p * patch_k.
 *  - F is the unitary 2-D DFT (1/P per 2-D transform), forward kernel exp(-2 pi i k n / P),
 *    no fftshift, so F^H = F^{-1} exactly as the gradient's definition requires.
 *  - Eq. 2 is 2 log|u| = log|u|^2; the implemented objective is
 *    F_eps = sum |u|^2 - d log(|u|^2 + eps) with 0*log(.) := 0 when d = 0, whose exact
 *    Wirtinger gradient is u - d u / (|u|^2 + eps) (Eq. 3 with d/u^* = d u/|u|^2).
 *    The guard eps (in counts, default 0.1) is an input of every function here.
 *  - Eq. 3 is used literally (derivative w.r.t. psi^*, no factor 2).
 *  - <a,b> in Eq. 6 is taken as Re sum conj(a) b; a denominator that is <= 0 or not
 *    finite restarts the direction with eta = -g.
 *  - Line search follows the paper's text: gamma starts at gamma0, is multiplied by tau
 *    BEFORE each trial (do-while), and shrinking stops at the first trial with
 *    F(psi + gamma eta) <= F(psi) + gamma t.  After max_halvings failed trials the solve
 *    stops with psi unchanged for that iteration ("stalled").
 *  - Scan positions are integer top-left corners (row, col) of the P x P patch.  Every
 *    entry point takes either one probe [P][P] shared by all positions (per_pos = 0) or
 *    one probe per position [K][P][P] (per_pos = 1); a fractional position s is taken as
 *    the window floor(s) with the probe shifted by s - floor(s) (orc_shift_probe).
 *  - The least-squares (Gaussian) estimator, which the paper names beside the ML estimate
 *    but does not write out, is taken on amplitudes: F_LS = sum (|u| - sqrt d)^2, guarded
 *    as F_LS,eps = sum |u|^2 - 2 sqrt(d) sqrt(|u|^2 + eps) + d, whose exact Wirtinger
 *    gradient is u - sqrt(d) u / sqrt(|u|^2 + eps) (equal to F_LS at eps = 0).
 *  - The gradient-descent solver is Eq. 4 with a constant step gamma (no line search).
 *  - Warm-started line search (an option; the paper leaves the initial step of Eq. 7's
 *    search free): from the second iteration of a solve on, the search starts at
 *    gamma_init = min(gamma0, gamma_{m-1} / tau), so that its first trial is the previous
 *    accepted step; every trial is still gamma0 tau^k for an integer k.
 *
 * Complex arrays are interleaved (re, im) doubles, layout-compatible with C99
 * double complex.  Object arrays are [H][W] row-major, per-position arrays [K][P][P].
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_BOUNDS 2
#define ORC_ERR_NOMEM 3
#define ORC_STALLED 4

static const double ORC_PI = 3.14159265358979323846264338327950288;

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* ------------------------------------------------------------------------- */
/* 1-D DFT by iterative radix-2 Cooley-Tukey (decimation in time).           */
/* x[i*stride], i < n, n a power of two; sign = -1 forward, +1 inverse; no   */
/* normalisation.  Twiddles exp(sign 2 pi i j / n) are taken from libm.      */
/* ------------------------------------------------------------------------- */
static void fft1(cplx *x, int n, long stride, int sign, const cplx *tw)
{
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = x[i * stride];
            x[i * stride] = x[j * stride];
            x[j * stride] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1, step = n / len;
        for (int i = 0; i < n; i += len) {
            for (int j = 0; j < half; j++) {
                cplx w = tw[j * step];
                if (sign > 0) w = conj(w);
                cplx a = x[(i + j) * stride];
                cplx b = x[(i + j + half) * stride] * w;
                x[(i + j) * stride] = a + b;
                x[(i + j + half) * stride] = a - b;
            }
        }
    }
}

/* exp(-2 pi i j / n), j < n/2 */
static cplx *make_twiddles(int n)
{
    cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)(n > 1 ? n / 2 : 1));
    if (!tw) return NULL;
    for (int j = 0; j < n / 2; j++) {
        double a = -2.0 * ORC_PI * (double)j / (double)n;
        tw[j] = cos(a) + I * sin(a);
    }
    return tw;
}

/* Unitary 2-D DFT of one P x P array in place (Eq. 1's F; inverse = F^H). */
static void fft2_unitary(cplx *x, int P, int inverse, const cplx *tw)
{
    int sign = inverse ? +1 : -1;
    for (int r = 0; r < P; r++) fft1(x + (long)r * P, P, 1, sign, tw);
    for (int c = 0; c < P; c++) fft1(x + c, P, P, sign, tw);
    double s = 1.0 / (double)P;
    for (long i = 0; i < (long)P * P; i++) x[i] *= s;
}

int orc_fft2(double *x, int P, int inverse)
{
    if (!is_pow2(P) || !x) return ORC_ERR_ARG;
    cplx *tw = make_twiddles(P);
    if (!tw) return ORC_ERR_NOMEM;
    fft2_unitary((cplx *)x, P, inverse, tw);
    free(tw);
    return ORC_OK;
}

/*
 * Sub-pixel shift of the probe by (dy, dx) pixels, for scan positions with a fractional
 * part (the paper's positions are float32; it does not say how a fraction enters Q).
 * Fourier shift theorem with the unitary F of Eq. 1:
 *   out = F^H[ F[p](ky, kx) * phi_dy(ky) * phi_dx(kx) ],
 *   phi_delta(kappa) = exp(-2 pi i kappa delta / P) for the signed frequency
 *   kappa = j (j < P/2) or j - P (j > P/2), and cos(pi delta) at the Nyquist index j = P/2
 *   (the real part of exp(+-i pi delta), so that a real probe stays real).
 * So out(r) = p(r - delta) for a probe band-limited below Nyquist, and an integer shift is
 * the circular shift of the P x P window.
 */
int orc_shift_probe(int P, const double *probe, double dy, double dx, double *out)
{
    if (!is_pow2(P) || P < 2 || !probe || !out || !isfinite(dy) || !isfinite(dx)) return ORC_ERR_ARG;
    cplx *tw = make_twiddles(P);
    cplx *fy = (cplx *)malloc(sizeof(cplx) * (size_t)P), *fx = (cplx *)malloc(sizeof(cplx) * (size_t)P);
    if (!tw || !fy || !fx) {
        free(tw);
        free(fy);
        free(fx);
        return ORC_ERR_NOMEM;
    }
    for (int j = 0; j < P; j++) {
        int kappa = j < P / 2 ? j : j - P;
        if (j == P / 2) {
            fy[j] = cos(ORC_PI * dy);
            fx[j] = cos(ORC_PI * dx);
        } else {
            fy[j] = cexp(-2.0 * ORC_PI * I * (double)kappa * dy / (double)P);
            fx[j] = cexp(-2.0 * ORC_PI * I * (double)kappa * dx / (double)P);
        }
    }
    cplx *x = (cplx *)out;
    memcpy(x, probe, sizeof(cplx) * (size_t)P * P);
    fft2_unitary(x, P, 0, tw);
    for (int y = 0; y < P; y++)
        for (int c = 0; c < P; c++) x[(long)y * P + c] *= fy[y] * fx[c];
    fft2_unitary(x, P, 1, tw);
    free(tw);
    free(fy);
    free(fx);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Argument checks shared by the operator entry points.                      */
/* ------------------------------------------------------------------------- */
static int check_geom(int H, int W, int P, int K, const int *pos)
{
    if (H < 1 || W < 1 || !is_pow2(P) || K < 1 || !pos) return ORC_ERR_ARG;
    if (P > H || P > W) return ORC_ERR_ARG;
    for (int k = 0; k < K; k++) {
        int r = pos[2 * k], c = pos[2 * k + 1];
        if (r < 0 || c < 0 || r + P > H || c + P > W) return ORC_ERR_BOUNDS;
    }
    return ORC_OK;
}

static int nthreads_eff(int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    return nthreads;
#else
    (void)nthreads;
    return 1;
#endif
}

/* Q (Eq. 1): e_k[y][x] = p_k[y][x] * psi[r_k + y][c_k + x], where p_k = p + k * ps is the
 * probe of position k: ps = 0 for one probe shared by all positions, ps = P*P for one
 * probe per position (sub-pixel positions, orc_shift_probe). */
static void apply_Q(int W, int P, const cplx *p, long ps, const int *pos, int k, const cplx *psi, cplx *e)
{
    int r = pos[2 * k], c = pos[2 * k + 1];
    p += (long)k * ps;
    for (int y = 0; y < P; y++)
        for (int x = 0; x < P; x++)
            e[(long)y * P + x] = p[(long)y * P + x] * psi[(long)(r + y) * W + (c + x)];
}

/* Q^H for one position (Eq. 3): acc[r_k + y][c_k + x] += conj(p_k[y][x]) * w[y][x]. */
static void apply_QH_add(int W, int P, const cplx *p, long ps, const int *pos, int k, const cplx *w, cplx *acc)
{
    int r = pos[2 * k], c = pos[2 * k + 1];
    p += (long)k * ps;
    for (int y = 0; y < P; y++)
        for (int x = 0; x < P; x++)
            acc[(long)(r + y) * W + (c + x)] += conj(p[(long)y * P + x]) * w[(long)y * P + x];
}

/* Q alone: out[K][P][P] = Q psi. */
int orc_Q(int H, int W, int P, const double *probe, int per_pos, int K, const int *pos, const double *psi,
          double *out)
{
    int st = check_geom(H, W, P, K, pos);
    if (st) return st;
    for (int k = 0; k < K; k++)
        apply_Q(W, P, (const cplx *)probe, (per_pos ? (long)P * P : 0), pos, k, (const cplx *)psi, (cplx *)out + (long)k * P * P);
    return ORC_OK;
}

/* Q^H alone: x[H][W] = sum_k shift_k(conj(p_k) * y_k). */
int orc_QH(int H, int W, int P, const double *probe, int per_pos, int K, const int *pos, const double *y,
           double *x)
{
    int st = check_geom(H, W, P, K, pos);
    if (st) return st;
    memset(x, 0, sizeof(cplx) * (size_t)H * W);
    for (int k = 0; k < K; k++)
        apply_QH_add(W, P, (const cplx *)probe, (per_pos ? (long)P * P : 0), pos, k, (const cplx *)y + (long)k * P * P, (cplx *)x);
    return ORC_OK;
}

/* G = F Q (Eq. 1): out[K][P][P] = unitary DFT2(p_k * patch_k). */
int orc_forward(int H, int W, int P, const double *probe, int per_pos, int K, const int *pos, const double *psi,
                double *out, int nthreads)
{
    int st = check_geom(H, W, P, K, pos);
    if (st) return st;
    cplx *tw = make_twiddles(P);
    if (!tw) return ORC_ERR_NOMEM;
    int T = nthreads_eff(nthreads);
#pragma omp parallel for num_threads(T) schedule(static)
    for (int k = 0; k < K; k++) {
        cplx *u = (cplx *)out + (long)k * P * P;
        apply_Q(W, P, (const cplx *)probe, (per_pos ? (long)P * P : 0), pos, k, (const cplx *)psi, u);
        fft2_unitary(u, P, 0, tw);
    }
    free(tw);
    return ORC_OK;
}

/*
 * Per-thread scatter-add helper: patterns are split into T contiguous chunks in index
 * order; chunk t accumulates into its own object buffer; the buffers are then summed in
 * chunk order, so the result depends only on (K, T), never on thread timing.
 */
typedef void (*pattern_fn)(int k, cplx *work, cplx *acc, double *fpart, void *ctx);

static int run_patterns_scatter(int K, int P, int H, int W, int T, pattern_fn fn, void *ctx,
                                cplx *acc_out, double *fpart)
{
    if (T < 1) T = 1;
    if (T > K) T = K;
    cplx *bufs = (cplx *)calloc((size_t)T * H * W, sizeof(cplx));
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)T * P * P);
    if (!bufs || !work) {
        free(bufs);
        free(work);
        return ORC_ERR_NOMEM;
    }
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int t = 0; t < T; t++) {
        long k0 = (long)K * t / T, k1 = (long)K * (t + 1) / T;
        for (long k = k0; k < k1; k++)
            fn((int)k, work + (long)t * P * P, bufs + (long)t * H * W, fpart ? fpart + k : NULL, ctx);
    }
    memset(acc_out, 0, sizeof(cplx) * (size_t)H * W);
    for (int t = 0; t < T; t++) {
        const cplx *b = bufs + (long)t * H * W;
        for (long i = 0; i < (long)H * W; i++) acc_out[i] += b[i];
    }
    free(bufs);
    free(work);
    return ORC_OK;
}

/* G^H = Q^H F^H (Eq. 3): x[H][W] = sum_k shift_k(conj(p) * IDFT2(y_k)). */
struct adj_ctx {
    int W, P;
    const cplx *p, *y;
    long ps;
    const int *pos;
    const cplx *tw;
};

static void adj_one(int k, cplx *work, cplx *acc, double *fpart, void *vctx)
{
    (void)fpart;
    struct adj_ctx *c = (struct adj_ctx *)vctx;
    long PP = (long)c->P * c->P;
    memcpy(work, c->y + (long)k * PP, sizeof(cplx) * PP);
    fft2_unitary(work, c->P, 1, c->tw);
    apply_QH_add(c->W, c->P, c->p, c->ps, c->pos, k, work, acc);
}

int orc_adjoint(int H, int W, int P, const double *probe, int per_pos, int K, const int *pos, const double *y,
                double *x, int nthreads)
{
    int st = check_geom(H, W, P, K, pos);
    if (st) return st;
    cplx *tw = make_twiddles(P);
    if (!tw) return ORC_ERR_NOMEM;
    struct adj_ctx c = {W, P, (const cplx *)probe, (const cplx *)y, (per_pos ? (long)P * P : 0), pos, tw};
    st = run_patterns_scatter(K, P, H, W, nthreads_eff(nthreads), adj_one, &c, (cplx *)x, NULL);
    free(tw);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Objective (Eq. 2) and gradient (Eq. 3).                                   */
/* ------------------------------------------------------------------------- */
struct obj_ctx {
    int W, P;
    const cplx *p, *psi;
    long ps;
    const int *pos;
    const float *d;
    double eps;
    int est;
    const cplx *tw;
};

#define ORC_EST_ML 0 /* Poisson maximum likelihood, Eq. 2 */
#define ORC_EST_LS 1 /* Gaussian least squares on amplitudes */

/* f for one detector pixel.
 *   ML (Eq. 2): |u|^2 - d log(|u|^2 + eps), with 0 log(.) := 0;
 *   LS:         |u|^2 - 2 sqrt(d) sqrt(|u|^2 + eps) + d, i.e. (|u| - sqrt d)^2 at eps = 0. */
static double pixel_objective(cplx u, double d, double eps, int est)
{
    double a = creal(u) * creal(u) + cimag(u) * cimag(u);
    if (!(d > 0.0)) return a;
    if (est == ORC_EST_LS) return a - 2.0 * sqrt(d) * sqrt(a + eps) + d;
    return a - d * log(a + eps);
}

/* Fourier-domain residual, the Wirtinger derivative of pixel_objective w.r.t. conj(u):
 *   ML (Eq. 3): u - d u / (|u|^2 + eps);   LS: u - sqrt(d) u / sqrt(|u|^2 + eps). */
static cplx pixel_residual(cplx u, double d, double eps, int est)
{
    double a = creal(u) * creal(u) + cimag(u) * cimag(u);
    if (!(d > 0.0)) return u;
    if (est == ORC_EST_LS) return u - (sqrt(d) / sqrt(a + eps)) * u;
    return u - (d / (a + eps)) * u;
}

static void obj_one(int k, cplx *work, cplx *acc, double *fpart, void *vctx)
{
    (void)acc;
    struct obj_ctx *c = (struct obj_ctx *)vctx;
    long PP = (long)c->P * c->P;
    apply_Q(c->W, c->P, c->p, c->ps, c->pos, k, c->psi, work);
    fft2_unitary(work, c->P, 0, c->tw);
    const float *dk = c->d + (long)k * PP;
    double s = 0.0;
    for (long j = 0; j < PP; j++) s += pixel_objective(work[j], (double)dk[j], c->eps, c->est);
    *fpart = s;
}

static void grad_one(int k, cplx *work, cplx *acc, double *fpart, void *vctx)
{
    struct obj_ctx *c = (struct obj_ctx *)vctx;
    long PP = (long)c->P * c->P;
    apply_Q(c->W, c->P, c->p, c->ps, c->pos, k, c->psi, work);
    fft2_unitary(work, c->P, 0, c->tw);
    const float *dk = c->d + (long)k * PP;
    double s = 0.0;
    for (long j = 0; j < PP; j++) {
        s += pixel_objective(work[j], (double)dk[j], c->eps, c->est);
        work[j] = pixel_residual(work[j], (double)dk[j], c->eps, c->est);
    }
    *fpart = s;
    fft2_unitary(work, c->P, 1, c->tw);
    apply_QH_add(c->W, c->P, c->p, c->ps, c->pos, k, work, acc);
}

/* Objective with per-pattern partials summed in pattern order. */
static int objective_impl(int H, int W, int P, const cplx *p, long ps, int K, const int *pos, const float *d,
                          double eps, int est, const cplx *psi, const cplx *tw, int T, double *F)
{
    double *fpart = (double *)malloc(sizeof(double) * (size_t)K);
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)(T < 1 ? 1 : T) * P * P);
    if (!fpart || !work) {
        free(fpart);
        free(work);
        return ORC_ERR_NOMEM;
    }
    struct obj_ctx c = {W, P, p, psi, ps, pos, d, eps, est, tw};
    (void)H;
#pragma omp parallel for num_threads(T) schedule(static)
    for (int k = 0; k < K; k++) {
#ifdef _OPENMP
        int t = omp_get_thread_num();
#else
        int t = 0;
#endif
        obj_one(k, work + (long)t * P * P, NULL, fpart + k, &c);
    }
    double s = 0.0;
    for (int k = 0; k < K; k++) s += fpart[k];
    *F = s;
    free(fpart);
    free(work);
    return ORC_OK;
}

static int gradient_impl(int H, int W, int P, const cplx *p, long ps, int K, const int *pos, const float *d,
                         double eps, int est, const cplx *psi, const cplx *tw, int T, cplx *g, double *F)
{
    double *fpart = (double *)malloc(sizeof(double) * (size_t)K);
    if (!fpart) return ORC_ERR_NOMEM;
    struct obj_ctx c = {W, P, p, psi, ps, pos, d, eps, est, tw};
    int st = run_patterns_scatter(K, P, H, W, T, grad_one, &c, g, fpart);
    if (st == ORC_OK && F) {
        double s = 0.0;
        for (int k = 0; k < K; k++) s += fpart[k];
        *F = s;
    }
    free(fpart);
    return st;
}

int orc_objective(int H, int W, int P, const double *probe, int per_pos, int K, const int *pos, const float *d,
                  double eps, int est, const double *psi, double *F, int nthreads)
{
    if (est != ORC_EST_ML && est != ORC_EST_LS) return ORC_ERR_ARG;
    int st = check_geom(H, W, P, K, pos);
    if (st) return st;
    if (!F || !d || !psi || !probe) return ORC_ERR_ARG;
    cplx *tw = make_twiddles(P);
    if (!tw) return ORC_ERR_NOMEM;
    st = objective_impl(H, W, P, (const cplx *)probe, (per_pos ? (long)P * P : 0), K, pos, d, eps, est,
                        (const cplx *)psi, tw,
                        nthreads_eff(nthreads), F);
    free(tw);
    return st;
}

int orc_gradient(int H, int W, int P, const double *probe, int per_pos, int K, const int *pos, const float *d,
                 double eps, int est, const double *psi, double *g, double *F, int nthreads)
{
    if (est != ORC_EST_ML && est != ORC_EST_LS) return ORC_ERR_ARG;
    int st = check_geom(H, W, P, K, pos);
    if (st) return st;
    if (!g || !d || !psi || !probe) return ORC_ERR_ARG;
    cplx *tw = make_twiddles(P);
    if (!tw) return ORC_ERR_NOMEM;
    st = gradient_impl(H, W, P, (const cplx *)probe, (per_pos ? (long)P * P : 0), K, pos, d, eps, est,
                       (const cplx *)psi, tw,
                       nthreads_eff(nthreads), (cplx *)g, F);
    free(tw);
    return st;
}

/* ------------------------------------------------------------------------- */
/* CG solve (Eq. 5, 6, 7; Algorithm 1 on one device).                        */
/* ------------------------------------------------------------------------- */
#define ORC_SOLVER_CG 0 /* Eq. 5-7, Algorithm 1 */
#define ORC_SOLVER_GD 1 /* Eq. 4, constant step */

typedef struct {
    double gamma0;     /* initial step, Algorithm 1: 1 */
    double tau;        /* shrink factor, Algorithm 1: 0.5 */
    double t;          /* Eq. 7 termination constant, "usually 0" */
    int max_halvings;  /* trials before the solve is declared stalled */
    double eps;        /* log / division guard of the implemented objective */
    int est;           /* ORC_EST_ML (Eq. 2) or ORC_EST_LS */
    int solver;        /* ORC_SOLVER_CG or ORC_SOLVER_GD */
    double gd_step;    /* constant step gamma of Eq. 4 (GD only) */
    int warm;          /* 1: warm-started line search (CG only) */
} orc_opts;

static double wall_seconds(void)
{
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return 0.0;
#endif
}

/* Re sum conj(a) b over n complex values. */
static double re_dot(const cplx *a, const cplx *b, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += creal(a[i]) * creal(b[i]) + cimag(a[i]) * cimag(b[i]);
    return s;
}

/*
 * niter iterations from psi (in place).  Outputs (each nullable):
 *   F_hist[niter+1]: F(psi_m) for m = 0..iters_done (F of the accepted trial at the end),
 *   gamma[niter], halvings[niter] (number of trials), alpha[niter] (Dai-Yuan coefficient,
 *   0 for the steepest-descent start or a restart).
 *   t_hist[niter]: wall-clock seconds from the start of the solve to the end of each
 *                  iteration (measurement only).
 * Returns ORC_OK, or ORC_STALLED when an iteration found no step within max_halvings
 * trials (psi keeps the last accepted iterate; *iters_done counts accepted iterations).
 * With opts->solver == ORC_SOLVER_GD the iterations are Eq. 4 instead: psi -= gd_step g,
 * gamma = gd_step, no trials (halvings 0), alpha 0; F_hist[m+1] = F(psi_{m+1}).
 */
int orc_cg_solve(int H, int W, int P, const double *probe, int per_pos, int K, const int *pos, const float *d,
                 const orc_opts *opts, double *psi_io, int niter, double *F_hist, double *gamma_out,
                 int *halvings_out, double *alpha_out, int *iters_done, double *t_hist, int nthreads)
{
    int st = check_geom(H, W, P, K, pos);
    if (st) return st;
    if (!opts || !psi_io || !d || !probe || niter < 0) return ORC_ERR_ARG;
    if ((opts->est != ORC_EST_ML && opts->est != ORC_EST_LS) ||
        (opts->solver != ORC_SOLVER_CG && opts->solver != ORC_SOLVER_GD))
        return ORC_ERR_ARG;
    const int est = opts->est;
    int T = nthreads_eff(nthreads);
    long n = (long)H * W;
    cplx *psi = (cplx *)psi_io;
    cplx *g = (cplx *)calloc((size_t)n, sizeof(cplx)), *g_prev = (cplx *)calloc((size_t)n, sizeof(cplx));
    cplx *eta = (cplx *)calloc((size_t)n, sizeof(cplx)), *trial = (cplx *)calloc((size_t)n, sizeof(cplx));
    cplx *tw = make_twiddles(P);
    if (!g || !g_prev || !eta || !trial || !tw) {
        st = ORC_ERR_NOMEM;
        goto done;
    }
    const cplx *p = (const cplx *)probe;
    const long ps = (per_pos ? (long)P * P : 0);
    int m;
    if (iters_done) *iters_done = 0;
    double gam_prev = 0.0; /* last accepted step of this solve (warm start) */
    const double t_begin = wall_seconds();
    for (m = 0; m < niter; m++) {
        /* GRAD stage: g_m = grad F(psi_m), F_m = F(psi_m) */
        double Fm;
        st = gradient_impl(H, W, P, p, ps, K, pos, d, opts->eps, est, psi, tw, T, g, &Fm);
        if (st) goto done;
        if (F_hist) F_hist[m] = Fm;
        if (opts->solver == ORC_SOLVER_GD) {
            /* Eq. 4: psi_{m+1} = psi_m - gamma grad F(psi_m), gamma constant */
            for (long i = 0; i < n; i++) psi[i] -= opts->gd_step * g[i];
            if (gamma_out) gamma_out[m] = opts->gd_step;
            if (halvings_out) halvings_out[m] = 0;
            if (alpha_out) alpha_out[m] = 0.0;
            if (F_hist && m + 1 == niter) {
                double Fn;
                st = objective_impl(H, W, P, p, ps, K, pos, d, opts->eps, est, psi, tw, T, &Fn);
                if (st) goto done;
                F_hist[m + 1] = Fn;
            }
            if (iters_done) *iters_done = m + 1;
            if (t_hist) t_hist[m] = wall_seconds() - t_begin;
            continue;
        }
        /* DIR stage: Dai-Yuan (Eq. 6), eta_0 = -g_0 */
        double alpha = 0.0;
        if (m > 0) {
            double num = re_dot(g, g, n);
            double den = 0.0;
            for (long i = 0; i < n; i++) {
                cplx dg = g[i] - g_prev[i];
                den += creal(eta[i]) * creal(dg) + cimag(eta[i]) * cimag(dg);
            }
            if (den > 0.0 && isfinite(den) && isfinite(num)) alpha = num / den;
        }
        if (m == 0 || alpha == 0.0) {
            for (long i = 0; i < n; i++) eta[i] = -g[i]; /* eta_0 = -grad F(psi_0); restart */
        } else {
            for (long i = 0; i < n; i++) eta[i] = -g[i] + alpha * eta[i];
        }
        if (alpha_out) alpha_out[m] = alpha;
        /* LS stage: gamma^(0) = gamma0; do { gamma *= tau; F(psi+gamma eta) } while Eq. 7 fails */
        double gam = opts->gamma0, Ft = 0.0;
        if (opts->warm && gam_prev > 0.0 && gam_prev / opts->tau < gam) gam = gam_prev / opts->tau;
        int k = 0, ok = 0;
        do {
            gam *= opts->tau;
            k++;
            for (long i = 0; i < n; i++) trial[i] = psi[i] + gam * eta[i];
            st = objective_impl(H, W, P, p, ps, K, pos, d, opts->eps, est, trial, tw, T, &Ft);
            if (st) goto done;
            ok = (Ft <= Fm + gam * opts->t);
        } while (!ok && k < opts->max_halvings);
        if (gamma_out) gamma_out[m] = gam;
        if (halvings_out) halvings_out[m] = k;
        if (!ok) {
            st = ORC_STALLED;
            if (F_hist) F_hist[m + 1] = Fm;
            goto done;
        }
        /* Update stage (Eq. 5) */
        for (long i = 0; i < n; i++) psi[i] = trial[i];
        if (F_hist) F_hist[m + 1] = Ft;
        memcpy(g_prev, g, sizeof(cplx) * n);
        gam_prev = gam;
        if (iters_done) *iters_done = m + 1;
        if (t_hist) t_hist[m] = wall_seconds() - t_begin;
    }
    st = ORC_OK;
done:
    free(g);
    free(g_prev);
    free(eta);
    free(trial);
    free(tw);
    return st;
}

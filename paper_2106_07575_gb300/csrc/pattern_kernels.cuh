// pattern_kernels.cuh -- the per-scan-position passes of ML-CG.  One pattern is owned by a
// thread-block cluster of CS = P / R CTAs (CS = 1: a single CTA) that keeps the P x P exit
// wave in shared memory and runs the 2-D DFTs of fft_tile.cuh on it.
//
//   k_forward      Eq. 1: u = F(p * patch(psi)) written out (pty_forward)
//   k_adjoint_fft  the F^H and conj(p) factors of G^H (pty_adjoint)
//   k_grad         GRAD stage: gather x probe -> F -> likelihood residual (Eq. 3) and the
//                  objective terms (Eq. 2) -> F^H -> x conj(p); one patch-sized result
//                  per pattern, summed into the object by the scatter kernel
//   k_grad_lin     GRAD stage in the linear form: u updated at the entries from the kept
//                  v = G eta of the last step, one inverse DFT of the sparse correction
//   k_ls_fft       LS stage, once per iteration: v = G eta for one pattern, kept at the
//                  detector pixels with counts, the two Parseval sums that the change
//                  of the objective needs at the other pixels, and the Jensen lower bounds
//                  of that change at the leading trials (certificate rows; the candidate
//                  windows run on the kept values: ls_entries.cu)
//   k_nz_*         create time: the compact list of detector pixels with counts
//
// The forward DFT leaves the spectrum in the permuted slot order of fft_tile.cuh, in
// column slabs; the measured data are stored in that order ("entries", one contiguous
// range per CTA of a pattern), and the inverse DFT returns to natural order, so no
// separate reordering pass exists.  Per-pattern sums are produced per CTA; the small
// reduction kernels add the CS partials of a pattern like any others.  Persistent
// single-CTA passes of one view sum their partials per thread over the CTA's patterns and
// write one column per CTA, and keep their threads' probe values in tensor memory.
#pragma once
#include "fft_tile.cuh"
#include "mathx.cuh"
#include "pty_internal.h"
#include "reduce.cuh"
#include "tc_ptx.cuh"

#ifndef PTY_GATHER_UNROLL
#define PTY_GATHER_UNROLL 8  // loads of the exit-wave gather in flight per thread
#endif

namespace pty {

constexpr int kGatherUnroll = PTY_GATHER_UNROLL;

// The tile or slab, the twiddles [P], and the row-step twiddles in item order [16 * P/16]
// (single-CTA configurations).
template <int P, int R>
constexpr size_t slab_bytes()
{
    return sizeof(float2) * (size_t)(Slab<P, R>::ELEMS + 2 * P);
}

// Resident CTAs per SM the register allocation may plan for: 1 where the tile or slab takes
// more than half of an SM's shared memory (only one CTA fits, so its threads may use the
// whole register file); 0 (no hint) otherwise.
template <int P, int R>
constexpr int min_ctas()
{
    return slab_bytes<P, R>() > 113 * 1024 ? 1 : 0;
}

// Pattern and cluster rank of this CTA.
template <int P, int R>
__device__ __forceinline__ void who(int &i, int &c)
{
    i = blockIdx.x / Slab<P, R>::CS;
    c = blockIdx.x % Slab<P, R>::CS;
}

// Twiddles [P] and, after them, the row-step twiddles in item order (fft_tile.cuh).
template <int P, int NT>
__device__ __forceinline__ void load_twiddles(float2 *tw, const float2 *__restrict__ g_tw)
{
    for (int m = threadIdx.x; m < P; m += NT) tw[m] = g_tw[m];
    load_row_twiddles<P, NT>(tw + P, g_tw);
}

// Row slab of Q psi: rows [cR, cR+R) of probe[y][x] * src[r0 + y][c0 + x]  (Eq. 1)
template <int P, int R, int NT>
__device__ __forceinline__ void gather_rows(float2 *buf, const float2 *__restrict__ probe,
                                            const float2 *__restrict__ src, int W, int r0, int c0, int c)
{
    constexpr int LDA = Slab<P, R>::LDA;
#pragma unroll kGatherUnroll
    for (int e = threadIdx.x; e < R * P; e += NT) {
        const int rl = e / P, x = e % P, y = c * R + rl;
        buf[rl * LDA + x] = cmul(__ldg(probe + y * P + x), __ldg(src + (size_t)(r0 + y) * W + (c0 + x)));
    }
}

// Probe cache in tensor memory (single-CTA configurations, R = P).  The gather of an exit
// wave and the emit of an adjoint result both run in the row stride step's work items
// (fft_tile.cuh: item ii of thread t is (row, n2), elements n2 + R2 n1), so thread t needs
// only the probe values of its items: NE = P^2 / NT values, 16 per item, in item order.
// They are stored once per kernel in the thread's TMEM lane (lane quarter warp % 4, columns
// from (warp / 4) 2 NE) and read back with tcgen05.ld, instead of 128 KB of L2 loads per
// pattern at P = 128.
template <int P, int NT>
struct ProbeCache {
    static constexpr int NE = P * P / NT;  // complex values per thread
    static constexpr int NCOL = 2 * NE;    // 32-bit TMEM columns per thread
    static constexpr int USED = NCOL * (NT / 128);
    static constexpr int COLS = USED <= 32 ? 32 : USED <= 64 ? 64 : USED <= 128 ? 128 : USED <= 256 ? 256 : 512;
    uint32_t base, addr;

    // All threads; ends with the cache filled and visible to this thread.
    __device__ __forceinline__ void init(uint32_t *slot, const float2 *__restrict__ probe)
    {
        static_assert(NT % 128 == 0 && NE % 4 == 0 && USED <= 512, "probe cache layout");
        const int warp = threadIdx.x >> 5;
        if (warp == 0) tcx::tmem_alloc(slot, COLS);
        tcx::tmem_fence_before_sync();
        __syncthreads();
        tcx::tmem_fence_after_sync();
        base = *slot;
        addr = base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * NCOL);
        constexpr int R2 = Tile<P>::R2;
#pragma unroll 1
        for (int k0 = 0; k0 < NE; k0 += 4) {
            int row, n2;
            row_item<P>(warp + (k0 / 16) * (NT / 32), threadIdx.x & 31, row, n2);
            float v[8];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float2 pv = __ldg(probe + row * P + n2 + R2 * ((k0 % 16) + j));
                v[2 * j] = pv.x;
                v[2 * j + 1] = pv.y;
            }
            tcx::tmem_st8(addr + 2 * k0, v);
        }
        tcx::tmem_wait_st();
    }
    // This thread's probe values k0 .. k0 + 3.
    __device__ __forceinline__ void get4(int k0, float2 (&p)[4]) const
    {
        float v[8];
        tcx::tmem_ld8(addr + 2 * k0, v);
#pragma unroll
        for (int j = 0; j < 4; j++) p[j] = make_float2(v[2 * j], v[2 * j + 1]);
    }
    // All threads, after the last use.
    __device__ __forceinline__ void release() const
    {
        tcx::tmem_fence_before_sync();
        __syncthreads();
        if ((threadIdx.x >> 5) == 0) tcx::tmem_dealloc(base, COLS);
    }
};

// Probe cache in tensor memory for the row slab of a cluster CTA (R < P): the gather of an
// exit wave (gather_rows) and the emit of an adjoint result (emit_adjoint) both visit slab
// element e = t + k NT (row e / P, column e % P) in thread t, so the thread's NE = R P / NT
// probe values are stored once per kernel in its TMEM lane (as ProbeCache does) instead of
// being read from L2 for every pattern (64 KB per CTA and pattern at P = 256, R = 32).
template <int P, int R, int NT>
struct SlabProbeCache {
    static constexpr int NE = R * P / NT;
    static constexpr int NCOL = 2 * NE;
    static constexpr int USED = NCOL * (NT / 128);
    static constexpr int COLS = USED <= 32 ? 32 : USED <= 64 ? 64 : USED <= 128 ? 128 : USED <= 256 ? 256 : 512;
    uint32_t base, addr;

    // All threads; ends with the cache filled and visible to this thread.
    __device__ __forceinline__ void init(uint32_t *slot, const float2 *__restrict__ probe, int c)
    {
        static_assert(NT % 128 == 0 && NE % 4 == 0 && USED <= 512, "slab probe cache layout");
        const int warp = threadIdx.x >> 5;
        if (warp == 0) tcx::tmem_alloc(slot, COLS);
        tcx::tmem_fence_before_sync();
        __syncthreads();
        tcx::tmem_fence_after_sync();
        base = *slot;
        addr = base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * NCOL);
#pragma unroll 1
        for (int k0 = 0; k0 < NE; k0 += 4) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int e = threadIdx.x + (k0 + j) * NT;
                const float2 pv = __ldg(probe + (c * R + e / P) * P + e % P);
                v[2 * j] = pv.x;
                v[2 * j + 1] = pv.y;
            }
            tcx::tmem_st8(addr + 2 * k0, v);
        }
        tcx::tmem_wait_st();
    }
    __device__ __forceinline__ void get4(int k0, float2 (&p)[4]) const
    {
        float v[8];
        tcx::tmem_ld8(addr + 2 * k0, v);
#pragma unroll
        for (int j = 0; j < 4; j++) p[j] = make_float2(v[2 * j], v[2 * j + 1]);
    }
    __device__ __forceinline__ void release() const
    {
        tcx::tmem_fence_before_sync();
        __syncthreads();
        if ((threadIdx.x >> 5) == 0) tcx::tmem_dealloc(base, COLS);
    }
};

// gather_rows with the probe from a SlabProbeCache: the object values of four elements are
// loaded before their probe values are read.
template <int P, int R, int NT>
__device__ __forceinline__ void gather_rows(float2 *buf, const SlabProbeCache<P, R, NT> &pc,
                                            const float2 *__restrict__ src, int W, int r0, int c0, int c)
{
    constexpr int LDA = Slab<P, R>::LDA, NE = SlabProbeCache<P, R, NT>::NE;
#pragma unroll 1
    for (int k0 = 0; k0 < NE; k0 += 4) {
        float2 o[4], pv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int e = threadIdx.x + (k0 + j) * NT, rl = e / P, x = e % P;
            o[j] = __ldg(src + (size_t)(r0 + c * R + rl) * W + (c0 + x));
        }
        pc.get4(k0, pv);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int e = threadIdx.x + (k0 + j) * NT, rl = e / P, x = e % P;
            buf[rl * LDA + x] = cmul(pv[j], o[j]);
        }
    }
}

// Loader of the forward row step (fft2_fwd_in): x[n1] = p(row, c) * src(r0 + row, c0 + c),
// c = n2 + R2 n1, the probe from the cache (pc) or from global memory (pk); all 16 loads of
// the object are issued before the first product.
template <int P, int NT>
struct ExitWaveLoader {
    const ProbeCache<P, NT> *pc;
    const float2 *pk;
    const float2 *src;
    int W, r0, c0;
    __device__ __forceinline__ void operator()(int ii, int row, int n2, float2 (&x)[16]) const
    {
        constexpr int R2 = Tile<P>::R2;
        const float2 *s0 = src + (size_t)(r0 + row) * W + (c0 + n2);
#pragma unroll
        for (int n1 = 0; n1 < 16; n1++) x[n1] = __ldg(s0 + R2 * n1);
#pragma unroll
        for (int k0 = 0; k0 < 16; k0 += 4) {
            float2 pv[4];
            if (pc) {
                pc->get4(ii * 16 + k0, pv);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) pv[j] = __ldg(pk + row * P + n2 + R2 * (k0 + j));
            }
#pragma unroll
            for (int j = 0; j < 4; j++) x[k0 + j] = cmul(pv[j], x[k0 + j]);
        }
    }
};

// Storer of the inverse row step (fft2_inv_out): w(row, c) = conj(p(row, c)) * x[n1],
// c = n2 + R2 n1, into one pattern's [P][P] result.
template <int P, int NT>
struct AdjointStorer {
    const ProbeCache<P, NT> *pc;
    const float2 *pk;
    float2 *wi;
    __device__ __forceinline__ void operator()(int ii, int row, int n2, const float2 (&x)[16]) const
    {
        constexpr int R2 = Tile<P>::R2;
        float2 *d0 = wi + row * P + n2;
#pragma unroll
        for (int k0 = 0; k0 < 16; k0 += 4) {
            float2 pv[4];
            if (pc) {
                pc->get4(ii * 16 + k0, pv);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) pv[j] = __ldg(pk + row * P + n2 + R2 * (k0 + j));
            }
#pragma unroll
            for (int j = 0; j < 4; j++) d0[R2 * (k0 + j)] = cconjmul(pv[j], x[k0 + j]);
        }
    }
};

// Kahan-compensated single-precision accumulation (per thread; the block sum is FP64).
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x)
{
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Cluster-wide barrier so that no CTA touches a peer's shared memory before the peer runs.
template <int P, int R>
__device__ __forceinline__ void cluster_start()
{
    if constexpr (P != R) cooperative_groups::this_cluster().sync();
}

// ------------------------------------------------------------------------------------
template <int P, int R, int NT>
__global__ void __launch_bounds__(NT, min_ctas<P, R>()) k_forward(PatternArgs a, const float2 *__restrict__ psi,
                                                float2 *__restrict__ out)
{
    extern __shared__ __align__(16) float2 sm[];
    float2 *buf = sm, *tw = sm + Slab<P, R>::ELEMS;
    int i, c;
    who<P, R>(i, c);
    const int2 rc = a.pos[i];
    cluster_start<P, R>();
    load_twiddles<P, NT>(tw, a.tw);
    gather_rows<P, R, NT>(buf, probe_of(a, i), psi, a.W, rc.x, rc.y, c);
    __syncthreads();
    fft2_fwd<P, R, NT>(buf, tw);
    float2 *o = out + (size_t)a.perm[i] * P * P;
    for (int e = threadIdx.x; e < P * R; e += NT) {
        const int r = e / R, xl = e % R;
        o[Tile<P>::nat(r) * P + Tile<P>::nat(c * R + xl)] = buf[r * Slab<P, R>::LDB + xl];
    }
}

// w[i] = conj(p) * (row slab of F^H r) of pattern i (cluster configurations).
template <int P, int R, int NT>
__device__ __forceinline__ void emit_adjoint(const PatternArgs &a, const float2 *buf, float2 *__restrict__ w, int i,
                                             int c)
{
    constexpr int LDA = Slab<P, R>::LDA;
    float2 *wi = w + (size_t)i * P * P;
    const float2 *pk = probe_of(a, i);
    for (int e = threadIdx.x; e < R * P; e += NT) {
        const int rl = e / P, x = e % P, yy = c * R + rl;
        wi[yy * P + x] = cconjmul(__ldg(pk + yy * P + x), buf[rl * LDA + x]);
    }
}

// emit_adjoint with the probe from a SlabProbeCache.
template <int P, int R, int NT>
__device__ __forceinline__ void emit_adjoint(const float2 *buf, const SlabProbeCache<P, R, NT> &pc,
                                             float2 *__restrict__ w, int i, int c)
{
    constexpr int LDA = Slab<P, R>::LDA, NE = SlabProbeCache<P, R, NT>::NE;
    float2 *wi = w + (size_t)i * P * P;
#pragma unroll 1
    for (int k0 = 0; k0 < NE; k0 += 4) {
        float2 pv[4];
        pc.get4(k0, pv);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int e = threadIdx.x + (k0 + j) * NT, rl = e / P, x = e % P;
            wi[(c * R + rl) * P + x] = cconjmul(pv[j], buf[rl * LDA + x]);
        }
    }
}

template <int P, int R, int NT>
__global__ void __launch_bounds__(NT, min_ctas<P, R>()) k_adjoint_fft(PatternArgs a, const float2 *__restrict__ y,
                                                    float2 *__restrict__ w)
{
    extern __shared__ __align__(16) float2 sm[];
    constexpr int LDA = Slab<P, R>::LDA, LDB = Slab<P, R>::LDB;
    float2 *buf = sm, *tw = sm + Slab<P, R>::ELEMS;
    int i, c;
    who<P, R>(i, c);
    cluster_start<P, R>();
    const float2 *yi = y + (size_t)a.perm[i] * P * P;
    load_twiddles<P, NT>(tw, a.tw);
    for (int e = threadIdx.x; e < P * R; e += NT) {
        const int r = e / R, xl = e % R;
        buf[r * LDB + xl] = __ldg(yi + Tile<P>::nat(r) * P + Tile<P>::nat(c * R + xl));
    }
    __syncthreads();
    fft2_inv<P, R, NT>(buf, tw);
    float2 *wi = w + (size_t)i * P * P;
    const float2 *pk = probe_of(a, i);
    for (int e = threadIdx.x; e < R * P; e += NT) {
        const int rl = e / P, x = e % P, yy = c * R + rl;
        wi[yy * P + x] = cconjmul(__ldg(pk + yy * P + x), buf[rl * LDA + x]);
    }
}

// Entry terms of the objective and the residual factor at one detector pixel with counts d,
// a = |u|^2 + eps.  Poisson likelihood (Eq. 2, 3): f = -d log a, r = u (1 - d / a).  Least
// squares on amplitudes: f = d - 2 sqrt(d) sqrt(a), r = u (1 - sqrt(d) / sqrt(a)).  The
// |u|^2 term every pixel contributes is added by the caller; kept is the factor k with
// r = u + k u, i.e. k = -d / a (likelihood) or -sqrt(d / a) (least squares).
__device__ __forceinline__ void entry_terms(int est, float dv, float a, float &f, float &k)
{
    if (est == 0) {
        f = -dv * logf(a);
        k = -dv / a;
    } else {
        const float sd = sqrtf(dv), sa = sqrtf(a);
        f = fmaf(-2.0f * sd, sa, dv);
        k = -sd / sa;
    }
}

// GRAD pattern pass (Eq. 2 and 3 for one pattern).
//   f = sum_j |u_j|^2 + sum_{entries} (entry term: -d log(|u|^2 + eps) for Eq. 2)
//   r = u, except r = u (1 + k) at the entries (k = -d / (|u|^2 + eps) for Eq. 3)
//   w = conj(p) F^H r;  u at the entries is kept for the line search of this iteration.
// One pattern of the GRAD pass (full form).
template <int P, int R, int NT>
__device__ __forceinline__ void grad_pattern(const PatternArgs &a, const float2 *__restrict__ psi,
                                             float2 *__restrict__ w, float2 *__restrict__ fpart, float2 *buf,
                                             const float2 *tw, float2 *red, float2 *tot, int i, int c,
                                             float2 *facc, const ProbeCache<P, NT> *pc,
                                             const SlabProbeCache<P, R, NT> *spc = nullptr)
{
    constexpr int LDB = Slab<P, R>::LDB, CS = Slab<P, R>::CS;
    const int2 rc = a.pos[i];
    if constexpr (R == P) {  // the gather feeds the first row step from registers
        fft2_fwd_in<P, NT>(buf, tw, tw + P, ExitWaveLoader<P, NT>{pc, probe_of(a, i), psi, a.W, rc.x, rc.y});
    } else {
        if (spc) gather_rows<P, R, NT>(buf, *spc, psi, a.W, rc.x, rc.y, c);
        else gather_rows<P, R, NT>(buf, probe_of(a, i), psi, a.W, rc.x, rc.y, c);
        __syncthreads();
        fft2_fwd<P, R, NT>(buf, tw);
    }
    float f = 0.0f;
    for (int e = threadIdx.x; e < P * R; e += NT) {
        const float2 u = buf[(e / R) * LDB + (e % R)];
        f = fmaf(u.x, u.x, fmaf(u.y, u.y, f));
    }
    __syncthreads();
    const int per = a.nzc / CS;  // entry chunks (of the finest column split) owned by this CTA
    const long long e0 = a.nz_off[i * a.nzc + c * per], e1 = a.nz_off[i * a.nzc + (c + 1) * per];
#pragma unroll 2
    for (long long e = e0 + threadIdx.x; e < e1; e += NT) {
        const int s = __ldg(a.nz_slot + e);  // global slot qy * P + qx
        const float dv = __ldg(a.nz_d + e);
        float2 *pu = buf + (s / P) * LDB + (s % P - c * R);
        float2 u = *pu;
        a.nz_u[e] = u;
        const float den = fmaf(u.x, u.x, u.y * u.y) + a.eps;
        float fe, k;
        entry_terms(a.est, dv, den, fe, k);
        f += fe;
        const float sc = 1.0f + k;
        u.x *= sc;
        u.y *= sc;
        *pu = u;
    }
    if (facc) {  // one view, persistent CTA: the thread's running sum over its patterns
        *facc = ff_add_f(*facc, f);
        __syncthreads();  // the residual writes before F^H
    } else {
        float v[1] = {f};
        block_sum_ff<NT, 1>(v, red, tot);  // its barriers also order the residual writes before F^H
        if (threadIdx.x == 0) fpart[i * CS + c] = tot[0];
    }
    if constexpr (R == P) {  // the last row step hands its rows to the emit
        fft2_inv_out<P, NT>(buf, tw, tw + P, AdjointStorer<P, NT>{pc, probe_of(a, i), w + (size_t)i * P * P});
    } else {
        fft2_inv<P, R, NT>(buf, tw);
        if (spc) emit_adjoint<P, R, NT>(buf, *spc, w, i, c);
        else emit_adjoint<P, R, NT>(a, buf, w, i, c);
    }
}

// Persistent passes: the CTAs (CS = 1) or clusters of the grid stride over the patterns.
template <int P, int R, int NT>
__global__ void __launch_bounds__(NT, min_ctas<P, R>()) k_grad(PatternArgs a, const float2 *__restrict__ psi,
                                             float2 *__restrict__ w, float2 *__restrict__ fpart,
                                             const DevState *__restrict__ st)
{
    extern __shared__ __align__(16) float2 sm[];
    constexpr int CS = Slab<P, R>::CS;
    __shared__ float2 red[NT / 32];
    __shared__ float2 tot[1];
    float2 *buf = sm, *tw = sm + Slab<P, R>::ELEMS;
    const int c = blockIdx.x % CS;
    if (st && a.V == 1 && (st->stalled || st->lin)) return;  // one view: decided for all patterns
    cluster_start<P, R>();
    load_twiddles<P, NT>(tw, a.tw);
    auto skip = [&](int i) {
        if (!st || a.V == 1) return false;  // one view: decided above for all patterns
        const DevState &sv = st[a.pat_view[i]];
        return sv.stalled || sv.lin;  // a view in the linear form runs k_grad_lin
    };
    if constexpr (CS == 1) {
        __shared__ uint32_t tmem_slot;
        ProbeCache<P, NT> pc;
        const bool cached = a.probe_stride == 0;  // one probe for all patterns: kept in TMEM
        if (cached) pc.init(&tmem_slot, a.probe);
        // one view: the objective terms are summed per thread over the CTA's patterns and
        // written as one column per CTA (same grid for k_grad and k_grad_lin)
        const bool percta = a.V == 1;
        float2 facc = make_float2(0.f, 0.f);
        for (int i = blockIdx.x; i < a.K; i += gridDim.x) {
            if (skip(i)) continue;
            __syncthreads();  // the previous pattern's reads of buf are done
            grad_pattern<P, R, NT>(a, psi, w, fpart, buf, tw, red, tot, i, 0, percta ? &facc : nullptr,
                                   cached ? &pc : nullptr);
        }
        if (percta) {
            float2 v[1] = {facc};
            block_sum_ff<NT, 1>(v, red, tot);
            if (threadIdx.x == 0) fpart[blockIdx.x] = tot[0];
        }
        if (cached) pc.release();
    } else if constexpr (P < 256) {
        // the optional clusters of smaller P: one pattern per cluster (a loop here raised the
        // register allocation, e.g. 64 -> 127 for the linear pass with clusters of 4)
        const int i = blockIdx.x / CS;
        if (skip(i)) return;  // uniform over the cluster
        grad_pattern<P, R, NT>(a, psi, w, fpart, buf, tw, red, tot, i, c, nullptr, nullptr);
    } else {
        // persistent clusters: each strides over the patterns (the pattern's first exchange
        // starts with a cluster barrier, so a peer writes into this CTA's slab only after
        // this CTA has finished with the previous pattern)
        __shared__ uint32_t tmem_slot;
        SlabProbeCache<P, R, NT> spc;
        // one probe for all patterns and several patterns per cluster: the slab's in TMEM
        const bool cached = a.probe_stride == 0 && (int)(gridDim.x / CS) < a.K;
        if (cached) spc.init(&tmem_slot, a.probe, c);
        for (int i = blockIdx.x / CS; i < a.K; i += gridDim.x / CS) {
            if (skip(i)) continue;  // uniform over the cluster
            __syncthreads();        // this CTA's reads of buf for the previous pattern are done
            grad_pattern<P, R, NT>(a, psi, w, fpart, buf, tw, red, tot, i, c, nullptr, nullptr,
                                   cached ? &spc : nullptr);
        }
        if (cached) spc.release();
    }
}

// LS pattern pass for a window of st->Leff <= L candidate steps gamma_l (Eq. 7 with Eq. 2):
//   F(psi + gamma eta) - F(psi) = sum_j q_j - sum_{entries} d log1p(q / (|u|^2 + eps)),
//   q_j = |u_j + gamma v_j|^2 - |u_j|^2 = gamma (2 Re conj(u_j) v_j + gamma |v_j|^2),
// with u = G psi (kept by the GRAD pass at the entries) and v = G eta (one forward DFT).
// Over all pixels, sum conj(u) v and sum |v|^2 equal P^2 sum conj(x) y and P^2 sum |y|^2
// of the real-space exit waves x = p psi / P, y = p eta / P (Parseval); the d = 0 part is
// that total minus the entries' part.
// GRAD stage in the linear form (Eq. 1 is linear in psi): after an accepted step
// psi_m = psi_{m-1} + gamma eta_{m-1}, the model at the entries is u_m = u_{m-1} + gamma v_{m-1}
// (both kept there), so no forward DFT is needed.  The residual of Eq. 3 differs from u only
// at the entries, r = u + Delta with Delta = k u (k of entry_terms); since F^H u = p psi, the
// pattern's contribution to the gradient is conj(p) F^H Delta plus |p|^2 psi, and the latter
// summed over positions is D psi (D the illumination map), added by the scatter-add.  The
// objective keeps only its entry terms here; sum |u|^2 = P^2 sum D |psi|^2 comes from the
// scatter-add too.  Runs only for views whose st->lin is set.
// One entry of the GRAD pass: slot, count, u and v; ok = false past the pattern's end.
struct EntryIn {
    int s = 0;
    float d = 0.f;
    float2 u = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
    bool ok = false;
    __device__ __forceinline__ void load(const PatternArgs &a, long long e, long long e1)
    {
        ok = e < e1;
        if (ok) {
            s = __ldg(a.nz_slot + e);
            d = __ldg(a.nz_d + e);
            u = a.nz_u[e];
            v = __ldg(a.nz_v + e);
        }
    }
};

// L2 prefetch of the entry arrays of pattern j (all its column chunks): one 128-byte line per
// thread and array, the addresses those of entries of the pattern (the last one included), so
// every address lies inside the arrays.  grad: also the counts and v, which only the GRAD pass
// reads.  Issued at the start of a pattern for the CTA's next one, the entries then arrive
// from L2 instead of HBM.
template <int NT>
__device__ __forceinline__ void prefetch_entries(const PatternArgs &a, int j, bool grad)
{
    const long long e0 = a.nz_off[(size_t)j * a.nzc], e1 = a.nz_off[(size_t)(j + 1) * a.nzc];
    if (e1 <= e0) return;
    const long long n = e1 - e0;
    const int ls = (int)((n + 63) / 64) + 1, ld = (int)((n + 31) / 32) + 1, lu = (int)((n + 15) / 16) + 1;
    const int tot = ls + lu + (grad ? ld + lu : 0);
    for (int t = threadIdx.x; t < tot; t += NT) {
        const void *ptr;
        if (t < ls) ptr = a.nz_slot + min(e0 + 64LL * t, e1 - 1);
        else if (t < ls + lu) ptr = a.nz_u + min(e0 + 16LL * (t - ls), e1 - 1);
        else if (t < ls + lu + ld) ptr = a.nz_d + min(e0 + 32LL * (t - ls - lu), e1 - 1);
        else ptr = a.nz_v + min(e0 + 16LL * (t - ls - lu - ld), e1 - 1);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
    }
}

template <int P, int R, int NT>
__device__ __forceinline__ void grad_lin_pattern(const PatternArgs &a, float2 *__restrict__ w,
                                                 float2 *__restrict__ fpart, float2 *buf, const float2 *tw,
                                                 float2 *red, float2 *tot, float gam, int i, int c, float2 *facc,
                                                 const ProbeCache<P, NT> *pc,
                                                 const SlabProbeCache<P, R, NT> *spc = nullptr)
{
    constexpr int LDB = Slab<P, R>::LDB, CS = Slab<P, R>::CS;
    const int per = a.nzc / CS;
    const long long e0 = a.nz_off[i * a.nzc + c * per], e1 = a.nz_off[i * a.nzc + (c + 1) * per];
    // single CTA with the entry masks: the first inverse pass reads only the entry slots, so
    // the tile is not zeroed (the caller's barrier already ordered the previous pattern's
    // reads before the entries' writes); the mask words are loaded first
    constexpr int NI = R == P ? block_items<P, NT>() : 1;
    const bool masked = R == P && a.nz_mask != nullptr;
    unsigned mw[NI];
    if (masked) {
        constexpr int R2 = Tile<P>::R2;
        const unsigned *m = a.nz_mask + (size_t)i * (P * P / 32);
#pragma unroll
        for (int q = 0; q < NI; q++) {
            const int t = threadIdx.x + q * NT, line = t % P, k1 = t / P;
            mw[q] = __ldg(m + line * (P / 32) + (R2 * k1) / 32) >> ((R2 * k1) % 32);
        }
    }
    // the thread's first two entries are loaded before the zeroing, which hides their latency
    EntryIn first[2];
#pragma unroll
    for (int q = 0; q < 2; q++) first[q].load(a, e0 + threadIdx.x + q * NT, e1);
    if (!masked) {
        // the column slab (permuted spectrum order) starts at zero
        static_assert((P * LDB) % 2 == 0, "16-byte zeroing");
        for (int e = threadIdx.x; e < P * LDB / 2; e += NT)
            reinterpret_cast<float4 *>(buf)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
    }
    float f = 0.0f;
    auto entry = [&](long long e, const EntryIn &x) {
        const float2 u = make_float2(fmaf(gam, x.v.x, x.u.x), fmaf(gam, x.v.y, x.u.y));
        a.nz_u[e] = u;
        const float den = fmaf(u.x, u.x, u.y * u.y) + a.eps;
        float fe, sc;
        entry_terms(a.est, x.d, den, fe, sc);
        f += fe;
        buf[(x.s / P) * LDB + (x.s % P - c * R)] = make_float2(u.x * sc, u.y * sc);
    };
#pragma unroll
    for (int q = 0; q < 2; q++)
        if (first[q].ok) entry(e0 + threadIdx.x + q * NT, first[q]);
#pragma unroll 2
    for (long long e = e0 + threadIdx.x + 2 * NT; e < e1; e += NT) {
        EntryIn x;
        x.load(a, e, e1);
        entry(e, x);
    }
    if (facc) {  // one view, persistent CTA: the thread's running sum over its patterns
        *facc = ff_add_f(*facc, f);
        __syncthreads();  // the writes before F^H
    } else {
        float vv[1] = {f};
        block_sum_ff<NT, 1>(vv, red, tot);  // its barriers also order the writes before F^H
        if (threadIdx.x == 0) fpart[i * CS + c] = tot[0];
    }
    if constexpr (R == P) {  // the last row step hands its rows to the emit
        fft2_inv_out<P, NT>(buf, tw, tw + P, AdjointStorer<P, NT>{pc, probe_of(a, i), w + (size_t)i * P * P},
                            masked ? &mw : nullptr);
    } else {
        fft2_inv<P, R, NT>(buf, tw);
        if (spc) emit_adjoint<P, R, NT>(buf, *spc, w, i, c);
        else emit_adjoint<P, R, NT>(a, buf, w, i, c);
    }
}

template <int P, int R, int NT>
__global__ void __launch_bounds__(NT, min_ctas<P, R>()) k_grad_lin(PatternArgs a, float2 *__restrict__ w, float2 *__restrict__ fpart,
                                                 const DevState *__restrict__ sts)
{
    extern __shared__ __align__(16) float2 sm[];
    constexpr int CS = Slab<P, R>::CS;
    __shared__ float2 red[NT / 32];
    __shared__ float2 tot[1];
    float2 *buf = sm, *tw = sm + Slab<P, R>::ELEMS;
    const int c = blockIdx.x % CS;
    if (a.V == 1 && (sts->stalled || !sts->lin)) return;  // one view: decided for all patterns
    cluster_start<P, R>();
    load_twiddles<P, NT>(tw, a.tw);
    if constexpr (CS == 1) {
        __shared__ uint32_t tmem_slot;
        ProbeCache<P, NT> pc;
        const bool cached = a.probe_stride == 0;  // one probe for all patterns: kept in TMEM
        if (cached) pc.init(&tmem_slot, a.probe);
        const bool percta = a.V == 1;  // as in k_grad
        float2 facc = make_float2(0.f, 0.f);
        const float gam1 = percta ? (float)sts->last_gamma : 0.f;  // one view: loop-invariant
        for (int i = blockIdx.x; i < a.K; i += gridDim.x) {
            float gam = gam1;
            if (!percta) {
                const DevState *st = sts + a.pat_view[i];
                if (st->stalled || !st->lin) continue;
                gam = (float)st->last_gamma;
            }
            if (i + (int)gridDim.x < a.K) prefetch_entries<NT>(a, i + gridDim.x, true);
            __syncthreads();  // the previous pattern's reads of buf are done
            grad_lin_pattern<P, R, NT>(a, w, fpart, buf, tw, red, tot, gam, i, 0, percta ? &facc : nullptr,
                                       cached ? &pc : nullptr);
        }
        if (percta) {
            float2 v[1] = {facc};
            block_sum_ff<NT, 1>(v, red, tot);
            if (threadIdx.x == 0) fpart[blockIdx.x] = tot[0];
        }
        if (cached) pc.release();
    } else if constexpr (P < 256) {  // as in k_grad
        const int i = blockIdx.x / CS;
        const DevState *st = sts + a.pat_view[i];
        if (st->stalled || !st->lin) return;  // uniform over the cluster
        grad_lin_pattern<P, R, NT>(a, w, fpart, buf, tw, red, tot, (float)st->last_gamma, i, c, nullptr, nullptr);
    } else {
        __shared__ uint32_t tmem_slot;
        SlabProbeCache<P, R, NT> spc;
        const bool cached = a.probe_stride == 0 && (int)(gridDim.x / CS) < a.K;  // as in k_grad
        if (cached) spc.init(&tmem_slot, a.probe, c);
        for (int i = blockIdx.x / CS; i < a.K; i += gridDim.x / CS) {  // persistent clusters (k_grad)
            const DevState *st = sts + a.pat_view[i];
            if (st->stalled || !st->lin) continue;  // uniform over the cluster
            __syncthreads();
            grad_lin_pattern<P, R, NT>(a, w, fpart, buf, tw, red, tot, (float)st->last_gamma, i, c, nullptr,
                                       nullptr, cached ? &spc : nullptr);
        }
        if (cached) spc.release();
    }
}

// Rows 2 .. 2 + 2 kCertN of the LS partials when a.dsum is set: a lower bound of this chunk's
// share of the objective change at the leading trials gamma_j = gamma0 tau^(j+1) (Eq. 2, 7).
// With t_e = q_e / (|u_e|^2 + eps) and weights d_e / D (D = sum of the chunk's counts),
// log1p is concave, so by Jensen's inequality
//   sum_e d_e log1p(t_e) <= D log1p(T / D),  T = sum_e d_e t_e = gamma S1 + gamma^2 S2,
//   S1 = sum_e d_e 2 Re conj(u) v / (|u|^2 + eps),  S2 = sum_e d_e |v|^2 / (|u|^2 + eps),
// and the chunk's exact entry term sum_e [q_e - d_e log1p(t_e)] is at least
//   lb_j = gamma (2 B + gamma C) - D log1p(T / D)   (B, C: sums of Re conj(u) v, |v|^2).
// Row 2 + j holds lb_j, row 2 + kCertN + j its magnitude (for the rounding margin); NaN
// where T / D is not safely above -1 (no certificate).  k: row - 2.
__device__ __forceinline__ float2 ls_cert_row(const PatternArgs &a, const DevState &sv, const float2 *tot, int col,
                                              int k)
{
    const int j = k % kCertN;
    const float g = sv.cert_f[j];
    const float B = -(tot[0].x + tot[0].y), C = -(tot[1].x + tot[1].y);
    const float S1 = tot[2].x + tot[2].y, S2 = tot[3].x + tot[3].y;
    const float quad = g * fmaf(g, C, 2.0f * B);
    const float D = a.dsum[col];
    float lb = quad, mag = fabsf(quad);
    if (D > 0.0f) {
        // fast division and log1p (a few ulp): the acceptance margin of k_ls_certify is 1e-4
        const float x = __fdividef(g * fmaf(g, S2, S1), D);
        const float l = x > -1.0f + 1e-6f ? log1p_fast(x) : __int_as_float(0x7fc00000);
        lb = fmaf(-D, l, quad);
        mag = fmaf(D, fabsf(l), mag);
    }
    return ff_from(k < kCertN ? lb : mag);
}

// Rows of the LS partials that the pass writes: 0, 1, and the certificate rows when set.
__device__ __forceinline__ int ls_rows(const PatternArgs &a) { return a.dsum ? 2 + 2 * kCertN : 2; }

// One pattern chunk of the LS pass; thread t < ls_rows(a) receives the chunk's value of row t.
// DEFER: the pass ends after writing its warp partials to red (no barrier); ls_rows_deferred
// turns them into the rows later.
template <int P, int R, int NT, bool DEFER = false>
__device__ __forceinline__ float2 ls_fft_pattern(const PatternArgs &a, const float2 *__restrict__ eta, float2 *buf,
                                                 const float2 *tw, float2 *red, float2 *tot,
                                                 const DevState *__restrict__ sts, int i, int c,
                                                 const ProbeCache<P, NT> *pc)
{
    constexpr int LDB = Slab<P, R>::LDB, CS = Slab<P, R>::CS;
    const int2 rc = a.pos[i];
    // p eta / P into the row slab
    if constexpr (R == P) {  // the gather feeds the first row step from registers
        fft2_fwd_in<P, NT>(buf, tw, tw + P, ExitWaveLoader<P, NT>{pc, probe_of(a, i), eta, a.W, rc.x, rc.y});
    } else {
        gather_rows<P, R, NT>(buf, probe_of(a, i), eta, a.W, rc.x, rc.y, c);
        __syncthreads();
        fft2_fwd<P, R, NT>(buf, tw);
    }
    // v = G eta at the entries (kept for the candidate windows), and the entries' share of
    // the two all-pixel sums, removed here so that rows 0 and 1 cover the pixels without
    // counts; with the certificate also the two weighted sums of its bound
    const bool cert = a.dsum != nullptr;
    float bp = 0.0f, cp = 0.0f, s1 = 0.0f, s2 = 0.0f;
    const int per = a.nzc / CS;
    const long long e0 = a.nz_off[i * a.nzc + c * per], e1 = a.nz_off[i * a.nzc + (c + 1) * per];
#pragma unroll 4
    for (long long e = e0 + threadIdx.x; e < e1; e += NT) {
        const int s = __ldg(a.nz_slot + e);
        const float2 u = __ldg(a.nz_u + e);
        const float2 v = buf[(s / P) * LDB + (s % P - c * R)];
        a.nz_v[e] = v;
        const float re = fmaf(u.x, v.x, u.y * v.y), vv = fmaf(v.x, v.x, v.y * v.y);  // Re conj(u) v, |v|^2
        bp += re;
        cp += vv;
        if (cert) {
            const float wgt = __fdividef(__ldg(a.nz_d + e), fmaf(u.x, u.x, u.y * u.y) + a.eps);
            s1 = fmaf(wgt, 2.0f * re, s1);
            s2 = fmaf(wgt, vv, s2);
        }
    }
    float vals[4] = {-bp, -cp, s1, s2};
    if constexpr (DEFER) {
        const float2 x[4] = {ff_from(vals[0]), ff_from(vals[1]), ff_from(vals[2]), ff_from(vals[3])};
        block_partials_ff<NT, 4>(x, red);
        return make_float2(0.f, 0.f);
    }
    block_sum_ff<NT, 4>(vals, red, tot);
    if (threadIdx.x < 2) return tot[threadIdx.x];
    if (threadIdx.x < ls_rows(a))
        return ls_cert_row(a, sts[a.V == 1 ? 0 : a.pat_view[i]], tot, i * CS + c, threadIdx.x - 2);
    return make_float2(0.f, 0.f);
}

// Warp 0, after a barrier that follows ls_fft_pattern<DEFER = true> of pattern i: the block
// totals from red, then lane l's rows l and l + 32 (zero beyond ls_rows(a)), as the
// undeferred pass gives them to threads l and l + 32.
template <int NT>
__device__ __forceinline__ void ls_rows_deferred(const PatternArgs &a, const DevState *__restrict__ sts,
                                                 const float2 *red, float2 *tot, int i, float2 &r0, float2 &r1)
{
    combine_partials_ff<NT, 4>(red, tot);
    __syncwarp();
    const int lane = threadIdx.x & 31, nr = ls_rows(a);
    const DevState &sv = sts[a.V == 1 ? 0 : a.pat_view[i]];
    r0 = lane < 2 ? tot[lane] : lane < nr ? ls_cert_row(a, sv, tot, i, lane - 2) : make_float2(0.f, 0.f);
    r1 = lane + 32 < nr ? ls_cert_row(a, sv, tot, i, lane + 30) : make_float2(0.f, 0.f);
}

template <int P, int R, int NT>
__global__ void __launch_bounds__(NT, min_ctas<P, R>()) k_ls_fft(PatternArgs a, const float2 *__restrict__ eta,
                                               float2 *__restrict__ part, const DevState *__restrict__ sts)
{
    extern __shared__ __align__(16) float2 sm[];
    constexpr int CS = Slab<P, R>::CS;
    __shared__ float2 red[(NT / 32) * 4];
    __shared__ float2 tot[4];
    float2 *buf = sm, *tw = sm + Slab<P, R>::ELEMS;
    const int c = blockIdx.x % CS;
    if (a.V == 1 && sts->stalled) return;  // one view: decided for all patterns
    cluster_start<P, R>();
    load_twiddles<P, NT>(tw, a.tw);
    const int KC = a.K * CS, nr = ls_rows(a);
    if constexpr (CS == 1) {
        // one view: one column per CTA, its patterns summed in their fixed order
        __shared__ uint32_t tmem_slot;
        ProbeCache<P, NT> pc;
        const bool cached = a.probe_stride == 0;  // one probe for all patterns: kept in TMEM
        if (cached) pc.init(&tmem_slot, a.probe);
        const bool percta = a.V == 1;
        // a pattern's block totals are combined by warp 0 after the next barrier (the next
        // pattern's first, or the one after the loop): lane l keeps rows l and l + 32
        float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
        int prev = -1;
        auto finish = [&]() {
            float2 r0, r1;
            ls_rows_deferred<NT>(a, sts, red, tot, prev, r0, r1);
            const int lane = threadIdx.x & 31;
            if (percta) {
                acc0 = ff_add(acc0, r0);
                acc1 = ff_add(acc1, r1);
            } else {
                if (lane < nr) part[(size_t)lane * KC + prev] = r0;
                if (lane + 32 < nr) part[(size_t)(lane + 32) * KC + prev] = r1;
            }
        };
        for (int i = blockIdx.x; i < a.K; i += gridDim.x) {
            if (!percta && sts[a.pat_view[i]].stalled) continue;  // one view: decided above
            if (i + (int)gridDim.x < a.K) prefetch_entries<NT>(a, i + gridDim.x, false);
            __syncthreads();  // the previous pattern's reads of buf and its partials are done
            if (prev >= 0 && threadIdx.x < 32) finish();
            ls_fft_pattern<P, R, NT, true>(a, eta, buf, tw, red, tot, sts, i, 0, cached ? &pc : nullptr);
            prev = i;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            if (prev >= 0) finish();
            const int lane = threadIdx.x;
            if (percta && lane < nr) part[(size_t)lane * KC + blockIdx.x] = acc0;
            if (percta && lane + 32 < nr) part[(size_t)(lane + 32) * KC + blockIdx.x] = acc1;
        }
        if (cached) pc.release();
    } else if constexpr (P < 256) {  // as in k_grad
        const int i = blockIdx.x / CS;
        if (sts[a.pat_view[i]].stalled) return;  // uniform over the cluster
        const float2 r = ls_fft_pattern<P, R, NT>(a, eta, buf, tw, red, tot, sts, i, c, nullptr);
        if (threadIdx.x < nr) part[(size_t)threadIdx.x * KC + i * CS + c] = r;
    } else {
        // persistent clusters as in k_grad; the probe from L2 (the slab cache measured slower
        // here: spiral LS pass 4.45 -> 4.61 ms with R = 64)
        for (int i = blockIdx.x / CS; i < a.K; i += gridDim.x / CS) {
            if (sts[a.pat_view[i]].stalled) continue;  // uniform over the cluster
            __syncthreads();
            const float2 r = ls_fft_pattern<P, R, NT>(a, eta, buf, tw, red, tot, sts, i, c, nullptr);
            if (threadIdx.x < nr) part[(size_t)threadIdx.x * KC + i * CS + c] = r;
        }
    }
}

// Global slot (qy * P + qx) and natural-order index of local slot s of column chunk c.
template <int P, int R>
__device__ __forceinline__ int chunk_slot(int s, int c)
{
    return (s / R) * P + c * R + (s % R);
}
template <int P, int R>
__device__ __forceinline__ int slot_to_natural(int s, int c)
{
    return Tile<P>::nat(s / R) * P + Tile<P>::nat(c * R + (s % R));
}

// Counts per (pattern, CTA) chunk.
template <int P, int R, int NT>
__global__ void __launch_bounds__(NT) k_nz_count(const float *__restrict__ d, const int *__restrict__ perm,
                                                 int *__restrict__ cnt)
{
    __shared__ int red[NT / 32];
    constexpr int CS = Slab<P, R>::CS;
    const int i = blockIdx.x / CS, c = blockIdx.x % CS;
    const float *dk = d + (size_t)perm[i] * P * P;
    int n = 0;
    for (int s = threadIdx.x; s < P * R; s += NT) n += dk[slot_to_natural<P, R>(s, c)] > 0.0f;
    n = __reduce_add_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w2 = 0; w2 < NT / 32; w2++) t += red[w2];
        cnt[blockIdx.x] = t;
    }
}

// Ordered compaction: entries of chunk (pattern i, column chunk c) in ascending local slot
// order, stored as global slots so that any configuration with R >= this R can read them.
template <int P, int R, int NT>
__global__ void __launch_bounds__(NT) k_nz_fill(const float *__restrict__ d, const int *__restrict__ perm,
                                                const long long *__restrict__ off, unsigned short *__restrict__ slot,
                                                float *__restrict__ dval)
{
    __shared__ int wsum[NT / 32];
    constexpr int CS = Slab<P, R>::CS;
    const int i = blockIdx.x / CS, c = blockIdx.x % CS;
    const float *dk = d + (size_t)perm[i] * P * P;
    const long long base = off[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long running = 0;
    for (int s0 = 0; s0 < P * R; s0 += NT) {
        const int s = s0 + threadIdx.x;
        const float v = dk[slot_to_natural<P, R>(s, c)];
        const bool flag = v > 0.0f;
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        int woff = 0, total = 0;
        for (int w2 = 0; w2 < NT / 32; w2++) {
            woff += (w2 < warp) ? wsum[w2] : 0;
            total += wsum[w2];
        }
        if (flag) {
            const long long p = base + running + woff + __popc(m & ((1u << lane) - 1u));
            slot[p] = (unsigned short)chunk_slot<P, R>(s, c);
            dval[p] = v;
        }
        running += total;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// Launch helpers: cluster launch when CS > 1.
template <typename... KArgs, typename... Args>
cudaError_t launch_pattern(void (*kern)(KArgs...), int nblocks, int nthreads, size_t smem, int cs, cudaStream_t s,
                           Args... args)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3((unsigned)nthreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (cs > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Grid of a persistent pattern kernel: with one CTA per pattern (cs = 1), the CTAs that fit
// on the device at once (by the kernel's occupancy), at most one per pattern; with clusters
// (cs > 1) and persist_clusters, the clusters that fit at once
// (cudaOccupancyMaxActiveClusters: fewer than the per-CTA occupancy suggests), each striding
// over the patterns, else one cluster per pattern.  Persistent clusters pay where a pattern
// needs them (P = 256; spiral workload, 10,000 positions: 13.82 -> 12.97 ms per iteration);
// the optional clusters of P = 128 keep one cluster per pattern and a kernel without the
// pattern loop (with it, the compiler's register allocation rose, e.g. 63 -> 99 registers
// for the LS pass with clusters of 4, and fewer CTAs fit on an SM).
template <typename... KArgs>
int persistent_blocks(void (*kern)(KArgs...), int nslices, int nthreads, size_t smem, int cs,
                      bool persist_clusters = false)
{
    if (cs > 1) {
        if (!persist_clusters) return nslices;
        // the clusters that fit on the device at once, at most one per pattern
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)nslices);
        cfg.blockDim = dim3((unsigned)nthreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) {
            cudaGetLastError();
            return nslices;
        }
        const long long g = (long long)ncl * cs;
        return g < nslices ? (int)g : nslices;
    }
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthreads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return nslices;
    }
    int g = nsm * per_sm;
    g -= g % cs;
    if (g < cs) g = cs;
    return g < nslices ? g : nslices;
}

// All launchers of one (P, R, NT) configuration.
template <int P, int R, int NT>
struct PatternOps {
    static constexpr int CS = Slab<P, R>::CS;
    static cudaError_t forward(const PatternArgs &a, const float2 *psi, float2 *out, cudaStream_t s)
    {
        return launch_pattern(k_forward<P, R, NT>, a.K * CS, NT, slab_bytes<P, R>(), CS, s, a, psi, out);
    }
    static cudaError_t adjoint(const PatternArgs &a, const float2 *y, float2 *w, cudaStream_t s)
    {
        return launch_pattern(k_adjoint_fft<P, R, NT>, a.K * CS, NT, slab_bytes<P, R>(), CS, s, a, y, w);
    }
    // One view, single CTA: both GRAD kernels run the same grid and write one objective
    // column per CTA (returned); otherwise 0 (one column per pattern chunk).
    static int grad_cols(const PatternArgs &a)
    {
        if (CS != 1 || a.V != 1) return 0;
        const int g1 = persistent_blocks(k_grad<P, R, NT>, a.K, NT, slab_bytes<P, R>(), CS);
        const int g2 = persistent_blocks(k_grad_lin<P, R, NT>, a.K, NT, slab_bytes<P, R>(), CS);
        return g1 < g2 ? g1 : g2;
    }
    static cudaError_t grad(const PatternArgs &a, const float2 *psi, float2 *w, float2 *fpart, const DevState *st,
                            cudaStream_t s)
    {
        const int gc = grad_cols(a);
        const int g = gc > 0 ? gc : persistent_blocks(k_grad<P, R, NT>, a.K * CS, NT, slab_bytes<P, R>(), CS, P >= 256);
        return launch_pattern(k_grad<P, R, NT>, g, NT, slab_bytes<P, R>(), CS, s, a, psi, w, fpart, st);
    }
    static cudaError_t grad_lin(const PatternArgs &a, float2 *w, float2 *fpart, const DevState *st, cudaStream_t s)
    {
        const int gc = grad_cols(a);
        const int g = gc > 0 ? gc : persistent_blocks(k_grad_lin<P, R, NT>, a.K * CS, NT, slab_bytes<P, R>(), CS, P >= 256);
        return launch_pattern(k_grad_lin<P, R, NT>, g, NT, slab_bytes<P, R>(), CS, s, a, w, fpart, st);
    }
    static cudaError_t ls(const PatternArgs &a, const float2 *eta, float2 *part, const DevState *st, cudaStream_t s)
    {
        const int g = persistent_blocks(k_ls_fft<P, R, NT>, a.K * CS, NT, slab_bytes<P, R>(), CS, P >= 256);
        return launch_pattern(k_ls_fft<P, R, NT>, g, NT, slab_bytes<P, R>(), CS, s, a, eta, part, st);
    }
    static int ls_cols(const PatternArgs &a)
    {
        if (CS != 1 || a.V != 1) return 0;
        return persistent_blocks(k_ls_fft<P, R, NT>, a.K * CS, NT, slab_bytes<P, R>(), CS, P >= 256);
    }
    static cudaError_t nz_count(const float *d, const int *perm, int K, int *cnt, cudaStream_t s)
    {
        k_nz_count<P, R, NT><<<K * CS, NT, 0, s>>>(d, perm, cnt);
        return cudaGetLastError();
    }
    static cudaError_t nz_fill(const float *d, const int *perm, int K, const long long *off, unsigned short *slot,
                               float *dval, cudaStream_t s)
    {
        k_nz_fill<P, R, NT><<<K * CS, NT, 0, s>>>(d, perm, off, slot, dval);
        return cudaGetLastError();
    }
};

template <int P, int R, int NT>
constexpr PatternImpl make_impl()
{
    using O = PatternOps<P, R, NT>;
    return PatternImpl{P, R, NT, &O::forward, &O::adjoint, &O::grad, &O::grad_lin, &O::ls, &O::ls_cols, &O::grad_cols, &O::nz_count,
                       &O::nz_fill};
}

}  // namespace pty

// pattern_kernels.cu -- the per-scan-position passes of ML-CG: one thread block owns one
// diffraction pattern, keeps its P x P exit wave in shared memory and runs the 2-D DFTs
// of fft_tile.cuh on it.
//
//   k_forward      Eq. 1: u = F(p * patch(psi)) written out (pty_forward)
//   k_adjoint_fft  the F^H and conj(p) factors of G^H (pty_adjoint)
//   k_grad         GRAD stage: gather x probe -> F -> likelihood residual (Eq. 3) and the
//                  objective terms (Eq. 2) -> F^H -> x conj(p); one patch-sized result
//                  per pattern, summed into the object by the scatter kernel
//   k_ls           LS stage: v = G eta for one pattern, then the change of the objective
//                  F(psi + gamma eta) - F(psi) (Eq. 2, 7) for a window of candidate steps
//                  gamma, using G(psi + gamma eta) = u + gamma v with u kept by k_grad
//   k_nz_*         create time: the compact list of detector pixels with counts
//
// The forward DFT leaves the spectrum in the permuted slot order of fft_tile.cuh; the
// measured data are stored in that order, and the inverse DFT returns to natural order,
// so no separate reordering pass exists.
#include "fft_tile.cuh"
#include "mathx.cuh"
#include "pty_internal.h"
#include "reduce.cuh"

namespace pty {

template <int P>
struct Cfg;
template <>
struct Cfg<64> {
    static constexpr int NT_A = 256;  // GRAD pass threads
    static constexpr int NT_B = 256;  // LS pass threads
    static constexpr int NT_F = 256;  // forward / adjoint / data compaction
};
template <>
struct Cfg<128> {
    static constexpr int NT_A = 512;
    static constexpr int NT_B = 512;
    static constexpr int NT_F = 512;
};

template <int P>
constexpr size_t tile_bytes()
{
    return sizeof(float2) * (size_t)(Tile<P>::ELEMS + P);
}

template <int P, int NT>
__device__ __forceinline__ void load_twiddles(float2 *tw, const float2 *__restrict__ g_tw)
{
    for (int m = threadIdx.x; m < P; m += NT) tw[m] = g_tw[m];
}

// tile[y][x] = probe[y][x] * src[r + y][c + x]  (Q of Eq. 1)
template <int P, int NT>
__device__ __forceinline__ void gather_patch(float2 *tile, const float2 *__restrict__ probe,
                                             const float2 *__restrict__ src, int W, int r, int c)
{
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int y = e / P, x = e % P;
        tile[y * Tile<P>::LD + x] = cmul(__ldg(probe + e), __ldg(src + (size_t)(r + y) * W + (c + x)));
    }
}

// ------------------------------------------------------------------------------------
template <int P, int NT>
__global__ void __launch_bounds__(NT) k_forward(PatternArgs a, const float2 *__restrict__ psi,
                                                float2 *__restrict__ out)
{
    extern __shared__ __align__(16) float2 sm[];
    float2 *tile = sm, *tw = sm + Tile<P>::ELEMS;
    const int i = blockIdx.x;
    const int2 rc = a.pos[i];
    load_twiddles<P, NT>(tw, a.tw);
    gather_patch<P, NT>(tile, a.probe, psi, a.W, rc.x, rc.y);
    __syncthreads();
    fft2_fwd<P, NT>(tile, tw);
    float2 *o = out + (size_t)a.perm[i] * P * P;
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int qy = e / P, qx = e % P;
        o[Tile<P>::nat(qy) * P + Tile<P>::nat(qx)] = tile[qy * Tile<P>::LD + qx];
    }
}

template <int P, int NT>
__global__ void __launch_bounds__(NT) k_adjoint_fft(PatternArgs a, const float2 *__restrict__ y,
                                                    float2 *__restrict__ w)
{
    extern __shared__ __align__(16) float2 sm[];
    float2 *tile = sm, *tw = sm + Tile<P>::ELEMS;
    const int i = blockIdx.x;
    const float2 *yi = y + (size_t)a.perm[i] * P * P;
    load_twiddles<P, NT>(tw, a.tw);
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int ky = e / P, kx = e % P;
        tile[Tile<P>::slot(ky) * Tile<P>::LD + Tile<P>::slot(kx)] = __ldg(yi + e);
    }
    __syncthreads();
    fft2_inv<P, NT>(tile, tw);
    float2 *wi = w + (size_t)i * P * P;
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int yy = e / P, xx = e % P;
        wi[e] = cconjmul(__ldg(a.probe + e), tile[yy * Tile<P>::LD + xx]);
    }
}

// Kahan-compensated single-precision accumulation (per thread; the block sum is FP64).
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x)
{
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// GRAD pattern pass (Eq. 2 and 3 for one pattern).
//   f = sum_j |u_j|^2 - sum_{entries} d log(|u|^2 + eps)
//   r = u, except r = u (1 - d / (|u|^2 + eps)) at the entries
//   w = conj(p) F^H r;  u at the entries is kept for the line search of this iteration.
template <int P, int NT>
__global__ void __launch_bounds__(NT) k_grad(PatternArgs a, const float2 *__restrict__ psi,
                                             float2 *__restrict__ w, double *__restrict__ fpart,
                                             const DevState *__restrict__ st)
{
    if (st && st->stalled) return;
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[NT / 32];
    __shared__ double tot[1];
    float2 *tile = sm, *tw = sm + Tile<P>::ELEMS;
    const int i = blockIdx.x;
    const int2 rc = a.pos[i];
    load_twiddles<P, NT>(tw, a.tw);
    gather_patch<P, NT>(tile, a.probe, psi, a.W, rc.x, rc.y);
    __syncthreads();
    fft2_fwd<P, NT>(tile, tw);
    float f = 0.0f;
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const float2 u = tile[(e / P) * Tile<P>::LD + (e % P)];
        f = fmaf(u.x, u.x, fmaf(u.y, u.y, f));
    }
    __syncthreads();
    const long long e0 = a.nz_off[i], e1 = a.nz_off[i + 1];
    for (long long e = e0 + threadIdx.x; e < e1; e += NT) {
        const int s = a.nz_slot[e];
        const float dv = a.nz_d[e];
        float2 *pu = tile + (s / P) * Tile<P>::LD + (s % P);
        float2 u = *pu;
        a.nz_u[e] = u;
        const float den = fmaf(u.x, u.x, u.y * u.y) + a.eps;
        f -= dv * logf(den);
        const float sc = 1.0f - dv / den;
        u.x *= sc;
        u.y *= sc;
        *pu = u;
    }
    double v[1] = {(double)f};
    block_sum<NT, 1>(v, red, tot);  // its barriers also order the residual writes before F^H
    if (threadIdx.x == 0) fpart[i] = tot[0];
    fft2_inv<P, NT>(tile, tw);
    float2 *wi = w + (size_t)i * P * P;
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int yy = e / P, xx = e % P;
        wi[e] = cconjmul(__ldg(a.probe + e), tile[yy * Tile<P>::LD + xx]);
    }
}

// LS pattern pass for a window of L candidate steps gamma_l (Eq. 7 with Eq. 2):
//   F(psi + gamma eta) - F(psi) = sum_j q_j - sum_{entries} d log1p(q / (|u|^2 + eps)),
//   q_j = |u_j + gamma v_j|^2 - |u_j|^2 = gamma (2 Re conj(u_j) v_j + gamma |v_j|^2),
// with u = G psi (kept by the GRAD pass at the entries) and v = G eta (one forward DFT).
// Over all pixels, sum conj(u) v and sum |v|^2 equal P^2 sum conj(x) y and P^2 sum |y|^2
// of the real-space exit waves x = p psi / P, y = p eta / P (Parseval); the d = 0 part is
// that total minus the entries' part.
template <int P, int NT, int L>
__global__ void __launch_bounds__(NT) k_ls(PatternArgs a, const float2 *__restrict__ psi,
                                           const float2 *__restrict__ g, const float2 *__restrict__ ep,
                                           double *__restrict__ part, const DevState *__restrict__ st)
{
    if (st->stalled || st->decided) return;
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[(NT / 32) * (L + 2)];
    __shared__ double tot[L + 2];
    float2 *tile = sm, *tw = sm + Tile<P>::ELEMS;
    const int i = blockIdx.x;
    const int2 rc = a.pos[i];
    const float alpha = (float)st->alpha;
    float gam[L];
#pragma unroll
    for (int l = 0; l < L; l++) gam[l] = (float)st->cand[l];
    load_twiddles<P, NT>(tw, a.tw);

    // y = p eta / P into the tile, with the real-space sums of Parseval's identity
    float sb = 0.f, sbc = 0.f, scc = 0.f, sccc = 0.f;
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int y = e / P, x = e % P;
        const size_t o = (size_t)(rc.x + y) * a.W + (rc.y + x);
        const float2 gv = __ldg(g + o), ev = __ldg(ep + o), pv = __ldg(a.probe + e);
        const float2 eta = make_float2(fmaf(alpha, ev.x, -gv.x), fmaf(alpha, ev.y, -gv.y));
        const float2 yv = cmul(pv, eta), xv = cmul(pv, __ldg(psi + o));
        tile[y * Tile<P>::LD + x] = yv;
        kahan_add(sb, sbc, fmaf(xv.x, yv.x, xv.y * yv.y));
        kahan_add(scc, sccc, fmaf(yv.x, yv.x, yv.y * yv.y));
    }
    __syncthreads();
    fft2_fwd<P, NT>(tile, tw);

    float bp = 0.0f, cp = 0.0f, acc[L];
#pragma unroll
    for (int l = 0; l < L; l++) acc[l] = 0.0f;
    const long long e0 = a.nz_off[i], e1 = a.nz_off[i + 1];
    for (long long e = e0 + threadIdx.x; e < e1; e += NT) {
        const int s = a.nz_slot[e];
        const float dv = a.nz_d[e];
        const float2 u = a.nz_u[e];
        const float2 v = tile[(s / P) * Tile<P>::LD + (s % P)];
        const float au = fmaf(u.x, u.x, u.y * u.y);
        const float bu = fmaf(u.x, v.x, u.y * v.y);  // Re conj(u) v
        const float cu = fmaf(v.x, v.x, v.y * v.y);
        bp += bu;
        cp += cu;
        const float inv = 1.0f / (au + a.eps);
        const float tmin = -au * inv;  // |u + gamma v|^2 >= 0
#pragma unroll
        for (int l = 0; l < L; l++) {
            const float q = gam[l] * fmaf(gam[l], cu, 2.0f * bu);
            const float t = fmaxf(q * inv, tmin);
            acc[l] += q - dv * log1p_fast(t);
        }
    }
    constexpr double PP = (double)P * (double)P;
    double vals[L + 2];
    vals[0] = PP * ((double)sb - (double)sbc) - (double)bp;
    vals[1] = PP * ((double)scc - (double)sccc) - (double)cp;
#pragma unroll
    for (int l = 0; l < L; l++) vals[2 + l] = acc[l];
    block_sum<NT, L + 2>(vals, red, tot);
    if (threadIdx.x < L + 2) part[(size_t)threadIdx.x * a.K + i] = tot[threadIdx.x];  // [L+2][K]
}

__global__ void k_selftest_log1p(const float *__restrict__ t, float *__restrict__ out, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = log1p_fast(t[i]);
}

cudaError_t launch_selftest_log1p(const float *t, float *out, int n, cudaStream_t s)
{
    k_selftest_log1p<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(t, out, n);
    return cudaGetLastError();
}

// Natural-order index of tile slot s.
template <int P>
__device__ __forceinline__ int slot_to_natural(int s)
{
    return Tile<P>::nat(s / P) * P + Tile<P>::nat(s % P);
}

template <int P, int NT>
__global__ void __launch_bounds__(NT) k_nz_count(const float *__restrict__ d, const int *__restrict__ perm,
                                                 int *__restrict__ cnt)
{
    __shared__ int red[NT / 32];
    const float *dk = d + (size_t)perm[blockIdx.x] * P * P;
    int c = 0;
    for (int s = threadIdx.x; s < P * P; s += NT) c += dk[slot_to_natural<P>(s)] > 0.0f;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < NT / 32; w++) t += red[w];
        cnt[blockIdx.x] = t;
    }
}

// Ordered compaction: entries of sorted pattern i in ascending slot order.
template <int P, int NT>
__global__ void __launch_bounds__(NT) k_nz_fill(const float *__restrict__ d, const int *__restrict__ perm,
                                                const long long *__restrict__ off, unsigned short *__restrict__ slot,
                                                float *__restrict__ dval)
{
    __shared__ int wsum[NT / 32];
    const float *dk = d + (size_t)perm[blockIdx.x] * P * P;
    const long long base = off[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long running = 0;
    for (int s0 = 0; s0 < P * P; s0 += NT) {
        const int s = s0 + threadIdx.x;
        const float v = dk[slot_to_natural<P>(s)];
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
            slot[p] = (unsigned short)s;
            dval[p] = v;
        }
        running += total;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
template <typename KernelT>
static cudaError_t set_smem(KernelT k, size_t bytes)
{
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

bool pattern_supported(int P) { return P == 64 || P == 128; }
int ls_window_supported(int L) { return L == 4 || L == 8 || L == 16 || L == 32; }

template <int P>
static cudaError_t forward_p(const PatternArgs &a, const float2 *psi, float2 *out, cudaStream_t s)
{
    constexpr int NT = Cfg<P>::NT_F;
    auto k = k_forward<P, NT>;
    cudaError_t e = set_smem(k, tile_bytes<P>());
    if (e != cudaSuccess) return e;
    k<<<a.K, NT, tile_bytes<P>(), s>>>(a, psi, out);
    return cudaGetLastError();
}

template <int P>
static cudaError_t adjoint_p(const PatternArgs &a, const float2 *y, float2 *w, cudaStream_t s)
{
    constexpr int NT = Cfg<P>::NT_F;
    auto k = k_adjoint_fft<P, NT>;
    cudaError_t e = set_smem(k, tile_bytes<P>());
    if (e != cudaSuccess) return e;
    k<<<a.K, NT, tile_bytes<P>(), s>>>(a, y, w);
    return cudaGetLastError();
}

template <int P>
static cudaError_t grad_p(const PatternArgs &a, const float2 *psi, float2 *w, double *fpart, const DevState *st,
                          cudaStream_t s)
{
    constexpr int NT = Cfg<P>::NT_A;
    auto k = k_grad<P, NT>;
    cudaError_t e = set_smem(k, tile_bytes<P>());
    if (e != cudaSuccess) return e;
    k<<<a.K, NT, tile_bytes<P>(), s>>>(a, psi, w, fpart, st);
    return cudaGetLastError();
}

template <int P, int L>
static cudaError_t ls_pl(const PatternArgs &a, const float2 *psi, const float2 *g, const float2 *ep, double *part,
                         const DevState *st, cudaStream_t s)
{
    constexpr int NT = Cfg<P>::NT_B;
    auto k = k_ls<P, NT, L>;
    cudaError_t e = set_smem(k, tile_bytes<P>());
    if (e != cudaSuccess) return e;
    k<<<a.K, NT, tile_bytes<P>(), s>>>(a, psi, g, ep, part, st);
    return cudaGetLastError();
}

template <int P>
static cudaError_t ls_p(const PatternArgs &a, int L, const float2 *psi, const float2 *g, const float2 *ep,
                        double *part, const DevState *st, cudaStream_t s)
{
    switch (L) {
    case 4: return ls_pl<P, 4>(a, psi, g, ep, part, st, s);
    case 8: return ls_pl<P, 8>(a, psi, g, ep, part, st, s);
    case 16: return ls_pl<P, 16>(a, psi, g, ep, part, st, s);
    case 32: return ls_pl<P, 32>(a, psi, g, ep, part, st, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int P>
static cudaError_t nz_count_p(const float *d, const int *perm, int K, int *cnt, cudaStream_t s)
{
    k_nz_count<P, Cfg<P>::NT_F><<<K, Cfg<P>::NT_F, 0, s>>>(d, perm, cnt);
    return cudaGetLastError();
}

template <int P>
static cudaError_t nz_fill_p(const float *d, const int *perm, int K, const long long *off, unsigned short *slot,
                             float *dval, cudaStream_t s)
{
    k_nz_fill<P, Cfg<P>::NT_F><<<K, Cfg<P>::NT_F, 0, s>>>(d, perm, off, slot, dval);
    return cudaGetLastError();
}

cudaError_t launch_nz_count(int P, const float *d, const int *perm, int K, int *cnt, cudaStream_t s)
{
    switch (P) {
    case 64: return nz_count_p<64>(d, perm, K, cnt, s);
    case 128: return nz_count_p<128>(d, perm, K, cnt, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_nz_fill(int P, const float *d, const int *perm, int K, const long long *off,
                           unsigned short *slot, float *dval, cudaStream_t s)
{
    switch (P) {
    case 64: return nz_fill_p<64>(d, perm, K, off, slot, dval, s);
    case 128: return nz_fill_p<128>(d, perm, K, off, slot, dval, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_forward(int P, const PatternArgs &a, const float2 *psi, float2 *out, cudaStream_t s)
{
    switch (P) {
    case 64: return forward_p<64>(a, psi, out, s);
    case 128: return forward_p<128>(a, psi, out, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_fft(int P, const PatternArgs &a, const float2 *y, float2 *w, cudaStream_t s)
{
    switch (P) {
    case 64: return adjoint_p<64>(a, y, w, s);
    case 128: return adjoint_p<128>(a, y, w, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_grad(int P, const PatternArgs &a, const float2 *psi, float2 *w, double *fpart,
                        const DevState *st, cudaStream_t s)
{
    switch (P) {
    case 64: return grad_p<64>(a, psi, w, fpart, st, s);
    case 128: return grad_p<128>(a, psi, w, fpart, st, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ls(int P, const PatternArgs &a, const LsArgs &ls, const float2 *psi, const float2 *g,
                      const float2 *eta_prev, double *part, const DevState *st, cudaStream_t s)
{
    switch (P) {
    case 64: return ls_p<64>(a, ls.L, psi, g, eta_prev, part, st, s);
    case 128: return ls_p<128>(a, ls.L, psi, g, eta_prev, part, st, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pty

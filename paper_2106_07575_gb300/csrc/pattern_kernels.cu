// pattern_kernels.cu -- the per-scan-position passes of ML-CG: one thread block owns one
// diffraction pattern, keeps its P x P exit wave in shared memory and runs the 2-D DFTs
// of fft_tile.cuh on it.
//
//   k_forward      Eq. 1: u = F(p * patch(psi)) written out (pty_forward)
//   k_adjoint_fft  the F^H and conj(p) factors of G^H (pty_adjoint)
//   k_grad         GRAD stage: gather x probe -> F -> likelihood residual (Eq. 3) and the
//                  objective terms (Eq. 2) -> F^H -> x conj(p); one patch-sized result
//                  per pattern, summed into the object by the scatter kernel
//   k_ls           LS stage: u = G psi and v = G eta for one pattern, then the change of
//                  the objective F(psi + gamma eta) - F(psi) (Eq. 2, 7) for a window of
//                  candidate steps gamma, using G(psi + gamma eta) = u + gamma v
//
// The forward DFT leaves the spectrum in the permuted slot order of fft_tile.cuh; the
// elementwise steps read the measured data at the matching natural index, and the
// inverse DFT returns to natural order, so no separate reordering pass exists.
#include "fft_tile.cuh"
#include "pty_internal.h"
#include "reduce.cuh"

namespace pty {

template <int P>
struct Cfg;
template <>
struct Cfg<64> {
    static constexpr int NT_A = 256;  // GRAD pass threads
    static constexpr int NT_B = 256;  // LS pass threads (holds u in registers: P*P/NT_B complex)
    static constexpr int NT_F = 256;  // forward / adjoint
};
template <>
struct Cfg<128> {
    static constexpr int NT_A = 512;
    static constexpr int NT_B = 256;
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

// Same with the Dai-Yuan direction eta = -g + alpha eta_prev formed on the fly (Eq. 6).
template <int P, int NT>
__device__ __forceinline__ void gather_direction(float2 *tile, const float2 *__restrict__ probe,
                                                 const float2 *__restrict__ g, const float2 *__restrict__ ep,
                                                 float alpha, int W, int r, int c)
{
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int y = e / P, x = e % P;
        const size_t o = (size_t)(r + y) * W + (c + x);
        const float2 gv = __ldg(g + o), ev = __ldg(ep + o);
        const float2 eta = make_float2(fmaf(alpha, ev.x, -gv.x), fmaf(alpha, ev.y, -gv.y));
        tile[y * Tile<P>::LD + x] = cmul(__ldg(probe + e), eta);
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

// GRAD pattern pass (Eq. 2 and 3 for one pattern).
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
    const float *d = a.data + (size_t)a.perm[i] * P * P;
    load_twiddles<P, NT>(tw, a.tw);
    gather_patch<P, NT>(tile, a.probe, psi, a.W, rc.x, rc.y);
    __syncthreads();
    fft2_fwd<P, NT>(tile, tw);
    // u - d u / (|u|^2 + eps) and |u|^2 - d log(|u|^2 + eps), slot by slot
    float f = 0.0f;
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int qy = e / P, qx = e % P;
        const float dv = __ldg(d + Tile<P>::nat(qy) * P + Tile<P>::nat(qx));
        float2 u = tile[qy * Tile<P>::LD + qx];
        const float au = fmaf(u.x, u.x, u.y * u.y);
        if (dv > 0.0f) {
            const float den = au + a.eps;
            f += au - dv * logf(den);
            const float s = 1.0f - dv / den;
            u.x *= s;
            u.y *= s;
            tile[qy * Tile<P>::LD + qx] = u;
        } else {
            f += au;
        }
    }
    double v[1] = {(double)f};
    block_sum<NT, 1>(v, red, tot);
    if (threadIdx.x == 0) fpart[i] = tot[0];
    fft2_inv<P, NT>(tile, tw);
    float2 *wi = w + (size_t)i * P * P;
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int yy = e / P, xx = e % P;
        wi[e] = cconjmul(__ldg(a.probe + e), tile[yy * Tile<P>::LD + xx]);
    }
}

// LS pattern pass for a window of L candidate steps.
template <int P, int NT, int L>
__global__ void __launch_bounds__(NT) k_ls(PatternArgs a, const float2 *__restrict__ psi,
                                           const float2 *__restrict__ g, const float2 *__restrict__ ep,
                                           double *__restrict__ part, const DevState *__restrict__ st)
{
    if (st->stalled || st->decided) return;
    constexpr int NS = P * P / NT;  // slots per thread
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[(NT / 32) * (L + 2)];
    __shared__ double tot[L + 2];
    float2 *tile = sm, *tw = sm + Tile<P>::ELEMS;
    const int i = blockIdx.x;
    const int2 rc = a.pos[i];
    const float *d = a.data + (size_t)a.perm[i] * P * P;
    const float alpha = (float)st->alpha;
    float gam[L];
#pragma unroll
    for (int l = 0; l < L; l++) gam[l] = (float)st->cand[l];

    load_twiddles<P, NT>(tw, a.tw);
    gather_patch<P, NT>(tile, a.probe, psi, a.W, rc.x, rc.y);
    __syncthreads();
    fft2_fwd<P, NT>(tile, tw);
    float2 u[NS];
#pragma unroll
    for (int j = 0; j < NS; j++) {
        const int e = threadIdx.x + NT * j, qy = e / P, qx = e % P;
        u[j] = tile[qy * Tile<P>::LD + qx];
    }
    __syncthreads();
    gather_direction<P, NT>(tile, a.probe, g, ep, alpha, a.W, rc.x, rc.y);
    __syncthreads();
    fft2_fwd<P, NT>(tile, tw);

    float b0 = 0.0f, c0 = 0.0f, acc[L];
#pragma unroll
    for (int l = 0; l < L; l++) acc[l] = 0.0f;
#pragma unroll
    for (int j = 0; j < NS; j++) {
        const int e = threadIdx.x + NT * j, qy = e / P, qx = e % P;
        const float2 v = tile[qy * Tile<P>::LD + qx];
        const float dv = __ldg(d + Tile<P>::nat(qy) * P + Tile<P>::nat(qx));
        const float au = fmaf(u[j].x, u[j].x, u[j].y * u[j].y);
        const float bu = fmaf(u[j].x, v.x, u[j].y * v.y);  // Re conj(u) v
        const float cu = fmaf(v.x, v.x, v.y * v.y);
        if (dv > 0.0f) {
            // |u + gamma v|^2 - |u|^2 = q; objective change q - d log1p(q / (|u|^2 + eps))
            const float inv = 1.0f / (au + a.eps);
            const float tmin = -au * inv;
#pragma unroll
            for (int l = 0; l < L; l++) {
                const float q = gam[l] * fmaf(gam[l], cu, 2.0f * bu);
                const float t = fmaxf(q * inv, tmin);
                acc[l] += q - dv * log1pf(t);
            }
        } else {
            b0 += bu;
            c0 += cu;
        }
    }
    double vals[L + 2];
    vals[0] = b0;
    vals[1] = c0;
#pragma unroll
    for (int l = 0; l < L; l++) vals[2 + l] = acc[l];
    block_sum<NT, L + 2>(vals, red, tot);
    if (threadIdx.x < L + 2) part[(size_t)i * (L + 2) + threadIdx.x] = tot[threadIdx.x];
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

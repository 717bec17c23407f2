// tc_cg.cu -- the per-pattern steps of ML-CG around the tensor-core DFT (tc_dft.cu), where
// the spectra u = G psi and v = G eta are materialised in natural DFT order.
//
//   k_tc_residual    Eq. 2 and 3 at one pattern: objective terms, residual in place at the
//                    pixels with counts, u kept there for the line search
//   k_tc_gather_eta  Q of Eq. 1 for the direction eta = -g + alpha eta_prev (Eq. 6), with the
//                    real-space sums that Parseval's identity equates to the spectral sums
//   k_tc_ls_entries  the objective change of Eq. 7 for a window of candidate steps
// The compact measured data ("entries") are stored with tile slots of the FFT path; the
// natural index of slot (qy, qx) is (nat(qy), nat(qx)).
#include "fft_tile.cuh"
#include "mathx.cuh"
#include "pty_internal.h"
#include "reduce.cuh"

namespace pty {
namespace {

constexpr int kNT = 256;

template <int P>
__device__ __forceinline__ int entry_natural(int s)
{
    return Tile<P>::nat(s / P) * P + Tile<P>::nat(s % P);
}

template <int P>
__global__ void __launch_bounds__(kNT) k_tc_residual(PatternArgs a, float2 *__restrict__ U, float2 *__restrict__ fpart,
                                                     const DevState *__restrict__ st)
{
    const int i = blockIdx.x;
    if (st && st[a.pat_view[i]].stalled) return;
    __shared__ float2 red[kNT / 32];
    __shared__ float2 tot[1];
    float2 *ui = U + (size_t)i * P * P;
    float f = 0.0f;
    for (int e = threadIdx.x; e < P * P; e += kNT) {
        const float2 u = ui[e];
        f = fmaf(u.x, u.x, fmaf(u.y, u.y, f));
    }
    __syncthreads();
    const long long e0 = a.nz_off[(size_t)i * a.nzc], e1 = a.nz_off[(size_t)(i + 1) * a.nzc];
    for (long long e = e0 + threadIdx.x; e < e1; e += kNT) {
        const int j = entry_natural<P>(a.nz_slot[e]);
        const float dv = a.nz_d[e];
        float2 u = ui[j];
        a.nz_u[e] = u;
        const float den = fmaf(u.x, u.x, u.y * u.y) + a.eps;
        f -= dv * logf(den);
        const float sc = 1.0f - dv / den;
        u.x *= sc;
        u.y *= sc;
        ui[j] = u;
    }
    float v[1] = {f};
    block_sum_ff<kNT, 1>(v, red, tot);
    if (threadIdx.x == 0) fpart[i] = tot[0];
}

__device__ __forceinline__ void kahan(float &sum, float &comp, float x)
{
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

template <int P>
__global__ void __launch_bounds__(kNT) k_tc_gather_eta(PatternArgs a, const float2 *__restrict__ psi,
                                                       const float2 *__restrict__ g, const float2 *__restrict__ ep,
                                                       float2 *__restrict__ X, float2 *__restrict__ pars,
                                                       const DevState *__restrict__ sts)
{
    const int i = blockIdx.x;
    const DevState *st = sts + a.pat_view[i];
    if (st->stalled) return;
    __shared__ float2 red[(kNT / 32) * 2];
    __shared__ float2 tot[2];
    const float alpha = st->alpha_f;
    const int2 rc = a.pos[i];
    float2 *xi = X + (size_t)i * P * P;
    float sb = 0.f, sbc = 0.f, sc = 0.f, scc = 0.f;
    for (int e = threadIdx.x; e < P * P; e += kNT) {
        const int y = e / P, x = e % P;
        const size_t o = (size_t)(rc.x + y) * a.W + (rc.y + x);
        const float2 gv = __ldg(g + o), ev = __ldg(ep + o), pv = __ldg(a.probe + e);
        const float2 eta = make_float2(fmaf(alpha, ev.x, -gv.x), fmaf(alpha, ev.y, -gv.y));
        const float2 yv = cmul(pv, eta), xv = cmul(pv, __ldg(psi + o));
        xi[e] = yv;
        kahan(sb, sbc, fmaf(xv.x, yv.x, xv.y * yv.y));
        kahan(sc, scc, fmaf(yv.x, yv.x, yv.y * yv.y));
    }
    // the compensated pairs are float-float values (sum - comp); P^2 is a power of two
    constexpr float PP = (float)P * (float)P;
    float2 v[2] = {make_float2(PP * sb, -PP * sbc), make_float2(PP * sc, -PP * scc)};
    block_sum_ff<kNT, 2>(v, red, tot);
    if (threadIdx.x < 2) pars[(size_t)threadIdx.x * a.K + i] = tot[threadIdx.x];
}

template <int P, int L>
__global__ void __launch_bounds__(kNT) k_tc_ls_entries(PatternArgs a, const float2 *__restrict__ V,
                                                       const float2 *__restrict__ pars, float2 *__restrict__ part,
                                                       const DevState *__restrict__ sts)
{
    const int i = blockIdx.x;
    const DevState *st = sts + a.pat_view[i];
    if (st->stalled || st->decided || st->Lsel != L) return;
    __shared__ float2 red[(kNT / 32) * L];
    __shared__ float2 tot[L + 2];
    const int Leff = st->Leff;
    float gam[L];
#pragma unroll
    for (int l = 0; l < L; l++) gam[l] = st->cand_f[l];
    const float2 *vi = V + (size_t)i * P * P;
    float bp = 0.0f, cp = 0.0f, acc[L];
#pragma unroll
    for (int l = 0; l < L; l++) acc[l] = 0.0f;
    const long long e0 = a.nz_off[(size_t)i * a.nzc], e1 = a.nz_off[(size_t)(i + 1) * a.nzc];
    for (long long e = e0 + threadIdx.x; e < e1; e += kNT) {
        const float2 v = vi[entry_natural<P>(a.nz_slot[e])];
        const float2 u = a.nz_u[e];
        const float dv = a.nz_d[e];
        const float au = fmaf(u.x, u.x, u.y * u.y);
        const float bu = fmaf(u.x, v.x, u.y * v.y);
        const float cu = fmaf(v.x, v.x, v.y * v.y);
        bp += bu;
        cp += cu;
        const float inv = 1.0f / (au + a.eps);
        const float tmin = -au * inv;
#pragma unroll
        for (int l = 0; l < L; l++) {
            if (l < Leff) {
                const float q = gam[l] * fmaf(gam[l], cu, 2.0f * bu);
                const float t = fmaxf(q * inv, tmin);
                acc[l] += q - dv * log1p_fast(t);
            }
        }
    }
    block_sum_ff<kNT, L>(acc, red, tot + 2);  // ends with a barrier: red is free again
    const float bc[2] = {-bp, -cp};
    block_sum_ff<kNT, 2>(bc, red, tot);
    if (threadIdx.x < L + 2) {
        float2 t = tot[threadIdx.x];
        if (threadIdx.x < 2) t = ff_add(t, pars[(size_t)threadIdx.x * a.K + i]);  // d = 0 part: total minus entries
        part[(size_t)threadIdx.x * a.K + i] = t;
    }
}

}  // namespace

cudaError_t launch_tc_residual(const PatternArgs &a, int P, float2 *U, float2 *fpart, const DevState *st,
                               cudaStream_t s)
{
    if (P == 64) k_tc_residual<64><<<a.K, kNT, 0, s>>>(a, U, fpart, st);
    else if (P == 128) k_tc_residual<128><<<a.K, kNT, 0, s>>>(a, U, fpart, st);
    else if (P == 256) k_tc_residual<256><<<a.K, kNT, 0, s>>>(a, U, fpart, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_tc_gather_eta(const PatternArgs &a, int P, const float2 *psi, const float2 *g, const float2 *ep,
                                 float2 *X, float2 *pars, const DevState *st, cudaStream_t s)
{
    if (P == 64) k_tc_gather_eta<64><<<a.K, kNT, 0, s>>>(a, psi, g, ep, X, pars, st);
    else if (P == 128) k_tc_gather_eta<128><<<a.K, kNT, 0, s>>>(a, psi, g, ep, X, pars, st);
    else if (P == 256) k_tc_gather_eta<256><<<a.K, kNT, 0, s>>>(a, psi, g, ep, X, pars, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <int P>
static cudaError_t ls_entries_p(const PatternArgs &a, int L, const float2 *V, const float2 *pars, float2 *part,
                                const DevState *st, cudaStream_t s)
{
    switch (L) {
    case 4: k_tc_ls_entries<P, 4><<<a.K, kNT, 0, s>>>(a, V, pars, part, st); break;
    case 8: k_tc_ls_entries<P, 8><<<a.K, kNT, 0, s>>>(a, V, pars, part, st); break;
    case 16: k_tc_ls_entries<P, 16><<<a.K, kNT, 0, s>>>(a, V, pars, part, st); break;
    case 32: k_tc_ls_entries<P, 32><<<a.K, kNT, 0, s>>>(a, V, pars, part, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_tc_ls_entries(const PatternArgs &a, int P, int L, const float2 *V, const float2 *pars,
                                 float2 *part, const DevState *st, cudaStream_t s)
{
    if (P == 64) return ls_entries_p<64>(a, L, V, pars, part, st, s);
    if (P == 128) return ls_entries_p<128>(a, L, V, pars, part, st, s);
    if (P == 256) return ls_entries_p<256>(a, L, V, pars, part, st, s);
    return cudaErrorInvalidValue;
}

}  // namespace pty

// ls_entries.cu -- line-search candidate windows over the detector pixels with counts.
//
// With u = G psi_m and v = G eta_m kept at every entry (pixel with d > 0) by the GRAD and
// LS pattern passes, the objective at a candidate step gamma changes by (Eq. 2, 7)
//   sum_entries [ q - d log(1 + q / (|u|^2 + eps)) ] + (pixels without counts: Parseval)
//   q = gamma (2 Re conj(u) v + gamma |v|^2) = |u + gamma v|^2 - |u|^2,
// and for the least-squares estimator on amplitudes (a = |u|^2 + eps)
//   sum_entries [ q - 2 sqrt(d) (sqrt(a + q) - sqrt(a)) ],  sqrt(a + q) - sqrt(a) = q / (sqrt(a + q) + sqrt(a))
// (the quotient form has no cancellation when q is small against a).
// One thread block per (pattern, chunk) of the entry layout sums the window's candidates in
// FP32 per thread and in float-float across the block (an FP64 butterfly over 16 values
// kept the FP64 pipe 72 % busy and set the kernel's time) into rows 2.. of [L+2][K * cs]:
// one column per unit, or with one view one column per CTA (its units summed in their fixed
// order), so that the decision kernel reads few partials.  The
// kernel needs no shared-memory tile and runs at full occupancy, which hides the latency
// of the logarithm chain.
#include "mathx.cuh"
#include "pty_internal.h"
#include "reduce.cuh"

namespace pty {

namespace {

constexpr int kNT = 256;

// Fixed grid of kBlocks CTAs striding over the (pattern, chunk) units, so that a window
// launched after the step was decided costs one short launch.  Units differ in their entry
// counts; smaller shares balance them (production workload, windows stage per iteration:
// 608 CTAs 0.149, 1216 0.139, 1824 0.128-0.132, 2280 0.132, 3600 0.131 ms).
constexpr int kBlocks = 152 * 12;

// Values of a window's block sum: L rounded up to a power of two, so that the float-float
// reduction takes its recursive-halving form (the padding values are zero).
template <int L>
constexpr int reduced_width()
{
    return L <= 4 ? 4 : L <= 8 ? 8 : L <= 16 ? 16 : 32;
}

template <int L>
__global__ void __launch_bounds__(kNT) k_ls_entries(PatternArgs a, int cs, int V, float2 *__restrict__ part,
                                                    const DevState *__restrict__ sts)
{
    // one view: a window with nothing to evaluate ends the whole launch at once
    if (V == 1 && (sts->stalled || sts->decided || sts->Lsel != L)) return;
    constexpr int LR = reduced_width<L>();
    __shared__ float2 red[(kNT / 32) * LR];
    __shared__ float2 tot[LR];
    const int nunits = a.K * cs;
    const size_t KC = (size_t)nunits;
    float2 cta = make_float2(0.f, 0.f);  // one view: thread l < L sums candidate l over the CTA's units
    for (int blk = blockIdx.x; blk < nunits; blk += gridDim.x) {
        const int i = blk / cs, c = blk % cs;
        const DevState *st = sts + (V == 1 ? 0 : a.pat_view[i]);
        if (st->stalled || st->decided || st->Lsel != L) continue;  // uniform over the block
        // candidates beyond the open window are evaluated at gamma = 0 and never read
        const int Leff = st->Leff;
        float gam[L];
#pragma unroll
        for (int l = 0; l < L; l++) gam[l] = l < Leff ? st->cand_f[l] : 0.0f;
        float acc[L];
#pragma unroll
        for (int l = 0; l < L; l++) acc[l] = 0.0f;
        const int per = a.nzc / cs;
        const long long e0 = a.nz_off[i * a.nzc + c * per], e1 = a.nz_off[i * a.nzc + (c + 1) * per];
        if (blk + (int)gridDim.x < nunits) {  // the CTA's next unit's entries into L2
            const int i2 = (blk + gridDim.x) / cs, c2 = (blk + gridDim.x) % cs;
            const long long f0 = a.nz_off[i2 * a.nzc + c2 * per], f1 = a.nz_off[i2 * a.nzc + (c2 + 1) * per];
            const int nd = (int)((f1 - f0 + 31) / 32) + 1, nu = (int)((f1 - f0 + 15) / 16) + 1;
            if (f1 > f0)
                for (int t = threadIdx.x; t < nd + 2 * nu; t += kNT) {
                    const void *ptr = t < nd        ? (const void *)(a.nz_d + min(f0 + 32LL * t, f1 - 1))
                                      : t < nd + nu ? (const void *)(a.nz_u + min(f0 + 16LL * (t - nd), f1 - 1))
                                                    : (const void *)(a.nz_v + min(f0 + 16LL * (t - nd - nu), f1 - 1));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
                }
        }
        // the next entry's values are loaded before this entry's candidates are evaluated
        long long e = e0 + threadIdx.x;
        float dn = 0.f;
        float2 un = make_float2(0.f, 0.f), vn = un;
        if (e < e1) {
            dn = __ldg(a.nz_d + e);
            un = __ldg(a.nz_u + e);
            vn = __ldg(a.nz_v + e);
        }
        for (; e < e1; e += kNT) {
            const float dv = dn;
            const float2 u = un, v = vn;
            if (e + kNT < e1) {
                dn = __ldg(a.nz_d + e + kNT);
                un = __ldg(a.nz_u + e + kNT);
                vn = __ldg(a.nz_v + e + kNT);
            }
            const float au = fmaf(u.x, u.x, u.y * u.y);
            const float bu2 = 2.0f * fmaf(u.x, v.x, u.y * v.y);  // 2 Re conj(u) v
            const float cu = fmaf(v.x, v.x, v.y * v.y);
            if (a.est == 0) {
                const float inv = 1.0f / (au + a.eps);
                const float tmin = -au * inv;  // |u + gamma v|^2 >= 0
#pragma unroll
                for (int l = 0; l < L; l++) {
                    const float q = gam[l] * fmaf(gam[l], cu, bu2);
                    const float t = fmaxf(q * inv, tmin);
                    acc[l] = fmaf(-dv, log1p_fast(t), acc[l] + q);
                }
            } else {
                const float s0 = sqrtf(au + a.eps), sd2 = 2.0f * sqrtf(dv);
#pragma unroll
                for (int l = 0; l < L; l++) {
                    const float q = fmaxf(gam[l] * fmaf(gam[l], cu, bu2), -au);  // |u + gamma v|^2 >= 0
                    const float den = s0 + sqrtf(au + a.eps + q);
                    acc[l] += den > 0.0f ? q - sd2 * (q / den) : q;
                }
            }
        }
        float accr[LR];
#pragma unroll
        for (int l = 0; l < LR; l++) accr[l] = l < L ? acc[l] : 0.0f;
        block_sum_ff<kNT, LR>(accr, red, tot);  // ends with a barrier: red is free again
        if (V == 1) {
            if (threadIdx.x < L) cta = ff_add(cta, tot[threadIdx.x]);
        } else if (threadIdx.x < L) {
            part[(size_t)(2 + threadIdx.x) * KC + blk] = tot[threadIdx.x];
        }
    }
    if (V == 1 && threadIdx.x < L) part[(size_t)(2 + threadIdx.x) * KC + blockIdx.x] = cta;
}

}  // namespace

int ls_entries_cols(const PatternArgs &a, int cs, int V)
{
    return V == 1 ? (a.K * cs < kBlocks ? a.K * cs : kBlocks) : 0;
}

cudaError_t launch_ls_entries(const PatternArgs &a, int cs, int V, int L, float2 *part, const DevState *st,
                              cudaStream_t s)
{
    const int nb = a.K * cs < kBlocks ? a.K * cs : kBlocks;
    switch (L) {
    case 4: k_ls_entries<4><<<nb, kNT, 0, s>>>(a, cs, V, part, st); break;
    case 6: k_ls_entries<6><<<nb, kNT, 0, s>>>(a, cs, V, part, st); break;
    case 8: k_ls_entries<8><<<nb, kNT, 0, s>>>(a, cs, V, part, st); break;
    case 16: k_ls_entries<16><<<nb, kNT, 0, s>>>(a, cs, V, part, st); break;
    case 32: k_ls_entries<32><<<nb, kNT, 0, s>>>(a, cs, V, part, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pty

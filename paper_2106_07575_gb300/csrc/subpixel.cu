// subpixel.cu -- one probe per scan position for fractional positions (pty_create_subpixel).
//
// The paper gives the scan positions of Algorithm 1 as float32 and does not say how a
// fraction enters Q.  A position s is taken as the window floor(s) with the probe moved by
// delta = s - floor(s) inside it, by the Fourier shift theorem:
//   p_delta = F^H[ F[p](ky, kx) phi_dy(ky) phi_dx(kx) ],
//   phi_d(kappa) = exp(-2 pi i kappa d / P) at the signed frequency kappa of index j
//   (j for j < P/2, j - P above), and cos(pi d) at the Nyquist index j = P/2.
// The factor is separable, so along one axis the shift is the circular convolution with
//   h_d[m] = (1/P) sum_j phi_d(kappa_j) exp(2 pi i kappa_j m / P),
// computed per position and axis, then applied along the rows (dx) and the columns (dy).
// This runs once, at context creation; the results replace the shared probe in every
// pattern kernel (PatternArgs::probe_stride = P * P).
#include <algorithm>

#include "pty_internal.h"

namespace pty {
namespace {

// h[(k * 2 + axis) * P + m], axis 0 = rows (dy), 1 = columns (dx); one block per (position,
// axis) of P threads.  Each term is exp(2 pi i ((kappa m) mod P) / P) exp(-2 pi i kappa d / P)
// with both phases reduced exactly before the sine and cosine; the sum over j is in FP64.
__global__ void k_shift_kernels(const float2 *__restrict__ frac, int P, float2 *__restrict__ h)
{
    const int k = blockIdx.x >> 1, ax = blockIdx.x & 1, m = threadIdx.x;
    const float d = ax == 0 ? frac[k].x : frac[k].y;
    float2 *hk = h + ((size_t)k * 2 + ax) * P;
    if (d == 0.0f) {  // no shift: the exact unit impulse
        hk[m] = make_float2(m == 0 ? 1.0f : 0.0f, 0.0f);
        return;
    }
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < P; j++) {
        if (j == P / 2) {
            const float cd = cospif(d);  // cos(pi d) exp(-i pi m) = cos(pi d) (-1)^m
            sr += (m & 1) ? -cd : cd;
            continue;
        }
        const int kap = j < P / 2 ? j : j - P;
        const int km = ((kap * m) % P + P) % P;
        float s1, c1, s2, c2;
        sincospif(2.0f * (float)km / (float)P, &s1, &c1);
        sincospif(-2.0f * ((float)kap * d) / (float)P, &s2, &c2);
        sr += (double)fmaf(c1, c2, -s1 * s2);
        si += (double)fmaf(s1, c2, c1 * s2);
    }
    hk[m] = make_float2((float)(sr / P), (float)(si / P));
}

__device__ __forceinline__ float2 cmadd(float2 a, float2 b, float2 acc)
{
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}

// Rows (shift by dx): tmp[kk][r][c] = sum_c' h_dx[(c - c') mod P] p[r][c'] for positions
// k0 + kk; one block per (kk, r) of P threads.
__global__ void k_shift_rows(const float2 *__restrict__ probe, const float2 *__restrict__ h, int P, int k0,
                             float2 *__restrict__ tmp)
{
    extern __shared__ float2 sm[];
    const int kk = blockIdx.x / P, r = blockIdx.x % P, c = threadIdx.x;
    sm[c] = probe[(size_t)r * P + c];
    sm[P + c] = h[((size_t)(k0 + kk) * 2 + 1) * P + c];
    __syncthreads();
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < P; q++) acc = cmadd(sm[P + ((c - q) & (P - 1))], sm[q], acc);
    tmp[((size_t)kk * P + r) * P + c] = acc;
}

constexpr int kColTile = 16;  // columns per block of the column pass
constexpr int kColNT = 256;

// Columns (shift by dy): out[k0 + kk][r][c] = sum_r' h_dy[(r - r') mod P] tmp[kk][r'][c]; one
// block per (kk, tile of kColTile columns), the tile's P x kColTile inputs in shared memory.
__global__ void __launch_bounds__(kColNT) k_shift_cols(const float2 *__restrict__ tmp, const float2 *__restrict__ h,
                                                       int P, int k0, float2 *__restrict__ out)
{
    extern __shared__ float2 sm[];  // [P][kColTile] inputs, then h_dy [P]
    const int ntile = P / kColTile;
    const int kk = blockIdx.x / ntile, c0 = (blockIdx.x % ntile) * kColTile;
    const float2 *src = tmp + (size_t)kk * P * P;
    for (int e = threadIdx.x; e < P * kColTile; e += kColNT)
        sm[e] = src[(size_t)(e / kColTile) * P + c0 + e % kColTile];
    const float2 *hy = h + ((size_t)(k0 + kk) * 2) * P;
    for (int e = threadIdx.x; e < P; e += kColNT) sm[P * kColTile + e] = hy[e];
    __syncthreads();
    const float2 *hs = sm + P * kColTile;
    const int cl = threadIdx.x % kColTile;
    float2 *dst = out + (size_t)(k0 + kk) * P * P;
    for (int r = threadIdx.x / kColTile; r < P; r += kColNT / kColTile) {
        float2 acc = make_float2(0.f, 0.f);
        for (int q = 0; q < P; q++) acc = cmadd(hs[(r - q) & (P - 1)], sm[q * kColTile + cl], acc);
        dst[(size_t)r * P + c0 + cl] = acc;
    }
}

}  // namespace

cudaError_t launch_shift_probes(int P, int K, const float2 *probe, const float2 *frac, float2 *out, cudaStream_t s)
{
    if (P < kColTile || P > 1024 || (P & (P - 1)) || K < 1) return cudaErrorInvalidValue;
    float2 *h = nullptr, *tmp = nullptr;
    const size_t PP = (size_t)P * P;
    const int chunk = (int)std::max<size_t>(1, ((size_t)64 << 20) / (PP * sizeof(float2)));
    cudaError_t e = cudaMallocAsync(&h, sizeof(float2) * 2 * (size_t)K * P, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&tmp, sizeof(float2) * (size_t)std::min(chunk, K) * PP, s);
    if (e == cudaSuccess) {
        k_shift_kernels<<<2 * K, P, 0, s>>>(frac, P, h);
        e = cudaGetLastError();
    }
    const size_t smem_c = sizeof(float2) * ((size_t)P * kColTile + P);
    if (e == cudaSuccess && smem_c > 48 * 1024)
        e = cudaFuncSetAttribute(k_shift_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
    for (int k0 = 0; k0 < K && e == cudaSuccess; k0 += chunk) {
        const int n = std::min(chunk, K - k0);
        k_shift_rows<<<n * P, P, sizeof(float2) * 2 * P, s>>>(probe, h, P, k0, tmp);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        k_shift_cols<<<n * (P / kColTile), kColNT, smem_c, s>>>(tmp, h, P, k0, out);
        e = cudaGetLastError();
    }
    if (tmp) cudaFreeAsync(tmp, s);
    if (h) cudaFreeAsync(h, s);
    return e;
}

}  // namespace pty

// noalloc.cu -- objective and gradient for callers that cannot allocate device memory.
//
// pty_gradient_noalloc computes the same objective and gradient as pty_gradient, without a
// context: every array is the caller's, and the only scratch is the file-scope device array
// below, of fixed size.  Typical callers are code that runs where device allocation is not
// allowed or not possible: inside another framework's memory budget with no allocator hook,
// in a plug-in that must not grow the process's device footprint, or on a path that must
// not synchronise the device the way cudaMalloc/cudaFree can.
//
// The scratch array lives in device memory on every device where this module is loaded and
// stays there until the process exits.  All calls share it and it keeps the last call's
// contents, so two calls that overlap on the GPU (different streams or threads, no ordering
// between them) race on it and give wrong results; calls on one stream are ordered and safe.
// Each call looks up the array's device address on the current device (cudaGetSymbolAddress,
// once per device), reads a status flag back and synchronises its stream, so it cannot be
// called while that stream is being captured into a CUDA graph.  The stream must belong to
// the current device.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "fft_tile.cuh"
#include "pty.h"
#include "reduce.cuh"

namespace {

// Scratch layout (byte offsets into the array); each region 256-byte aligned.
constexpr long long kNaMaxPixels = 1LL << 22;  // K * P * P complex values of the per-pattern results
constexpr int kNaMaxK = 16384;                 // scan positions
constexpr size_t kNaOffW = 0;
constexpr size_t kNaOffF = kNaOffW + sizeof(float2) * (size_t)kNaMaxPixels;  // fpart[K] (double)
constexpr size_t kNaOffTw = kNaOffF + sizeof(double) * (size_t)kNaMaxK;      // twiddles [P] (float2)
constexpr size_t kNaOffFlag = kNaOffTw + 256 * sizeof(float2);                // int: bad position seen
constexpr size_t kNaBytes = kNaOffFlag + 256;                                  // 32 MiB + 130.25 KiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDev = 64;
std::mutex g_na_mutex;
void *g_na_base[kNaMaxDev] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t na_base(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_base[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_base[dev] = p;
    }
    *out = g_na_base[dev];
    return cudaSuccess;
}

struct NaArgs {
    unsigned char *base;
    int H, W, P, K;
    const float2 *probe;  // [P][P], unscaled
    const int2 *pos;      // [K] (row, col), caller order
    const float *data;    // [K][P][P], natural DFT order
    float eps;
    const float2 *psi;
    float2 *grad;
    double *F;
};

__device__ __forceinline__ float2 *na_w(const NaArgs &a) { return (float2 *)(a.base + kNaOffW); }
__device__ __forceinline__ double *na_fpart(const NaArgs &a) { return (double *)(a.base + kNaOffF); }
__device__ __forceinline__ float2 *na_tw(const NaArgs &a) { return (float2 *)(a.base + kNaOffTw); }
__device__ __forceinline__ int *na_flag(const NaArgs &a) { return (int *)(a.base + kNaOffFlag); }

// Twiddles exp(-2 pi i m / P) in double, rounded once; position check; flag cleared first.
__global__ void k_na_prep(NaArgs a)
{
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int m = threadIdx.x; m < a.P; m += blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)a.P, &s, &c);
        na_tw(a)[m] = make_float2((float)c, (float)s);
    }
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const int2 rc = a.pos[k];
        if (rc.x < 0 || rc.y < 0 || rc.x > a.H - a.P || rc.y > a.W - a.P) atomicOr(&bad, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *na_flag(a) = bad;
}

// Per pattern: u = F(p/P * patch), f and the residual at pixels with counts, w = conj(p/P) F^H r.
template <int P, int NT>
__global__ void __launch_bounds__(NT) k_na_grad(NaArgs a)
{
    if (*na_flag(a)) return;
    using pty::Tile;
    extern __shared__ __align__(16) float2 sm[];
    __shared__ float2 red[NT / 32];
    __shared__ float2 tot[1];
    float2 *tile = sm, *tw = sm + Tile<P>::ELEMS;
    const int k = blockIdx.x;
    const int2 rc = a.pos[k];
    const float inv = 1.0f / (float)P;  // exact: P is a power of two
    for (int m = threadIdx.x; m < P; m += NT) tw[m] = na_tw(a)[m];
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int y = e / P, x = e % P;
        float2 p = a.probe[e];
        p.x *= inv;
        p.y *= inv;
        tile[y * Tile<P>::LD + x] = pty::cmul(p, a.psi[(size_t)(rc.x + y) * a.W + (rc.y + x)]);
    }
    __syncthreads();
    pty::fft2_fwd<P, NT>(tile, tw);
    const float *d = a.data + (size_t)k * P * P;
    float f = 0.0f;
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int qy = e / P, qx = e % P;
        const float dv = d[Tile<P>::nat(qy) * P + Tile<P>::nat(qx)];
        float2 u = tile[qy * Tile<P>::LD + qx];
        const float au = fmaf(u.x, u.x, u.y * u.y);
        f += au;
        if (dv > 0.0f) {
            const float den = au + a.eps;
            f -= dv * logf(den);
            const float s = 1.0f - dv / den;
            u.x *= s;
            u.y *= s;
            tile[qy * Tile<P>::LD + qx] = u;
        }
    }
    float v[1] = {f};
    pty::block_sum_ff<NT, 1>(v, red, tot);
    if (threadIdx.x == 0) na_fpart(a)[k] = pty::ff_value(tot[0]);
    pty::fft2_inv<P, NT>(tile, tw);
    float2 *wk = na_w(a) + (size_t)k * P * P;
    for (int e = threadIdx.x; e < P * P; e += NT) {
        const int y = e / P, x = e % P;
        float2 p = a.probe[e];
        p.x *= inv;
        p.y *= inv;
        wk[e] = pty::cconjmul(p, tile[y * Tile<P>::LD + x]);
    }
}

// Scatter-add: one block per 32 x 64 object tile, patterns in caller order (fixed order).
template <int P>
__global__ void __launch_bounds__(256) k_na_scatter(NaArgs a, int ntile_x)
{
    if (*na_flag(a)) return;
    const int ty = blockIdx.x / ntile_x, tx = blockIdx.x % ntile_x;
    const int x = tx * 64 + (threadIdx.x % 64);
    const int y0 = ty * 32 + threadIdx.x / 64;
    float2 acc[8];
#pragma unroll
    for (int j = 0; j < 8; j++) acc[j] = make_float2(0.f, 0.f);
    for (int k = 0; k < a.K; k++) {
        const int2 rc = a.pos[k];
        if (rc.x >= ty * 32 + 32 || rc.x + P <= ty * 32 || rc.y >= tx * 64 + 64 || rc.y + P <= tx * 64) continue;
        const int dx = x - rc.y;
        if (dx < 0 || dx >= P) continue;
        const float2 *wk = na_w(a) + (size_t)k * P * P + dx;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int yy = y0 + 4 * j - rc.x;
            if (yy >= 0 && yy < P) {
                const float2 v = wk[yy * P];
                acc[j].x += v.x;
                acc[j].y += v.y;
            }
        }
    }
    if (x < a.W) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int y = y0 + 4 * j;
            if (y < a.H) a.grad[(size_t)y * a.W + x] = acc[j];
        }
    }
}

__global__ void __launch_bounds__(256) k_na_sum(NaArgs a)
{
    if (*na_flag(a)) return;
    __shared__ double red[8];
    __shared__ double tot[1];
    double s = 0.0;
    for (int k = threadIdx.x; k < a.K; k += 256) s += na_fpart(a)[k];
    double v[1] = {s};
    pty::block_sum<256, 1>(v, red, tot);
    if (threadIdx.x == 0 && a.F) *a.F = tot[0];
}

template <int P, int NT>
cudaError_t na_launch(const NaArgs &a, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (size_t)(pty::Tile<P>::ELEMS + P);
    cudaError_t e = cudaFuncSetAttribute(k_na_grad<P, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_na_grad<P, NT><<<a.K, NT, smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int ntx = (a.W + 63) / 64, nty = (a.H + 31) / 32;
    k_na_scatter<P><<<ntx * nty, 256, 0, s>>>(a, ntx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_na_sum<<<1, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// The kernels read positions as int2 and complex values as float2 / double: 8-byte loads.
bool na_aligned8(const void *p) { return ((uintptr_t)p & 7) == 0; }

bool na_is_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int pty_gradient_noalloc(int32_t H, int32_t W, int32_t P, const float *probe, int32_t K,
                                    const int32_t *pos, const float *data, double eps, const float *psi,
                                    float *grad, double *F, void *stream)
{
    if (P != 64 && P != 128) return PTY_ERR_ARG;
    if (K < 1 || K > kNaMaxK || (long long)K * P * P > kNaMaxPixels) return PTY_ERR_ARG;
    if (H < P || W < P || (long long)H * W > (1LL << 31) || !(eps >= 0.0 && std::isfinite(eps))) return PTY_ERR_ARG;
    if (!probe || !pos || !data || !psi || !grad) return PTY_ERR_ARG;
    if (!na_is_device(probe) || !na_is_device(pos) || !na_is_device(data) || !na_is_device(psi) ||
        !na_is_device(grad) || (F && !na_is_device(F)))
        return PTY_ERR_ARG;
    if (!na_aligned8(probe) || !na_aligned8(pos) || !na_aligned8(psi) || !na_aligned8(grad) ||
        (F && !na_aligned8(F)))
        return PTY_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int cur = 0, sdev = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return PTY_ERR_CUDA;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
        cudaGetLastError();
        return PTY_ERR_ARG;
    }
    if (sdev != cur) return PTY_ERR_ARG;
    void *base = nullptr;
    if (na_base(&base) != cudaSuccess) return PTY_ERR_CUDA;
    NaArgs a;
    a.base = (unsigned char *)base;
    a.H = H;
    a.W = W;
    a.P = P;
    a.K = K;
    a.probe = (const float2 *)probe;
    a.pos = (const int2 *)pos;
    a.data = data;
    a.eps = (float)eps;
    a.psi = (const float2 *)psi;
    a.grad = (float2 *)grad;
    a.F = F;
    k_na_prep<<<1, 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = P == 64 ? na_launch<64, 256>(a, s) : na_launch<128, 512>(a, s);
    int flag = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&flag, a.base + kNaOffFlag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return PTY_ERR_CUDA;
    return flag ? PTY_ERR_BOUNDS : PTY_OK;
}

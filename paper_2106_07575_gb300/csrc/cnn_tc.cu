// cnn_tc.cu -- the hidden 3x3 convolutions of the learned initial guess (kC -> kC channels) as
// implicit GEMMs on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One tile = 128 consecutive pixels of one output row (P = 128: a row, P = 256: half a row)
// and all kC output channels:
//   D[px][co] = sum over taps (dy, dx) and input channels ci of A_tap[px][ci] W[co][ci][tap],
// a GEMM with M = 128, N = kC, K = 9 kC.  The three input rows y - 1, y, y + 1 of the tile's
// pixels and a one-pixel halo are staged once per tile, channels in groups of 8: a group of
// 8 consecutive pixels is one canonical K-major core matrix (8 rows x 8 BF16 = 128 contiguous
// bytes), so the A operand of every tap is the same buffer at an offset of dx x 16 bytes.
// The FP32 activations are split into three BF16 parts (hi = rn(a), mid = rn(a - hi),
// lo = rn(a - hi - mid), 24 significant bits in all), the weights are BF16 already, and the
// products accumulate in FP32 in tensor memory: the FP32 convolution up to the order of its
// sums.  Forward: z = D + bias, a = GELU(z).  Backward-data (flipped transposed weights):
// out = D * GELU'(zprev).
//
// Two CTAs of 256 threads per SM each take a contiguous range of tiles in strip-major order,
// so that a tile usually stages only its one new input row into a three-row ring (the rows
// y - 1 and y are the previous tile's).  Thread 0 issues the tile's 54 MMAs (3 parts x 9 taps
// x 2 K-steps of 16 channels, M = 128, N = kC) and commits them to an mbarrier; the eight
// warps read the accumulator back (warp w: TMEM lanes 32 (w % 4) .. + 31 = 32 of the tile's
// pixels, channels 16 (w / 4) .. + 15).  The wait for the MMAs is bounded: after a timeout the
// CTA records it in *err, waits (bounded by the default limit) for its MMAs, frees its tensor
// memory and returns.
#include <cuda_bf16.h>

#include <atomic>

#include "cnn_internal.h"
#include "tc_ptx.cuh"

namespace pty {
namespace cnn {

namespace {
using namespace tcx;

constexpr int kTcNT = 256;                         // threads: two per tile pixel (channel halves)
constexpr int kNpx = 128;                          // pixels per tile (M)
constexpr int kSP = 136;                           // staged pixels per row and channel group (130 used)
constexpr int kGroups = kC / 8;                    // channel groups of 8
constexpr int kGroupBytes = kSP * 16;              // one row of one channel group
constexpr int kRowBytes = kGroups * kGroupBytes;   // one staged row, all channels
constexpr int kPartBytes = 3 * kRowBytes;          // one BF16 part of the three rows
constexpr int kABytes = 3 * kPartBytes;            // hi, mid, lo
constexpr int kBBytes = 9 * kGroups * kC * 16;     // weights [tap][group][co][8 ci]
constexpr size_t kTcSmem = (size_t)kABytes + kBBytes + 64;
static_assert(kGroupBytes % 16 == 0 && kPartBytes % 128 == 0 && kABytes % 128 == 0, "layout");

constexpr float kInvSqrt2PiTc = 0.398942280401432678f;
__device__ __forceinline__ float gelu_tc(float z) { return z * normcdff(z); }
__device__ __forceinline__ float gelu_grad_tc(float z)
{
    return normcdff(z) + z * kInvSqrt2PiTc * expf(-0.5f * z * z);
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = kC.
__host__ __device__ constexpr uint32_t conv_idesc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kC >> 3) << 17) | ((uint32_t)(kNpx >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// Stage input row yy (zero outside the image) of image b, pixels x0 - 1 .. x0 + 128, into row
// slot `slot` of the three BF16 parts: thread t takes pixel t % 128 and channel half t / 128;
// threads with t % 128 < 2 also one halo pixel.
template <int P>
__device__ __forceinline__ void stage_row(uint8_t *As, const float *__restrict__ in, int b, int yy, int x0, int slot)
{
    const int px = threadIdx.x % kNpx, half = threadIdx.x / kNpx;
    const bool row_in = yy >= 0 && yy < P;
#pragma unroll 1
    for (int h = 0; h < (px < 2 ? 2 : 1); h++) {
        const int p = h == 0 ? px + 1 : (px == 0 ? 0 : kNpx + 1);  // staged index: pixel x0 + p - 1
        const int x = x0 + p - 1;
        const bool in_img = row_in && x >= 0 && x < P;
        const float *src = in + (((size_t)b * kC + 16 * half) * P + (in_img ? yy : 0)) * P + (in_img ? x : 0);
        float v[16];
#pragma unroll
        for (int ci = 0; ci < 16; ci++) v[ci] = in_img ? __ldg(src + (size_t)ci * P * P) : 0.0f;
#pragma unroll
        for (int gg = 0; gg < 2; gg++) {
            const int g = 2 * half + gg;
            uint16_t hb[8], mb[8], lb[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const float a = v[8 * gg + j];
                hb[j] = to_half_bits<true>(a);
                const float r1 = a - from_half_bits<true>(hb[j]);
                mb[j] = to_half_bits<true>(r1);
                lb[j] = to_half_bits<true>(r1 - from_half_bits<true>(mb[j]));
            }
            const size_t off = (size_t)slot * kRowBytes + (size_t)g * kGroupBytes + (size_t)p * 16;
            *(uint4 *)(As + off) =
                make_uint4(pack2(hb[0], hb[1]), pack2(hb[2], hb[3]), pack2(hb[4], hb[5]), pack2(hb[6], hb[7]));
            *(uint4 *)(As + kPartBytes + off) =
                make_uint4(pack2(mb[0], mb[1]), pack2(mb[2], mb[3]), pack2(mb[4], mb[5]), pack2(mb[6], mb[7]));
            *(uint4 *)(As + 2 * kPartBytes + off) =
                make_uint4(pack2(lb[0], lb[1]), pack2(lb[2], lb[3]), pack2(lb[4], lb[5]), pack2(lb[6], lb[7]));
        }
    }
}

// Row slot of input row yy (yy >= -1) in the three-row ring.
__device__ __forceinline__ int ring_slot(int yy) { return (yy + 3) % 3; }

template <int P, bool BWD>
__global__ void __launch_bounds__(kTcNT, 2)
    k_conv_tc(const float *__restrict__ in, const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias,
              const float *__restrict__ zprev, float *__restrict__ zout, float *__restrict__ aout, int B,
              int *__restrict__ err, long long spin_limit)
{
    static_assert(P % kNpx == 0, "tiles of 128 pixels within a row");
    constexpr int TPR = P / kNpx;  // tiles per row
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *As = sm, *Bs = sm + kABytes;
    uint64_t *done = (uint64_t *)(sm + kABytes + kBBytes);
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    // tiles in strip-major order (image b, strip of 128 columns, row y fastest); CTA c takes
    // the contiguous range [c chunk, (c + 1) chunk), so consecutive tiles of a CTA are
    // consecutive rows of one strip and share two of their three input rows
    const int ntiles = B * TPR * P;
    const int chunk = (ntiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * chunk, t1 = min(ntiles, t0 + chunk);

    if (tid == 0) {
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, 32);
    // weights, once per CTA: element (co, ci, tap) at [(tap * kGroups + ci / 8) * kC + co][ci % 8]
    for (int e = tid; e < kC * kC * 9; e += kTcNT) {
        const int co = e / (kC * 9), rem = e % (kC * 9), ci = rem / 9, tap = rem % 9;
        *(__nv_bfloat16 *)(Bs + ((tap * kGroups + ci / 8) * kC + co) * 16 + (ci % 8) * 2) = w[e];
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = conv_idesc();

    int it = 0, prev_strip = -1, prev_y = -2;
    for (int tile = t0; tile < t1; tile++, it++) {
        const int strip = tile / P, y = tile % P;  // strip = b * TPR + column strip
        const int b = strip / TPR, x0 = (strip % TPR) * kNpx;
        // ---- input rows: only the new one when the previous tile was the row above
        if (strip == prev_strip && y == prev_y + 1) {
            stage_row<P>(As, in, b, y + 1, x0, ring_slot(y + 1));
        } else {
#pragma unroll 1
            for (int dy = 0; dy < 3; dy++) stage_row<P>(As, in, b, y - 1 + dy, x0, ring_slot(y - 1 + dy));
        }
        prev_strip = strip;
        prev_y = y;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        // ---- the tile's MMAs
        if (tid == 0) {
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
            int n = 0;
            // smallest part first: the lo and mid products are summed among themselves before
            // they meet the large hi products in the FP32 accumulator
#pragma unroll 1
            for (int part = 2; part >= 0; part--)
#pragma unroll 1
                for (int tap = 0; tap < 9; tap++)
#pragma unroll
                    for (int kk = 0; kk < kGroups / 2; kk++) {
                        const int dy = tap / 3, dx = tap % 3;
                        const uint64_t ad =
                            umma_desc(a0 + (uint32_t)(part * kPartBytes + ring_slot(y - 1 + dy) * kRowBytes +
                                                      2 * kk * kGroupBytes + dx * 16),
                                      kGroupBytes, 128);
                        const uint64_t bd = umma_desc(b0 + (uint32_t)((tap * kGroups + 2 * kk) * kC * 16), kC * 16, 128);
                        umma_f16(tmem, ad, bd, idesc, n > 0 ? 1u : 0u);
                        n++;
                    }
            umma_commit(done);  // arrives once every MMA of the tile has completed
        }
        // ---- epilogue: warp w reads lanes 32 (w % 4) .. + 31 (pixels), channels 16 (w / 4) .. + 15
        bool ok = mbar_wait(done, (uint32_t)(it & 1), spin_limit);
        ok = __syncthreads_and(ok) != 0;
        if (!ok) {
            if (tid == 0) atomicOr(err, 1);
            mbar_wait(done, (uint32_t)(it & 1));  // the MMAs finish before the TMEM is freed
            break;
        }
        tmem_fence_after_sync();
        const int q = warp & 3, ch = warp >> 2;
        float acc[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * ch), acc);
        const int x = x0 + 32 * q + (tid & 31);
        const size_t o = (((size_t)b * kC + 16 * ch) * P + y) * P + x;
#pragma unroll
        for (int c = 0; c < 16; c++) {
            const size_t oc = o + (size_t)c * P * P;
            if constexpr (BWD) {
                zout[oc] = acc[c] * gelu_grad_tc(__ldg(zprev + oc));
            } else {
                const float z = acc[c] + __ldg(bias + 16 * ch + c);
                zout[oc] = z;
                aout[oc] = gelu_tc(z);
            }
        }
        tmem_fence_before_sync();
        __syncthreads();  // TMEM read and staged rows free for the next tile
    }
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

template <int P, bool BWD>
cudaError_t run_conv_tc(int B, const float *in, const __nv_bfloat16 *w, const float *bias, const float *zprev,
                        float *z, float *a, int *err, cudaStream_t s)
{
    auto k = k_conv_tc<P, BWD>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int ntiles = B * P * (P / kNpx);
    const int nb = ntiles < 2 * nsm ? ntiles : 2 * nsm;
    k<<<nb, kTcNT, kTcSmem, s>>>(in, w, bias, zprev, z, a, B, err, tc_wait_limit());
    return cudaGetLastError();
}

}  // namespace

bool conv_tc_supported(int P, int cin) { return cin == kC && (P == 128 || P == 256); }

namespace {
std::atomic<bool> g_conv_tc{true};
}
void set_conv_tc(bool on) { g_conv_tc.store(on); }
bool conv_tc_on() { return g_conv_tc.load(); }

cudaError_t launch_conv_tc(int P, int B, bool bwd, const float *in, const __nv_bfloat16 *w, const float *bias,
                           const float *zprev, float *z, float *a, int *err, cudaStream_t s)
{
    if (!err || B < 1) return cudaErrorInvalidValue;
    if (P == 128) return bwd ? run_conv_tc<128, true>(B, in, w, bias, zprev, z, a, err, s)
                             : run_conv_tc<128, false>(B, in, w, bias, zprev, z, a, err, s);
    if (P == 256) return bwd ? run_conv_tc<256, true>(B, in, w, bias, zprev, z, a, err, s)
                             : run_conv_tc<256, false>(B, in, w, bias, zprev, z, a, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace cnn
}  // namespace pty

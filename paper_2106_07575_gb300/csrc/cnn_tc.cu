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

#include <algorithm>
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
constexpr size_t kTcSmem = (size_t)kABytes + kBBytes + 64 + 256;  // + the halo copies of the next row
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

// Four bytes global -> shared without a register round trip; src_ok = false writes zero.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool src_ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_ok ? 4 : 0)
                 : "memory");
}

// The 16 channels of channel half `half` at staged pixel p (pixel x0 + p - 1) split into the
// three BF16 parts of row slot `slot`.
__device__ __forceinline__ void split_px(uint8_t *As, int slot, int p, int half, const float (&v)[16])
{
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

// The 16 channels of half `half` of input row yy (zero outside the image) at pixel x.
template <int P>
__device__ __forceinline__ void load_px(const float *__restrict__ in, int b, int yy, int x, int half, float (&v)[16])
{
    const bool in_img = yy >= 0 && yy < P && x >= 0 && x < P;
    const float *src = in + (((size_t)b * kC + 16 * half) * P + (in_img ? yy : 0)) * P + (in_img ? x : 0);
#pragma unroll
    for (int ci = 0; ci < 16; ci++) v[ci] = in_img ? __ldg(src + (size_t)ci * P * P) : 0.0f;
}

// Stage input row yy (zero outside the image) of image b, pixels x0 - 1 .. x0 + 128, into row
// slot `slot` of the three BF16 parts: thread t takes pixel t % 128 and channel half t / 128;
// threads with t % 128 < 2 also one halo pixel.
template <int P>
__device__ __forceinline__ void stage_row(uint8_t *As, const float *__restrict__ in, int b, int yy, int x0, int slot)
{
    const int px = threadIdx.x % kNpx, half = threadIdx.x / kNpx;
#pragma unroll 1
    for (int h = 0; h < (px < 2 ? 2 : 1); h++) {
        const int p = h == 0 ? px + 1 : (px == 0 ? 0 : kNpx + 1);  // staged index: pixel x0 + p - 1
        float v[16];
        load_px<P>(in, b, yy, x0 + p - 1, half, v);
        split_px(As, slot, p, half, v);
    }
}

// The halo pixel (staged index 0 for t % 128 = 0, 129 for t % 128 = 1) of input row yy, 16
// channels of half t / 128, copied into H[(t % 128) * 32 + 16 half + ci] by cp.async (zeros
// outside the image).
template <int P>
__device__ __forceinline__ void halo_async(float *H, const float *__restrict__ in, int b, int yy, int x0)
{
    const int px = threadIdx.x % kNpx, half = threadIdx.x / kNpx;
    if (px >= 2) return;
    const int x = x0 + (px == 0 ? -1 : kNpx);
    const bool in_img = yy >= 0 && yy < P && x >= 0 && x < P;
    const float *src = in + (((size_t)b * kC + 16 * half) * P + (in_img ? yy : 0)) * P + (in_img ? x : 0);
#pragma unroll
    for (int ci = 0; ci < 16; ci++) cp_async4(H + px * 32 + 16 * half + ci, src + (size_t)ci * P * P, in_img);
    asm volatile("cp.async.commit_group;" ::: "memory");
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
    float *H = (float *)(sm + kABytes + kBBytes + 64);  // halo pixels of the next row [2][32]
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

    // The new input row of the next tile is loaded (this thread's pixel into registers, the
    // halo pixels by cp.async) right after this tile's MMAs are issued, so its latency is spent
    // behind the MMAs and the epilogue; it is split at the top of the next iteration.
    int it = 0, prev_strip = -1, prev_y = -2;
    bool have_pf = false;
    float vpf[16];
    for (int tile = t0; tile < t1; tile++, it++) {
        const int strip = tile / P, y = tile % P;  // strip = b * TPR + column strip
        const int b = strip / TPR, x0 = (strip % TPR) * kNpx;
        // ---- input rows: only the new one when the previous tile was the row above
        if (strip == prev_strip && y == prev_y + 1) {
            if (have_pf) {
                const int px = tid % kNpx, half = tid / kNpx;
                split_px(As, ring_slot(y + 1), px + 1, half, vpf);
                if (px < 2) {
                    asm volatile("cp.async.wait_all;" ::: "memory");  // this thread's halo copies
                    float hv[16];
#pragma unroll
                    for (int ci = 0; ci < 16; ci++) hv[ci] = H[px * 32 + 16 * half + ci];
                    split_px(As, ring_slot(y + 1), px == 0 ? 0 : kNpx + 1, half, hv);
                }
            } else {
                stage_row<P>(As, in, b, y + 1, x0, ring_slot(y + 1));
            }
        } else {
#pragma unroll 1
            for (int dy = 0; dy < 3; dy++) stage_row<P>(As, in, b, y - 1 + dy, x0, ring_slot(y - 1 + dy));
        }
        prev_strip = strip;
        prev_y = y;
        have_pf = false;
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
        if (tile + 1 < t1 && (tile + 1) % P != 0) {  // the next tile continues the strip: row y + 2
            load_px<P>(in, b, y + 2, x0 + tid % kNpx, tid / kNpx, vpf);
            halo_async<P>(H, in, b, y + 2, x0);
            have_pf = true;
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
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the CTA
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


namespace {

// ---------------------------------------------------------------------------------------
// Weight gradient of a hidden layer on the tensor cores:
//   dW[co][ci][dy][dx] = sum over pixels of dz[co][y][x] a[ci][y + dy - 1][x + dx - 1]
//                      = sum over (y, x') of a[ci][y + dy - 1][x'] dz[co][y][x' - dx + 1],
//   db[co] = sum over pixels of dz[co][y][x],
// written as per-CTA partials that launch_wgrad's fixed-order reduction adds (the layout of
// the CUDA-core kernel).  The work is B * (P / 32) * P units (image, 32-pixel column chunk,
// row) in that order, cut into wgrad_tc_blocks(P, B) contiguous ranges, one per CTA.  For each
// unit (chunk x', row y) the GEMM is D[m][n] += A[m][x'] Z[n][x'] with m = (dy, ci) (96 rows;
// M = 128, rows 96..127 read scratch and are not used), n = (dx, co) (N = 96) and K = the
// chunk's 32 pixels.  Both operands are split into three BF16 parts and the six products
// above 2^-24 are accumulated, smallest first: FP32-level products, FP32 sums.
//
// Each input row is split once: its 32 channels x 32 pixels go to ring slot (yy + 3) % 3 of
// the A region and, for slots 0 and 1, to the mirror slots 3 and 4, so the three rows of any
// unit (y - 1, y, y + 1) are the consecutive slots from the one of y - 1 and one MMA per
// K-step and product covers all three dy.  Each dz value is split once: a thread splits ten
// values (8 pixels and their halo) and writes the three shifted copies that carry dx (a
// canonical K-major tile cannot start one element into a core matrix).  Raw values come
// straight from global memory into registers, one unit ahead.  db is summed on the CUDA
// cores from the unshifted dz values.
constexpr int kWgTcRB = 16;                  // rows per CTA of the CUDA-core kernel (its partial count)
constexpr int kWgKC = 32;                    // pixels per unit (K)
constexpr int kWgCore = 128;                 // one core matrix (8 rows x 16 bytes)
constexpr int kWgGBytes = (kWgKC / 8) * kWgCore;   // one M- or N-group of 8 rows: 4 K-groups
constexpr int kWgSlotBytes = (kC / 8) * kWgGBytes; // one input row: 4 M-groups (32 channels)
constexpr int kWgSlots = 6;                        // ring 0..2, mirrors 3, 4, scratch 5
constexpr int kWgAPart = kWgSlots * kWgSlotBytes;  // one BF16 part of A (12 KB)
constexpr int kWgNG = 12;                          // Z N-groups of 8 rows: 3 dx x 4 co groups
constexpr int kWgBPart = kWgNG * kWgGBytes;        // one BF16 part of Z (6 KB)
constexpr int kWgN = 3 * kC;                       // N of the MMAs
constexpr size_t kWgSmem = 3 * (size_t)kWgAPart + 3 * (size_t)kWgBPart + 64;
constexpr int kWgPerSM = 4;                        // resident CTAs per SM (shared memory, TMEM, threads)
constexpr int kWgGrid = kWgPerSM * 152;            // CTAs of one wave on 152 SMs
static_assert(kTcNT == 256, "thread roles: 128 activation-row threads, 128 dz-row threads");

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = 96.
__host__ __device__ constexpr uint32_t wgrad_idesc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kWgN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void split3(float a, uint16_t &h, uint16_t &m, uint16_t &l)
{
    h = to_half_bits<true>(a);
    const float r1 = a - from_half_bits<true>(h);
    m = to_half_bits<true>(r1);
    l = to_half_bits<true>(r1 - from_half_bits<true>(m));
}

// Eight values v[o .. o + 7] of split parts h, m, l as three 16-byte BF16 rows at dst, dst +
// stride, dst + 2 stride.
template <int N>
__device__ __forceinline__ void store_parts8(uint8_t *dst, size_t stride, const uint16_t (&h)[N],
                                             const uint16_t (&m)[N], const uint16_t (&l)[N], int o)
{
    *(uint4 *)dst = make_uint4(pack2(h[o], h[o + 1]), pack2(h[o + 2], h[o + 3]), pack2(h[o + 4], h[o + 5]),
                               pack2(h[o + 6], h[o + 7]));
    *(uint4 *)(dst + stride) = make_uint4(pack2(m[o], m[o + 1]), pack2(m[o + 2], m[o + 3]),
                                          pack2(m[o + 4], m[o + 5]), pack2(m[o + 6], m[o + 7]));
    *(uint4 *)(dst + 2 * stride) = make_uint4(pack2(l[o], l[o + 1]), pack2(l[o + 2], l[o + 3]),
                                              pack2(l[o + 4], l[o + 5]), pack2(l[o + 6], l[o + 7]));
}

// Activation-row thread t < 128: channel ci = t / 4, pixels x0 + 8 (t % 4) .. + 7 of row yy
// (zeros outside the image), two aligned 16-byte loads.
template <int P>
__device__ __forceinline__ void load_arow(const float *__restrict__ a, int b, int yy, int x0, int t, float (&v)[8])
{
    if (yy < 0 || yy >= P) {
#pragma unroll
        for (int j = 0; j < 8; j++) v[j] = 0.f;
        return;
    }
    const float4 *src = reinterpret_cast<const float4 *>(a + (((size_t)b * kC + t / 4) * P + yy) * P + x0 + 8 * (t % 4));
    const float4 p0 = __ldg(src), p1 = __ldg(src + 1);
    v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w;
    v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
}

// dz-row thread t' = t - 128: channel co = t' / 4, pixels x0 + 8 (t' % 4) - 1 .. + 8 of row y
// (zeros outside the image): the 8 aligned values and the two halo values.
template <int P>
__device__ __forceinline__ void load_zrow(const float *__restrict__ dz, int b, int y, int x0, int tz, float (&v)[10])
{
    const int xs = x0 + 8 * (tz % 4);
    const float *row = dz + (((size_t)b * kC + tz / 4) * P + y) * P;
    const float4 *src = reinterpret_cast<const float4 *>(row + xs);
    const float4 p0 = __ldg(src), p1 = __ldg(src + 1);
    v[0] = xs > 0 ? __ldg(row + xs - 1) : 0.f;
    v[1] = p0.x; v[2] = p0.y; v[3] = p0.z; v[4] = p0.w;
    v[5] = p1.x; v[6] = p1.y; v[7] = p1.z; v[8] = p1.w;
    v[9] = xs + 8 < P ? __ldg(row + xs + 8) : 0.f;
}

// The activation row in v (thread t) split into ring slot (yy + 3) % 3 and its mirror.
__device__ __forceinline__ void store_arow(uint8_t *As, int yy, int t, const float (&v)[8])
{
    uint16_t h[8], m[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; j++) split3(v[j], h[j], m[j], l[j]);
    const int slot = (yy + 3) % 3, ci = t / 4, kg = t % 4;
    const size_t off = (size_t)(ci / 8) * kWgGBytes + kg * kWgCore + (ci % 8) * 16;
    store_parts8<8>(As + (size_t)slot * kWgSlotBytes + off, kWgAPart, h, m, l, 0);
    if (slot < 2) store_parts8<8>(As + (size_t)(slot + 3) * kWgSlotBytes + off, kWgAPart, h, m, l, 0);
}

// The dz row in v (thread t') split once; copy dx (pixels x' - dx + 1) is v[2 - dx .. 9 - dx]
// -> row co % 8 of core matrix (N-group dx * 4 + co / 8, K-group t' % 4).
__device__ __forceinline__ void store_zrow(uint8_t *Zs, int tz, const float (&v)[10])
{
    uint16_t h[10], m[10], l[10];
#pragma unroll
    for (int j = 0; j < 10; j++) split3(v[j], h[j], m[j], l[j]);
    const int co = tz / 4, kg = tz % 4;
#pragma unroll
    for (int dx = 0; dx < 3; dx++)
        store_parts8<10>(Zs + (size_t)(dx * 4 + co / 8) * kWgGBytes + kg * kWgCore + (co % 8) * 16, kWgBPart, h, m, l,
                         2 - dx);
}

template <int P>
__global__ void __launch_bounds__(kTcNT, kWgPerSM)
    k_wgrad_tc(const float *__restrict__ a, const float *__restrict__ dz, float *__restrict__ part, int *__restrict__ err,
               long long spin_limit, int nunits)
{
    static_assert(P % kWgKC == 0, "chunks");
    constexpr int NPL = kC * kC * 9 + kC;
    constexpr int NC = P / kWgKC;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *As = sm, *Zs = sm + 3 * (size_t)kWgAPart;
    uint64_t *done = (uint64_t *)(Zs + 3 * (size_t)kWgBPart);
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool arow = tid < 128;  // threads 0..127: activation rows; 128..255: dz rows
    const int tz = tid - 128;
    // this CTA's units [u0, u1); the host keeps every range non-empty
    const int u0 = (int)((long long)blockIdx.x * nunits / gridDim.x);
    const int u1 = (int)((long long)(blockIdx.x + 1) * nunits / gridDim.x);

    if (tid == 0) {
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, 128);
    // finite values in every slot: rows 96..127 of an MMA read the slot after a unit's three
    for (int e = tid; e < 3 * kWgAPart / 16; e += kTcNT) reinterpret_cast<uint4 *>(As)[e] = make_uint4(0, 0, 0, 0);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = wgrad_idesc();

    auto geo = [&](int u, int &b, int &x0, int &y) {
        b = u / (NC * P);
        x0 = ((u / P) % NC) * kWgKC;
        y = u % P;
    };
    bool started = false;
    // thread 0: the unit's 12 MMAs, (A part, Z part) smallest product first
    auto issue = [&](int u) {
        if (tid != 0) return;
        int b, x0, y;
        geo(u, b, x0, y);
        const uint32_t a0 = smem_u32(As) + (uint32_t)(((y + 2) % 3) * kWgSlotBytes);  // slot of row y - 1
        const uint32_t z0 = smem_u32(Zs);
        const int pa[6] = {2, 1, 0, 1, 0, 0}, pz[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll 1
        for (int ks = 0; ks < kWgKC / 16; ks++)
#pragma unroll
            for (int q = 0; q < 6; q++) {
                const uint64_t ad = umma_desc(a0 + (uint32_t)(pa[q] * kWgAPart + 2 * ks * kWgCore), kWgCore, kWgGBytes);
                const uint64_t zd = umma_desc(z0 + (uint32_t)(pz[q] * kWgBPart + 2 * ks * kWgCore), kWgCore, kWgGBytes);
                umma_f16(tmem, ad, zd, idesc, started ? 1u : 0u);
                started = true;
            }
        umma_commit(done);
    };
    float va[8], vz[10];  // raw values of the next unit
    float dbacc = 0.f;
    // a unit's operands from the raw registers: the new activation row (all three when the
    // unit starts a column) and the dz row
    auto stage = [&](int u, bool fresh) {
        int b, x0, y;
        geo(u, b, x0, y);
        if (arow) {
            if (fresh) {
#pragma unroll 1
                for (int dy = 0; dy < 3; dy++) {
                    load_arow<P>(a, b, y - 1 + dy, x0, tid, va);
                    store_arow(As, y - 1 + dy, tid, va);
                }
            } else {
                store_arow(As, y + 1, tid, va);
            }
        } else {
            store_zrow(Zs, tz, vz);
#pragma unroll
            for (int j = 1; j <= 8; j++) dbacc += vz[j];
        }
    };
    auto prefetch = [&](int u) {
        if (u >= u1) return;
        int b, x0, y;
        geo(u, b, x0, y);
        if (arow) {
            if (y != 0) load_arow<P>(a, b, y + 1, x0, tid, va);  // a unit continuing its column
        } else {
            load_zrow<P>(dz, b, y, x0, tz, vz);
        }
    };

    prefetch(u0);
    stage(u0, true);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    issue(u0);
    prefetch(u0 + 1);
    bool ok = true;
    int i = 0;
#pragma unroll 1
    for (int u = u0; u < u1; u++, i++) {
        ok = mbar_wait(done, (uint32_t)(i & 1), spin_limit);
        ok = __syncthreads_and(ok) != 0;  // the unit's MMAs have read both operands
        if (!ok) {
            if (tid == 0) atomicOr(err, 1);
            mbar_wait(done, (uint32_t)(i & 1));
            break;
        }
        if (u + 1 >= u1) break;
        // the next unit's new row goes to the slot of row y - 1 of this unit (read above)
        stage(u + 1, (u + 1) % P == 0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        issue(u + 1);
        prefetch(u + 2);  // the registers were stored above
    }
    if (ok) {
        // warps 0..3: TMEM lane quarter w = rows m = 32 w + lane (m = dy * 32 + ci), columns
        // 32 dx + co; warps 4..7: db from the dz threads' sums (4 threads per channel)
        tmem_fence_after_sync();
        float *pb = part + (size_t)blockIdx.x * NPL;
        if (warp < 4) {
            const int m = 32 * warp + lane;
#pragma unroll 1
            for (int dx = 0; dx < 3; dx++) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * dx), v);
                if (m < 96) {
                    const int dy = m / kC, ci = m % kC;
#pragma unroll
                    for (int co = 0; co < kC; co++) pb[((size_t)co * kC + ci) * 9 + dy * 3 + dx] = v[co];
                }
            }
        } else {
            dbacc += __shfl_xor_sync(0xffffffffu, dbacc, 1);
            dbacc += __shfl_xor_sync(0xffffffffu, dbacc, 2);
            if (tz % 4 == 0) pb[kC * kC * 9 + tz / 4] = dbacc;
        }
    }
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

}  // namespace

bool wgrad_tc_supported(int P, int cin, int cout) { return cin == kC && cout == kC && (P == 128 || P == 256); }

// One wave (at most kWgGrid CTAs), at least 32 units per CTA.
int wgrad_tc_blocks(int P, int B) { return std::max(1, std::min(kWgGrid, B * (P / kWgKC) * P / 32)); }

cudaError_t launch_wgrad_tc(int P, int B, const float *a, const float *dz, float *part, int *err, cudaStream_t s)
{
    if (!err || B < 1) return cudaErrorInvalidValue;
    const int nunits = B * (P / kWgKC) * P;
    auto run = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
        if (e != cudaSuccess) return e;
        kern<<<wgrad_tc_blocks(P, B), kTcNT, kWgSmem, s>>>(a, dz, part, err, tc_wait_limit(), nunits);
        return cudaGetLastError();
    };
    if (P == 128) return run(k_wgrad_tc<128>);
    if (P == 256) return run(k_wgrad_tc<256>);
    return cudaErrorInvalidValue;
}

}  // namespace cnn
}  // namespace pty

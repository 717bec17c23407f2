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


namespace {

// ---------------------------------------------------------------------------------------
// Weight gradient of a hidden layer on the tensor cores:
//   dW[co][ci][dy][dx] = sum over pixels of dz[co][y][x] a[ci][y + dy - 1][x + dx - 1]
//                      = sum over (y, x') of a[ci][y + dy - 1][x'] dz[co][y][x' - dx + 1],
//   db[co] = sum over pixels of dz[co][y][x],
// written as per-CTA partials that launch_wgrad's fixed-order reduction adds (the layout of
// the CUDA-core kernel).  The work is B * (P / 32) * P units (image, 32-pixel column chunk,
// row) in that order, cut into wgrad_tc_blocks(P, B) contiguous ranges, one per CTA: one
// wave of CTAs with equal shares.  For each unit (chunk x', row y) the GEMM is D[m][n] += A[m][x'] Z[n][x'] with m = (dy, ci)
// (96 rows, padded to M = 128), n = (dx, co) (N = 96) and K = the chunk's pixels: the row
// shift dy is a choice of staged row and the column shift dx is carried by three shifted
// copies of the dz row (a canonical K-major tile cannot start one element into a core
// matrix), so one MMA per K-step and product covers all nine taps.  Padding row 96 of A
// holds ones, so D[96][(dx = 1, co)] is db.  Activations and dz are both split into three
// BF16 parts and the six products above 2^-24 are accumulated, smallest first: FP32-level
// products, FP32 sums.
constexpr int kWgTcRB = 16;                  // rows per CTA of the CUDA-core kernel (its partial count)
constexpr int kWgKC = 32;                    // pixels per chunk (K)
constexpr int kWgMG = 16;                    // A M-groups of 8 rows: 12 used (3 dy x 4 ci groups), 4 padding
constexpr int kWgNG = 12;                    // Z N-groups of 8 rows: 3 dx x 4 co groups
constexpr int kWgCore = 128;                 // one core matrix (8 rows x 16 bytes)
constexpr int kWgGBytes = (kWgKC / 8) * kWgCore;   // one M- or N-group: 4 K-groups
constexpr int kWgAPart = kWgMG * kWgGBytes;        // one BF16 part of A
constexpr int kWgBPart = kWgNG * kWgGBytes;        // one BF16 part of Z
constexpr int kWgN = 3 * kC;                       // N of the MMAs
constexpr int kWgALd = kWgKC + 1;                  // raw activation row stride (floats, odd)
constexpr int kWgZLd = kWgKC + 3;                  // raw dz row stride: pixels x0 - 1 .. x0 + 32, odd
constexpr int kWgRing = 4;                        // raw activation rows held (a tile reads 3)
constexpr int kWgRawBytes = (kWgRing * kC * kWgALd + 2 * kC * kWgZLd) * 4;
constexpr int kWgGrid = 3 * 152;                   // CTAs of one wave: 3 resident per SM, 152 SMs
constexpr size_t kWgSmem = 3 * (size_t)kWgAPart + 3 * (size_t)kWgBPart + kWgRawBytes + 64;

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

// Eight consecutive values as three 16-byte BF16 rows (parts hi, mid, lo) at dst, dst + stride,
// dst + 2 stride.
__device__ __forceinline__ void store_split8(uint8_t *dst, size_t stride, const float (&v)[8])
{
    uint16_t h[8], m[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; j++) split3(v[j], h[j], m[j], l[j]);
    *(uint4 *)dst = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
    *(uint4 *)(dst + stride) = make_uint4(pack2(m[0], m[1]), pack2(m[2], m[3]), pack2(m[4], m[5]), pack2(m[6], m[7]));
    *(uint4 *)(dst + 2 * stride) =
        make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
}

// Four bytes global -> shared without a register round trip; src_ok = false writes zero.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool src_ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_ok ? 4 : 0)
                 : "memory");
}

template <int P>
__global__ void __launch_bounds__(kTcNT, 3)
    k_wgrad_tc(const float *__restrict__ a, const float *__restrict__ dz, float *__restrict__ part, int *__restrict__ err,
               long long spin_limit, int nunits)
{
    static_assert(P % kWgKC == 0, "chunks");
    constexpr int NPL = kC * kC * 9 + kC;
    constexpr int NC = P / kWgKC;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *As = sm, *Zs = sm + 3 * (size_t)kWgAPart;
    float *Ra = (float *)(Zs + 3 * (size_t)kWgBPart);  // raw activation rows [kWgRing][ci][kWgALd]
    float *Rz = Ra + kWgRing * kC * kWgALd;              // two raw dz rows [2][co][kWgZLd]
    uint64_t *done = (uint64_t *)((uint8_t *)Ra + kWgRawBytes);
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // this CTA's units [u0, u1); the host keeps every range non-empty
    const int u0 = (int)((long long)blockIdx.x * nunits / gridDim.x);
    const int u1 = (int)((long long)(blockIdx.x + 1) * nunits / gridDim.x);

    if (tid == 0) {
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, 128);
    // padding M-groups 12..15 of the three parts of A: zero, except row 96 (M-group 12, row 0
    // of each core matrix) of the high part: ones (BF16 1.0 = 0x3f80)
    for (int e = tid; e < 3 * 4 * (kWgGBytes / 16); e += kTcNT) {
        const int c16 = e % (kWgGBytes / 16), t = e / (kWgGBytes / 16);
        const int g = 12 + t % 4, pt = t / 4;
        const bool ones = pt == 0 && g == 12 && (c16 % 8) == 0;
        const uint32_t v = ones ? 0x3f803f80u : 0u;
        *(uint4 *)(As + (size_t)pt * kWgAPart + (size_t)g * kWgGBytes + c16 * 16) = make_uint4(v, v, v, v);
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = wgrad_idesc();

    // Unit u = (image b, chunk x0, row y).  The i-th unit of the CTA reads its rows y - 1 + r
    // (r = 0, 1, 2) from ring slots (i + r) % kWgRing and its dz row from buffer u & 1.  When
    // unit u + 1 continues the column (same chunk, row y + 1) it needs one new row, r = 2, in
    // slot (i + 3) % kWgRing, which unit u does not read: that copy and its dz row are issued
    // before unit u's split.  A unit that starts a column (y = 0) loads all three rows after
    // unit u's split has read the ring.
    auto load_rows = [&](int u, int r0, int nrow, int i) {
        const int b = u / (NC * P), x0 = ((u / P) % NC) * kWgKC, y = u % P;
        for (int e = tid; e < nrow * kC * kWgKC; e += kTcNT) {
            const int px = e % kWgKC, ci = (e / kWgKC) % kC, r = r0 + e / (kWgKC * kC);
            const int yy = y - 1 + r;
            const bool in = yy >= 0 && yy < P;
            cp_async4(Ra + (((i + r) % kWgRing) * kC + ci) * kWgALd + px,
                      in ? a + (((size_t)b * kC + ci) * P + yy) * P + x0 + px : a, in);
        }
        float *z = Rz + (u & 1) * kC * kWgZLd;
        for (int e = tid; e < kC * (kWgKC + 2); e += kTcNT) {
            const int q = e % (kWgKC + 2), co = e / (kWgKC + 2), x = x0 - 1 + q;
            const bool in = x >= 0 && x < P;
            cp_async4(z + co * kWgZLd + q, in ? dz + (((size_t)b * kC + co) * P + y) * P + x : dz, in);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    load_rows(u0, 0, 3, 0);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    bool started = false, ok = true;
#pragma unroll 1
    for (int u = u0; u < u1; u++) {
        const int i = u - u0;
        const bool next = u + 1 < u1, next_starts = next && (u + 1) % P == 0;
        if (next && !next_starts) load_rows(u + 1, 2, 1, i + 1);
        // ---- A: task (dy, ci, kg): pixels x0 + 8 kg .. + 7 of channel ci in row y + dy - 1
        // -> row ci % 8 of core matrix (M-group dy * 4 + ci / 8, K-group kg)
        for (int t = tid; t < 3 * kC * (kWgKC / 8); t += kTcNT) {
            const int ci = t % kC, kg = (t / kC) % (kWgKC / 8), dy = t / (kC * (kWgKC / 8));
            const float *r = Ra + (((i + dy) % kWgRing) * kC + ci) * kWgALd + 8 * kg;
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; j++) v[j] = r[j];
            store_split8(As + (size_t)(dy * 4 + ci / 8) * kWgGBytes + kg * kWgCore + (ci % 8) * 16, kWgAPart, v);
        }
        // ---- Z: task (dx, co, kg): dz[co] at pixels x' - dx + 1, x' = x0 + 8 kg .. + 7
        // -> row co % 8 of core matrix (N-group dx * 4 + co / 8, K-group kg)
        const float *zr = Rz + (u & 1) * kC * kWgZLd;
        for (int t = tid; t < 3 * kC * (kWgKC / 8); t += kTcNT) {
            const int co = t % kC, kg = (t / kC) % (kWgKC / 8), dx = t / (kC * (kWgKC / 8));
            const float *r = zr + co * kWgZLd + 8 * kg + 2 - dx;  // raw index of pixel x' - dx + 1
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; j++) v[j] = r[j];
            store_split8(Zs + (size_t)(dx * 4 + co / 8) * kWgGBytes + kg * kWgCore + (co % 8) * 16, kWgBPart, v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        if (tid == 0) {
            const uint32_t a0 = smem_u32(As), z0 = smem_u32(Zs);
            // (A part, Z part), smallest product first: lo*hi, mid*mid, hi*lo, mid*hi, hi*mid, hi*hi
            const int pa[6] = {2, 1, 0, 1, 0, 0}, pz[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll 1
            for (int ks = 0; ks < kWgKC / 16; ks++)
#pragma unroll
                for (int q = 0; q < 6; q++) {
                    const uint64_t ad =
                        umma_desc(a0 + (uint32_t)(pa[q] * kWgAPart + 2 * ks * kWgCore), kWgCore, kWgGBytes);
                    const uint64_t zd =
                        umma_desc(z0 + (uint32_t)(pz[q] * kWgBPart + 2 * ks * kWgCore), kWgCore, kWgGBytes);
                    umma_f16(tmem, ad, zd, idesc, started ? 1u : 0u);
                    started = true;
                }
            umma_commit(done);
        }
        if (next_starts) load_rows(u + 1, 0, 3, i + 1);  // the split above has read the ring
        ok = mbar_wait(done, (uint32_t)(i & 1), spin_limit);
        asm volatile("cp.async.wait_all;" ::: "memory");
        ok = __syncthreads_and(ok) != 0;  // the MMAs have read the tiles; the next rows have landed
        if (!ok) {
            if (tid == 0) atomicOr(err, 1);
            mbar_wait(done, (uint32_t)(i & 1));
            break;
        }
    }
    if (ok) {
        // warps 0..3: TMEM lane quarter w = rows m = 32 w + lane (m = dy * 32 + ci; m = 96: db),
        // columns 32 dx + co
        tmem_fence_after_sync();
        if (warp < 4) {
            const int m = 32 * warp + lane;
            float *pb = part + (size_t)blockIdx.x * NPL;
#pragma unroll 1
            for (int dx = 0; dx < 3; dx++) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * dx), v);
                if (m < 96) {
                    const int dy = m / kC, ci = m % kC;
#pragma unroll
                    for (int co = 0; co < kC; co++) pb[((size_t)co * kC + ci) * 9 + dy * 3 + dx] = v[co];
                } else if (m == 96 && dx == 1) {
#pragma unroll
                    for (int co = 0; co < kC; co++) pb[kC * kC * 9 + co] = v[co];
                }
            }
        }
    }
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

}  // namespace

bool wgrad_tc_supported(int P, int cin, int cout) { return cin == kC && cout == kC && (P == 128 || P == 256); }

// One wave (at most kWgGrid CTAs) and never more partials than the CUDA-core kernel writes
// (B * P / 16, which the caller's partial buffer holds); every CTA gets at least P / 2 units.
int wgrad_tc_blocks(int P, int B) { return std::min(kWgGrid, B * (P / kWgTcRB)); }

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

// tc_ws.cu -- the row DFT of the tensor-core form (split BF16) as a persistent,
// warp-specialised tcgen05 GEMM on sm_103a.
//
// The product is that of tc_dft.cu: for every row of a batch of P x P complex arrays, the
// row's DFT, stored transposed within its array, as [Ah | Al | Ah] x [Bh; Bh; Bl] with
// A = the row (re, im), B = the real block form of the DFT matrix, hi/lo BF16 halves and FP32
// accumulation.  Here the K dimension interleaves the real and imaginary parts of each
// input point (k = 2n + c), so a K-chunk of 64 is the contiguous 32-point segment of a row,
// and the three products are taken chunk by chunk.
//
// P = 256 (N = 2P = 512) takes two MMAs of N = 256 per K step into a single 512-column
// accumulator (no double buffering), with a 2-stage B ring of 64 KB images.
//
// One CTA per SM loops over tiles of 128 rows.  Roles (warps):
//   0       loader: bulk copies of the B chunk images (4-stage ring: every tile streams the
//           whole split DFT matrix from L2), each completing on an mbarrier with its bytes;
//   1       MMA: one thread issues tcgen05.mma (M = 128, N = 2P, K = 16) per A/B chunk pair
//           into one of two TMEM accumulator buffers and commits to the ring barriers;
//   2 - 9   split: the rows' 32-point segments straight from global memory (loads issued
//           before waiting for a free A slot) -> BF16 hi and lo in the canonical K-major
//           layout (A ring);
//   10 - 13 epilogue: tcgen05.ld of the finished buffer (warp w reads lane quarter w % 4),
//           transposed store, optional conjugate product; the buffer is then released.
// So the split of chunk c + 1, the MMAs of chunk c and the epilogue of the previous tile
// overlap.  Every pipeline wait is bounded (tc_wait_limit polls) and also gives up when
// another role has failed; after a failure the loader waits for the copies it issued and the
// MMA thread for its MMAs (bounded by the default limit, whatever the pipeline limit) before
// the TMEM is freed; err |= 1 records the failure.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "pty_internal.h"
#include "tc_ptx.cuh"

namespace pty {
namespace {
using namespace tcx;

constexpr int kWsRows = 128;  // M per tile
constexpr int kWsKC = 64;     // K per chunk: 32 complex points
#ifndef PTY_WS_SA
#define PTY_WS_SA 2
#endif
#ifndef PTY_WS_EPI
#define PTY_WS_EPI 4
#endif
constexpr int kWsSA = PTY_WS_SA, kWsSB = 4;
constexpr int kWsSplitWarps = 8;
constexpr int kWsEpiWarps = PTY_WS_EPI;  // 4 or 8: one or two per TMEM lane quarter
constexpr int kWsWarps = 2 + kWsSplitWarps + kWsEpiWarps;
constexpr int kWsThreads = 32 * kWsWarps;
constexpr int kWsSplitThreads = 32 * kWsSplitWarps;
constexpr int kAPart = kWsRows * kWsKC * 2;  // one BF16 part of an A chunk
constexpr int kAStage = 2 * kAPart;          // hi, lo
constexpr int kSBO = 128 * (kWsKC / 8);      // row-group stride of a chunk (A and B)

// P = 64, 128: one MMA per K step (N = 2P <= 256), two accumulator buffers in TMEM, a
// 4-stage B ring.  P = 256: N = 512 is taken as two MMAs of N = 256 per K step into one
// accumulator of 512 columns (all of TMEM), and the B ring has 2 stages of 64 KB.
template <int P>
struct WsGeo {
    static constexpr int N = 2 * P;                        // accumulator columns: re | im
    static constexpr int NM = N < 256 ? N : 256;           // N of one MMA instruction
    static constexpr int NSPLIT = N / NM;                  // MMAs per K step
    static constexpr int NBUF = 2 * N <= 512 ? 2 : 1;      // accumulator buffers
    static constexpr int SB = P >= 256 ? 2 : kWsSB;        // B ring stages
    static constexpr int NKC = 2 * P / kWsKC;
    static constexpr int BIMG = N * kWsKC * 2;
    static constexpr int TMEM_COLS = NBUF * N;
    static constexpr size_t OFF_A = 0;
    static constexpr size_t OFF_B = OFF_A + (size_t)kWsSA * kAStage;
    static constexpr size_t OFF_BAR = OFF_B + (size_t)SB * BIMG;
    static constexpr int NBAR = 2 * kWsSA + 2 * SB + 2 * NBUF + 1;
    static constexpr size_t SMEM = OFF_BAR + 8 * NBAR + 16;
    static_assert(OFF_A % 1024 == 0 && OFF_B % 1024 == 0, "ring alignment");
    static_assert(TMEM_COLS <= 512 && NM % 16 == 0 && SMEM <= 227 * 1024, "geometry");
};

template <int N>
__device__ __forceinline__ uint32_t idesc_bf16()
{
    // D = F32 (bit 4), A = B = BF16 (bits 7, 10), K-major, N >> 3 at bit 17, M >> 4 at bit 24
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kWsRows >> 4) << 24);
}

// Bounded wait that also gives up when another role has recorded a failure.
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, volatile int *fail, long long limit)
{
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < limit; it++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 1023) == 1023 && *fail) return false;
    }
    return false;
}

__device__ __forceinline__ void ws_fail(volatile int *fail, int *err)
{
    *fail = 1;
    atomicOr(err, 1);
}

template <int P>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_dft_rows_ws(const float2 *__restrict__ X, float2 *__restrict__ Y, const uint8_t *__restrict__ Bimg, int nrows,
                  const int *__restrict__ out_index, const float2 *__restrict__ conj_mul, int *__restrict__ err,
                  long long spin_limit)
{
    using G = WsGeo<P>;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *as = sm + G::OFF_A, *bs = sm + G::OFF_B;
    uint64_t *bar = (uint64_t *)(sm + G::OFF_BAR);
    uint64_t *afull = bar, *aempty = afull + kWsSA;
    uint64_t *bfull = aempty + kWsSA, *bempty = bfull + G::SB, *tfull = bempty + G::SB, *tempty = tfull + G::NBUF;
    uint64_t *mdone = tempty + G::NBUF;
    uint32_t *tmem_slot = (uint32_t *)(mdone + 1);
    __shared__ int fail_s;
    volatile int *fail = &fail_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (nrows + kWsRows - 1) / kWsRows;

    if (tid == 0) {
        fail_s = 0;
        for (int s = 0; s < kWsSA; s++) {
            mbar_init(afull + s, kWsSplitWarps);
            mbar_init(aempty + s, 1);
        }
        for (int s = 0; s < G::SB; s++) {
            mbar_init(bfull + s, 1);
            mbar_init(bempty + s, 1);
        }
        for (int b = 0; b < G::NBUF; b++) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, kWsEpiWarps);
        }
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)G::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------------- loader
        if (lane == 0) {
            int ub = 0;
            int lastb[G::SB];  // last use issued per stage (-1: none)
            for (int s = 0; s < G::SB; s++) lastb[s] = -1;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
                for (int kc = 0; kc < G::NKC && ok; kc++)
                    for (int part = 0; part < 2 && ok; part++) {
                        const int sb = ub % G::SB;
                        if (!(ok = ws_wait(bempty + sb, ((ub / G::SB) & 1) ^ 1, fail, spin_limit))) break;
                        mbar_expect_tx(bfull + sb, (uint32_t)G::BIMG);
                        bulk_g2s(bs + (size_t)sb * G::BIMG, Bimg + (size_t)(2 * kc + part) * G::BIMG, G::BIMG,
                                 bfull + sb);
                        lastb[sb] = ub++;
                    }
            if (!ok) {
                ws_fail(fail, err);
                // let every issued copy land before the CTA can exit (bounded)
                for (int s = 0; s < G::SB; s++)
                    if (lastb[s] >= 0) mbar_wait(bfull + s, (lastb[s] / G::SB) & 1);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16<G::NM>();
            int ua = 0, ub = 0, lt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, lt++) {
                const int tb = lt % G::NBUF;
                if (!(ok = ws_wait(tempty + tb, ((lt / G::NBUF) & 1) ^ 1, fail, spin_limit))) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(tb * G::N);
                for (int kc = 0; kc < G::NKC && ok; kc++) {
                    const int sa = ua % kWsSA;
                    if (!(ok = ws_wait(afull + sa, (ua / kWsSA) & 1, fail, spin_limit))) break;
                    const uint32_t ah = smem_u32(as + (size_t)sa * kAStage), al = ah + kAPart;
                    for (int part = 0; part < 2 && ok; part++) {
                        const int sb = ub % G::SB;
                        if (!(ok = ws_wait(bfull + sb, (ub / G::SB) & 1, fail, spin_limit))) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t b = smem_u32(bs + (size_t)sb * G::BIMG);
#pragma unroll
                        for (int k = 0; k < kWsKC / 16; k++)
#pragma unroll
                            for (int nh = 0; nh < G::NSPLIT; nh++) {
                                // rows [nh NM, nh NM + NM) of the B chunk: NM / 8 row groups further
                                const uint64_t bd = umma_desc(b + (uint32_t)(nh * (G::NM / 8) * kSBO) + 2 * k * 128,
                                                              128, kSBO);
                                const uint32_t dn = d + (uint32_t)(nh * G::NM);
                                // part 0 (Bh): Ah Bh + Al Bh; part 1 (Bl): Ah Bl
                                umma_f16(dn, umma_desc(ah + 2 * k * 128, 128, kSBO), bd, idesc,
                                         (kc > 0 || part > 0 || k > 0) ? 1u : 0u);
                                if (part == 0) umma_f16(dn, umma_desc(al + 2 * k * 128, 128, kSBO), bd, idesc, 1u);
                            }
                        umma_commit(bempty + sb);
                        ub++;
                    }
                    if (!ok) break;
                    umma_commit(aempty + sa);
                    ua++;
                }
                if (!ok) break;
                umma_commit(tfull + tb);
            }
            if (!ok) ws_fail(fail, err);
            umma_commit(mdone);  // arrives once every issued MMA has completed
            mbar_wait(mdone, 0);
        }
        __syncwarp();
    } else if (warp < 2 + kWsSplitWarps) {
        // ---------------------------------------------------------------- split
        constexpr int TPT = (kWsRows * 4) / kWsSplitThreads;  // tasks per thread per chunk
        const int ct = tid - 64;
        int ua = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int row0 = t * kWsRows;
            for (int kc = 0; kc < G::NKC && ok; kc++) {
                // the chunk's loads first (in flight while waiting for a free A slot)
                // task (row m, j): points 4j .. 4j + 3 (K group j) and 16 + 4j .. 16 + 4j + 3
                // (K group 4 + j), so that one store instruction of a warp covers the four
                // adjacent core matrices of a row group: 512 contiguous bytes, no bank conflict
                float v[TPT][16];  // re, im of the 4 + 4 points
#pragma unroll
                for (int q4 = 0; q4 < TPT; q4++) {
                    const int task = ct + kWsSplitThreads * q4;
                    const int m = (task >> 5) * 8 + (task & 7), j = (task >> 3) & 3;
                    if (row0 + m < nrows) {
                        const float4 *src = (const float4 *)(X + (size_t)(row0 + m) * P + 32 * kc + 4 * j);
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const float4 f = __ldg(src + (q < 2 ? q : 8 + (q - 2)));  // points 4j.. and 16 + 4j..
                            v[q4][4 * q] = f.x;
                            v[q4][4 * q + 1] = f.y;
                            v[q4][4 * q + 2] = f.z;
                            v[q4][4 * q + 3] = f.w;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; q++) v[q4][q] = 0.0f;
                    }
                }
                const int sa = ua % kWsSA;
                if (lane == 0) ok = ws_wait(aempty + sa, ((ua / kWsSA) & 1) ^ 1, fail, spin_limit);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
                uint8_t *ahi = as + (size_t)sa * kAStage, *alo = ahi + kAPart;
#pragma unroll
                for (int q4 = 0; q4 < TPT; q4++) {
                    const int task = ct + kWsSplitThreads * q4;
                    const int m = (task >> 5) * 8 + (task & 7), j = (task >> 3) & 3;
                    uint32_t hw[8], lw[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const float a0 = v[q4][2 * q], a1 = v[q4][2 * q + 1];
                        const uint16_t h0 = to_half_bits<true>(a0), h1 = to_half_bits<true>(a1);
                        const uint16_t l0 = to_half_bits<true>(a0 - from_half_bits<true>(h0));
                        const uint16_t l1 = to_half_bits<true>(a1 - from_half_bits<true>(h1));
                        hw[q] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                        lw[q] = (uint32_t)l0 | ((uint32_t)l1 << 16);
                    }
                    // K group j (K = 8j .. 8j + 7) and K group 4 + j of row m
                    const size_t o0 = (size_t)(m >> 3) * kSBO + j * 128 + (m & 7) * 16;
                    *(uint4 *)(ahi + o0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *(uint4 *)(ahi + o0 + 512) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
                    *(uint4 *)(alo + o0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    *(uint4 *)(alo + o0 + 512) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(afull + sa);
                ua++;
            }
        }
        if (!ok && lane == 0) ws_fail(fail, err);
    } else {
        // ---------------------------------------------------------------- epilogue
        // warp w: lane quarter w % 4, column half (w - first epilogue warp) / 4 when 8 warps
        const int q4 = warp & 3, half = (warp - (2 + kWsSplitWarps)) >> 2;
        constexpr int KSPAN = P / (kWsEpiWarps / 4);  // accumulator columns per warp (each of re, im)
        const int m = q4 * 32 + lane;
        int lt = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, lt++) {
            const int tb = lt % G::NBUF;
            if (lane == 0) ok = ws_wait(tfull + tb, (lt / G::NBUF) & 1, fail, spin_limit);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = t * kWsRows + m;
            const int b = row / P, y = row % P;
            const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(tb * G::N);
            float2 *dst = Y + (size_t)(row < nrows ? (out_index ? out_index[b] : b) : 0) * P * P + y;
#pragma unroll 1
            for (int k0 = half * KSPAN; k0 < (half + 1) * KSPAN; k0 += 32) {
                float re[32], im[32];
                tmem_ld32(tl + k0, re);
                tmem_ld32(tl + P + k0, im);
                if (row < nrows) {
                    if (conj_mul) {  // element (k, y) of the 2-D result times conj(conj_mul[k][y])
#pragma unroll
                        for (int q = 0; q < 32; q++) {
                            const float2 c = __ldg(conj_mul + (size_t)(k0 + q) * P + y);
                            dst[(size_t)(k0 + q) * P] =
                                make_float2(fmaf(c.x, re[q], c.y * im[q]), fmaf(c.x, im[q], -c.y * re[q]));
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; q++) dst[(size_t)(k0 + q) * P] = make_float2(re[q], im[q]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + tb);
        }
        if (!ok && lane == 0) ws_fail(fail, err);
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)G::TMEM_COLS));
}

// Host: B chunk images in the interleaved-K layout: chunk kc covers points n = 32 kc ..
// 32 kc + 31, K index 2 (n - 32 kc) + c (c = 0 real, 1 imaginary part of the input point);
// image (kc, 0) holds the BF16 high halves, (kc, 1) the low halves, each N x 64 in the
// canonical K-major shared-memory layout.
template <int P>
std::vector<uint8_t> build_ws_images(int sign)
{
    using G = WsGeo<P>;
    const int N = G::N;
    std::vector<uint8_t> img((size_t)G::NKC * 2 * G::BIMG);
    const double pi = 3.14159265358979323846;
    for (int kc = 0; kc < G::NKC; kc++)
        for (int n = 0; n < N; n++)
            for (int kl = 0; kl < kWsKC; kl++) {
                const int pt = 32 * kc + kl / 2, c = kl % 2, k = n % P;
                const double th = 2.0 * pi * (double)((long long)pt * k % P) / (double)P;
                const double cs = std::cos(th), sn = sign * std::sin(th);
                // input real part: (C | sS); input imaginary part: (-sS | C)
                const double v = (c == 0) ? ((n < P) ? cs : sn) : ((n < P) ? -sn : cs);
                const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
                const __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
                const size_t off = (size_t)(n >> 3) * kSBO + (kl >> 3) * 128 + (n & 7) * 16 + (kl & 7) * 2;
                const uint16_t hb = __bfloat16_as_ushort(h), lb = __bfloat16_as_ushort(l);
                uint8_t *hi = img.data() + (size_t)(2 * kc) * G::BIMG, *lo = hi + G::BIMG;
                hi[off] = (uint8_t)(hb & 0xff);
                hi[off + 1] = (uint8_t)(hb >> 8);
                lo[off] = (uint8_t)(lb & 0xff);
                lo[off + 1] = (uint8_t)(lb >> 8);
            }
    return img;
}

template <int P>
cudaError_t run_ws(const float2 *X, float2 *Y, const void *img, int nrows, const int *out_index,
                   const float2 *conj_mul, int *err, cudaStream_t s)
{
    using G = WsGeo<P>;
    auto k = k_dft_rows_ws<P>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int ntiles = (nrows + kWsRows - 1) / kWsRows;
    const int nb = ntiles < nsm ? ntiles : nsm;
    if (nb < 1) return cudaSuccess;
    k<<<nb, kWsThreads, G::SMEM, s>>>(X, Y, (const uint8_t *)img, nrows, out_index, conj_mul, err, tc_wait_limit());
    return cudaGetLastError();
}

}  // namespace

cudaError_t tc_ws_images(int P, int sign, std::vector<uint8_t> &out)
{
    if (P == 64) out = build_ws_images<64>(sign);
    else if (P == 128) out = build_ws_images<128>(sign);
    else if (P == 256) out = build_ws_images<256>(sign);
    else return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t tc_ws_rows(int P, const float2 *X, float2 *Y, const void *img, int nrows, const int *out_index,
                       const float2 *conj_mul, int *err, cudaStream_t s)
{
    if (P == 64) return run_ws<64>(X, Y, img, nrows, out_index, conj_mul, err, s);
    if (P == 128) return run_ws<128>(X, Y, img, nrows, out_index, conj_mul, err, s);
    if (P == 256) return run_ws<256>(X, Y, img, nrows, out_index, conj_mul, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace pty

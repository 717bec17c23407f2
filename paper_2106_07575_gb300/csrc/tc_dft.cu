// tc_dft.cu -- the DFT of Eq. 1 (and F^H of Eq. 3) as a tensor-core GEMM on sm_103a: the
// FP16 split form (per-tile scaling, one tile per CTA) and the dispatch; the BF16 split form
// runs the persistent warp-specialised kernel of tc_ws.cu.
//
// One application transforms every row of a batch of P x P complex arrays and stores the
// result transposed within each array, so two applications give the unnormalised 2-D DFT
// (the DFT matrix is symmetric: (X F)^T F = F X^T F = (F X F)^T).  Row m of the batch,
// [xr(0..P-1) | xi(0..P-1)], times the real block matrix
//     B = [[ C,  sS], [-sS,  C]],  C = cos(2 pi n k / P), S = sin(2 pi n k / P), s = sign,
// gives [yr | yi] of the row's DFT.  Both operands are split into a high and a low
// half-precision part (BF16 or FP16): A B ~ Ah Bh + Al Bh + Ah Bl, evaluated as ONE GEMM
// with K' = 3 * 2P, A' = [Ah | Al | Ah], B' = [Bh; Bh; Bl], accumulated in FP32 in TMEM.
//
// Per CTA (512 threads): 128 consecutive rows.  For FP16 the tile is first scaled by a power
// of two so that its largest magnitude is 2^14 at most (undone exactly on the results).  The
// threads split the FP32 rows into Ah and Al in shared memory (canonical K-major layout without swizzle: 8 x 16-byte core
// matrices, K-adjacent core matrices 128 bytes apart).  B' is stored in global memory as
// a sequence of exact shared-memory images of 64-column chunks (built on the host from
// FP64), streamed by cp.async.bulk through a 3-stage mbarrier pipeline.  One thread issues
// tcgen05.mma (M = 128, N = 2P, K = 16 per instruction); the accumulator is read back with
// tcgen05.ld and stored transposed.  Every mbarrier wait is bounded: on timeout the kernel
// records an error, waits (bounded) for its own operations, frees TMEM and returns.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <vector>

#include "pty_internal.h"
#include "tc_ptx.cuh"

namespace pty {
namespace {
using namespace tcx;

constexpr int kTcThreads = 512;  // 16 warps: loads in flight for the operand split; 4 per TMEM lane quarter
constexpr int kTcRows = 128;    // M per CTA
constexpr int kTcChunk = 64;    // K' elements per pipeline stage
constexpr int kTcStages = 3;

template <int P>
struct TcGeo {
    static constexpr int N = 2 * P;                      // accumulator columns
    static constexpr int KF = 2 * P;                     // K of one part
    static constexpr int NCHUNK = 3 * KF / kTcChunk;     // K' chunks
    static constexpr int A_BYTES = kTcRows * KF * 2;     // one half-precision part
    static constexpr int B_BYTES = N * kTcChunk * 2;     // one B chunk image
    static constexpr int SBO_A = 128 * (KF / 8);         // row-group stride of A
    static constexpr int SBO_B = 128 * (kTcChunk / 8);   // row-group stride of a B chunk
    static constexpr int TMEM_COLS = N < 32 ? 32 : N;
    static constexpr size_t SMEM = 2 * (size_t)A_BYTES + kTcStages * (size_t)B_BYTES + 256;
};

// kind::f16 instruction descriptor: D = F32, A = B = BF16 or F16, both K-major, M = 128.
template <int N, bool BF16>
__device__ __forceinline__ uint32_t umma_idesc()
{
    const uint32_t fmt = BF16 ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

// Y[b][k][y] = sum_n X[b][y][n] W^{n k}  (W = exp(sign 2 pi i / P)) for all rows (b, y).
template <int P, bool BF16>
__global__ void __launch_bounds__(kTcThreads, 1) k_dft_rows_tc(const float2 *__restrict__ X, float2 *__restrict__ Y,
                                                               const uint8_t *__restrict__ Bimg, int nrows,
                                                               const int *__restrict__ out_index,
                                                               const float2 *__restrict__ conj_mul,
                                                               int *__restrict__ err, long long spin_limit)
{
    using G = TcGeo<P>;
    extern __shared__ __align__(1024) uint8_t tsm[];
    uint8_t *A_hi = tsm, *A_lo = tsm + G::A_BYTES, *Bst = tsm + 2 * G::A_BYTES;
    uint64_t *bar = (uint64_t *)(Bst + kTcStages * G::B_BYTES);  // full[S], empty[S], done
    uint64_t *full = bar, *empty = bar + kTcStages, *done = bar + 2 * kTcStages;
    uint32_t *tmem_slot = (uint32_t *)(bar + 2 * kTcStages + 1);
    __shared__ int fail_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTcRows;

    if (tid == 0) {
        fail_s = 0;
        for (int s = 0; s < kTcStages; s++) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)G::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }

    // FP16 has a narrow range: scale the tile by a power of two so that its largest
    // magnitude is at most 2^14 (exact), and undo it on the FP32 results.
    float scale = 1.0f;
    if constexpr (!BF16) {
        __shared__ unsigned int amax_bits;
        if (tid == 0) amax_bits = 0u;
        __syncthreads();
        float mx = 0.0f;
        for (int t = tid; t < kTcRows * (P / 8); t += kTcThreads) {
            const int row = m0 + t / (P / 8), j = t % (P / 8);
            if (row < nrows) {
                const float4 *src = (const float4 *)(X + (size_t)row * P + 8 * j);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const float4 v = __ldg(src + q);
                    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
                }
            }
        }
        atomicMax(&amax_bits, __float_as_uint(mx));  // non-negative floats order as integers
        __syncthreads();
        const float amax = __uint_as_float(amax_bits);
        if (amax > 0.0f && isfinite(amax)) {
            int e;
            frexpf(amax, &e);  // amax < 2^e
            scale = ldexpf(1.0f, 14 - e);
        }
    }

    // A: split the FP32 rows into high and low halves, canonical K-major layout.
    // Task (row m, group j of 8 complex values) -> core-matrix rows of re and im.
#pragma unroll 4
    for (int t = tid; t < kTcRows * (P / 8); t += kTcThreads) {
        const int m = t / (P / 8), j = t % (P / 8);
        const int row = m0 + m;
        float re[8], im[8];
        if (row < nrows) {
            const float4 *src = (const float4 *)(X + (size_t)row * P + 8 * j);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float4 v = __ldg(src + q);
                re[2 * q] = v.x * scale;
                im[2 * q] = v.y * scale;
                re[2 * q + 1] = v.z * scale;
                im[2 * q + 1] = v.w * scale;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; q++) re[q] = im[q] = 0.0f;
        }
        uint16_t hr[8], lr[8], hi_[8], li[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            hr[q] = to_half_bits<BF16>(re[q]);
            lr[q] = to_half_bits<BF16>(re[q] - from_half_bits<BF16>(hr[q]));
            hi_[q] = to_half_bits<BF16>(im[q]);
            li[q] = to_half_bits<BF16>(im[q] - from_half_bits<BF16>(hi_[q]));
        }
        const int i = m >> 3, r = m & 7;
        // re at K group j, im at K group P/8 + j
        const int off_re = i * G::SBO_A + j * 128 + r * 16;
        const int off_im = i * G::SBO_A + (P / 8 + j) * 128 + r * 16;
        uint4 v;
        v = make_uint4(hr[0] | (hr[1] << 16), hr[2] | (hr[3] << 16), hr[4] | (hr[5] << 16), hr[6] | (hr[7] << 16));
        *(uint4 *)(A_hi + off_re) = v;
        v = make_uint4(lr[0] | (lr[1] << 16), lr[2] | (lr[3] << 16), lr[4] | (lr[5] << 16), lr[6] | (lr[7] << 16));
        *(uint4 *)(A_lo + off_re) = v;
        v = make_uint4(hi_[0] | (hi_[1] << 16), hi_[2] | (hi_[3] << 16), hi_[4] | (hi_[5] << 16),
                       hi_[6] | (hi_[7] << 16));
        *(uint4 *)(A_hi + off_im) = v;
        v = make_uint4(li[0] | (li[1] << 16), li[2] | (li[3] << 16), li[4] | (li[5] << 16), li[6] | (li[7] << 16));
        *(uint4 *)(A_lo + off_im) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async proxy
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        const uint32_t idesc = umma_idesc<G::N, BF16>();
        bool ok = true;
        int issued = 0, consumed = 0;  // chunks whose copies were issued / whose MMAs were issued
        for (int c = 0; c < kTcStages && c < G::NCHUNK; c++) {
            mbar_expect_tx(full + c, G::B_BYTES);
            bulk_g2s(Bst + c * G::B_BYTES, Bimg + (size_t)c * G::B_BYTES, G::B_BYTES, full + c);
            issued = c + 1;
        }
        for (int c = 0; c < G::NCHUNK && ok; c++) {
            const int s = c % kTcStages;
            if (!mbar_wait(full + s, (c / kTcStages) & 1, spin_limit)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int part = c / (G::KF / kTcChunk), kc = c % (G::KF / kTcChunk);
            const uint8_t *Abuf = (part == 1) ? A_lo : A_hi;
#pragma unroll
            for (int k = 0; k < kTcChunk / 16; k++) {
                const uint64_t ad = umma_desc(smem_u32(Abuf + (kc * (kTcChunk / 8) + 2 * k) * 128), 128, G::SBO_A);
                const uint64_t bd = umma_desc(smem_u32(Bst + s * G::B_BYTES + 2 * k * 128), 128, G::SBO_B);
                umma_f16(tmem, ad, bd, idesc, (c > 0 || k > 0) ? 1u : 0u);
            }
            umma_commit(empty + s);
            consumed = c + 1;
            // refill the stage of the previous chunk once its MMAs have finished reading it
            const int pc = c - 1;
            if (pc >= 0 && pc + kTcStages < G::NCHUNK) {
                const int ps = pc % kTcStages;
                if (!mbar_wait(empty + ps, (pc / kTcStages) & 1, spin_limit)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(full + ps, G::B_BYTES);
                bulk_g2s(Bst + ps * G::B_BYTES, Bimg + (size_t)(pc + kTcStages) * G::B_BYTES, G::B_BYTES, full + ps);
                issued = pc + kTcStages + 1;
            }
        }
        umma_commit(done);  // arrives once every issued MMA has completed
        if (!ok) {
            fail_s = 1;
            // every copy issued but not consumed lands before the CTA can exit
            for (int c = consumed; c < issued; c++) mbar_wait(full + c % kTcStages, (c / kTcStages) & 1);
        }
    }
    __syncthreads();
    const bool ok = mbar_wait(done, 0) && !fail_s;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (tid == 0) atomicOr(err, 1);
    } else {
        // epilogue: warp w reads TMEM lane quarter w % 4 (lane = row) and the column group
        // w / 4 of P/4 columns; columns [0, P) hold real parts, [P, 2P) imaginary parts
        constexpr int CW = P / (kTcThreads / 128);  // columns per warp: 32 (P = 128) or 16 (P = 64)
        const int q4 = warp & 3, k0 = (warp >> 2) * CW;
        const int m = q4 * 32 + lane, row = m0 + m;
        const int b = row / P, y = row % P;
        const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16);
        const float unscale = 1.0f / scale;  // exact: a power of two
        float re[CW], im[CW];
        if constexpr (CW == 32) {
            tmem_ld32(tl + k0, re);
            tmem_ld32(tl + P + k0, im);
        } else {
            tmem_ld16(tl + k0, re);
            tmem_ld16(tl + P + k0, im);
        }
#pragma unroll
        for (int q = 0; q < CW; q++) {
            re[q] *= unscale;
            im[q] *= unscale;
        }
        if (row < nrows) {
            float2 *dst = Y + (size_t)(out_index ? out_index[b] : b) * P * P + y;
            if (conj_mul) {  // element (k, y) of the 2-D result times conj(conj_mul[k][y])
#pragma unroll
                for (int q = 0; q < CW; q++) {
                    const float2 c = __ldg(conj_mul + (size_t)(k0 + q) * P + y);
                    dst[(size_t)(k0 + q) * P] = make_float2(fmaf(c.x, re[q], c.y * im[q]), fmaf(c.x, im[q], -c.y * re[q]));
                }
            } else {
#pragma unroll
                for (int q = 0; q < CW; q++) dst[(size_t)(k0 + q) * P] = make_float2(re[q], im[q]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)G::TMEM_COLS));
}

// Host: B' images (shared-memory layout of each 64-column K' chunk) from FP64 values.
template <int P, bool BF16>
std::vector<uint8_t> build_images(int sign)
{
    using G = TcGeo<P>;
    const int N = G::N, KF = G::KF;
    // full block matrix Bfull[kk][n] in FP64, split into high and low halves
    std::vector<uint16_t> bh((size_t)KF * N), bl((size_t)KF * N);
    const double pi = 3.14159265358979323846;
    for (int kk = 0; kk < KF; kk++)
        for (int n = 0; n < N; n++) {
            const int nn = kk % P, k = n % P;
            const double th = 2.0 * pi * (double)((long long)nn * k % P) / (double)P;
            const double c = std::cos(th), s = sign * std::sin(th);
            double v;
            if (kk < P)
                v = (n < P) ? c : s;
            else
                v = (n < P) ? -s : c;
            float hf, lf;
            uint16_t hb, lb;
            if (BF16) {
                __nv_bfloat16 h = __float2bfloat16_rn((float)v);
                hf = __bfloat162float(h);
                __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)hf));
                hb = __bfloat16_as_ushort(h);
                lb = __bfloat16_as_ushort(l);
            } else {
                __half h = __float2half_rn((float)v);
                hf = __half2float(h);
                __half l = __float2half_rn((float)(v - (double)hf));
                hb = __half_as_ushort(h);
                lb = __half_as_ushort(l);
            }
            (void)lf;
            bh[(size_t)kk * N + n] = hb;
            bl[(size_t)kk * N + n] = lb;
        }
    std::vector<uint8_t> img((size_t)G::NCHUNK * G::B_BYTES);
    for (int c = 0; c < G::NCHUNK; c++) {
        const int part = c / (KF / kTcChunk), kc = c % (KF / kTcChunk);
        const std::vector<uint16_t> &src = (part == 2) ? bl : bh;  // B' = [Bh; Bh; Bl]
        uint8_t *dst = img.data() + (size_t)c * G::B_BYTES;
        for (int n = 0; n < N; n++)
            for (int k = 0; k < kTcChunk; k++) {
                const int kk = kc * kTcChunk + k;
                const size_t off = (size_t)(n >> 3) * G::SBO_B + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
                const uint16_t val = src[(size_t)kk * N + n];
                dst[off] = (uint8_t)(val & 0xff);
                dst[off + 1] = (uint8_t)(val >> 8);
            }
    }
    return img;
}

template <int P, bool BF16>
cudaError_t run_rows(const float2 *X, float2 *Y, const void *img, int nrows, const int *out_index,
                     const float2 *conj_mul, int *err, cudaStream_t s)
{
    using G = TcGeo<P>;
    auto k = k_dft_rows_tc<P, BF16>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    const int nb = (nrows + kTcRows - 1) / kTcRows;
    k<<<nb, kTcThreads, G::SMEM, s>>>(X, Y, (const uint8_t *)img, nrows, out_index, conj_mul, err, tc_wait_limit());
    return cudaGetLastError();
}

}  // namespace

// Split BF16 (warp-specialised kernel): P = 64, 128, 256.  Split FP16 (the whole A tile in
// shared memory): P = 64, 128.
bool tc_dft_supported(int P, bool bf16) { return P == 64 || P == 128 || (bf16 && P == 256); }

namespace {
std::atomic<long long> g_tc_wait_limit{tcx::kSpinLimit};
}
long long tc_wait_limit() { return g_tc_wait_limit.load(); }
void tc_set_wait_limit(long long polls) { g_tc_wait_limit.store(polls > 0 ? polls : tcx::kSpinLimit); }

cudaError_t tc_dft_images(int P, bool bf16, int sign, std::vector<uint8_t> &out)
{
    if (bf16) return tc_ws_images(P, sign, out);  // the warp-specialised kernel's layout
    if (P == 64) out = bf16 ? build_images<64, true>(sign) : build_images<64, false>(sign);
    else if (P == 128) out = bf16 ? build_images<128, true>(sign) : build_images<128, false>(sign);
    else return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t tc_dft_rows(int P, bool bf16, const float2 *X, float2 *Y, const void *img, int nrows,
                        const int *out_index, const float2 *conj_mul, int *err, cudaStream_t s)
{
    if (bf16) return tc_ws_rows(P, X, Y, img, nrows, out_index, conj_mul, err, s);
    if (P == 64)
        return bf16 ? run_rows<64, true>(X, Y, img, nrows, out_index, conj_mul, err, s)
                    : run_rows<64, false>(X, Y, img, nrows, out_index, conj_mul, err, s);
    if (P == 128)
        return bf16 ? run_rows<128, true>(X, Y, img, nrows, out_index, conj_mul, err, s)
                    : run_rows<128, false>(X, Y, img, nrows, out_index, conj_mul, err, s);
    return cudaErrorInvalidValue;
}

// X[i] = (probe / P) * patch of sorted pattern i (Q of Eq. 1), for the tensor-core path.
__global__ void k_gather_patches(PatternArgs a, int P, const float2 *__restrict__ psi, float2 *__restrict__ X)
{
    const int i = blockIdx.x;
    const int2 rc = a.pos[i];
    float2 *xi = X + (size_t)i * P * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        const int y = e / P, x = e % P;
        const float2 p = __ldg(a.probe + e), v = __ldg(psi + (size_t)(rc.x + y) * a.W + (rc.y + x));
        xi[e] = make_float2(fmaf(p.x, v.x, -p.y * v.y), fmaf(p.x, v.y, p.y * v.x));
    }
}

cudaError_t launch_gather_patches(const PatternArgs &a, int P, const float2 *psi, float2 *X, cudaStream_t s)
{
    k_gather_patches<<<a.K, 256, 0, s>>>(a, P, psi, X);
    return cudaGetLastError();
}

}  // namespace pty

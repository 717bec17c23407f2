// scatter_tma.cu -- the object-tile scatter-add (Q^H of Eq. 3 summed over positions) with the
// per-pattern results fetched by the tensor memory accelerator.
//
// The per-pattern results W [K][P][P] (complex, written by the GRAD pass) are read once.  The
// plain scatter-add loads each pattern's window of the tile with per-thread loads, which keeps
// too few bytes in flight to use HBM fully.  Here thread 0 of a CTA (one 16 x 64 object tile)
// issues, per pattern of the tile's list, one 3-D tensor copy of the window into a ring of
// kStages shared-memory stages; the CTA adds the stage into its pixels' sums in list order
// (the same sums, in the same order, as the plain form).  W is described as a tensor of
// floats [K][P][2P]; a window is a box of 2 (kScTX + 2) floats x kScTY rows starting at an
// even complex column, so the copy's x coordinate is a multiple of 4 floats (16 bytes).
// Rows and columns outside the pattern are filled with zeros by the copy, which adds nothing.
// A ring of 4 stages (34 KB, 6 CTAs per SM) measured best at the 1024^2 workload: the scatter
// 0.126 ms with per-thread streaming loads, 0.115 ms here; consuming the stages two at a time
// (one block barrier per two patterns) 0.113 ms.
// Every mbarrier wait is bounded (spin_limit polls): on a timeout the CTA records it in *err,
// waits (bounded by the default limit) for its copies still in flight and returns without
// writing.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "pty_internal.h"
#include "reduce.cuh"
#include "scatter_tail.cuh"
#include "tc_ptx.cuh"

namespace pty {

namespace {

constexpr int kTY = kTileY, kTX = kTileX, kNT = 256, kNJ = kTY * kTX / kNT, kRowStep = kNT / kTX;
#ifndef PTY_TMA_STAGES
#define PTY_TMA_STAGES 4  // shared-memory stages of the window ring (2: 0.120, 3: 0.117, 4: 0.115, 6: 0.136 ms)
#endif
constexpr int kStages = PTY_TMA_STAGES;
// stages added per block barrier and refilled together (production workload, stages/group:
// 4/1 0.118, 4/2 0.113, 6/2 0.131, 6/3 0.126, 8/2 0.138, 8/4 0.128 ms)
constexpr int kGroup = 2;
static_assert(kStages % kGroup == 0, "whole groups of stages");
constexpr int kBoxX = kTX + 2;                  // complex columns per box (even start)
constexpr int kBoxFloats = 2 * kBoxX;           // 132 floats = 528 bytes, a multiple of 16
constexpr int kStageBytes = kBoxFloats * 4 * kTY;  // 8448 bytes, a multiple of 128
static_assert(kStageBytes % 128 == 0 && (kBoxFloats * 4) % 16 == 0 && kBoxFloats <= 256, "box shape");

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(tcx::smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(tcx::smem_u32(bar))
        : "memory");
}

template <int P>
__global__ void __launch_bounds__(kNT) k_scatter_tma(PatternArgs a, ScatterPlan plan, const __grid_constant__ CUtensorMap wmap,
                                                     float2 *__restrict__ out, int dy, const float2 *__restrict__ ep,
                                                     const float2 *__restrict__ gp, float2 *__restrict__ part,
                                                     const DevState *__restrict__ st, const float2 *__restrict__ psi,
                                                     const float *__restrict__ D, float p2, int *__restrict__ err,
                                                     long long spin_limit)
{
    const int b = blockIdx.x;
    if (st && st[plan.tile_view[b]].stalled) return;
    const bool lin = st && st[plan.tile_view[b]].lin;
    extern __shared__ __align__(128) unsigned char stage_mem[];
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ float2 red[(kNT / 32) * 3];
    __shared__ float2 tot[3];
    const int ty = b / plan.ntile_x, tx = b % plan.ntile_x;
    const int x = tx * kTX + (threadIdx.x % kTX);
    const int y0 = ty * kTY + threadIdx.x / kTX;
    const int q0 = plan.tile_start[b], n = plan.tile_start[b + 1] - q0;
    float2 acc[kNJ];
#pragma unroll
    for (int j = 0; j < kNJ; j++) acc[j] = make_float2(0.f, 0.f);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) tcx::mbar_init(full + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // thread 0: the copy of the k-th listed pattern's window into stage k % kStages
    auto issue = [&](int k) {
        const int i = __ldg(plan.tile_list + q0 + k);
        const int2 rc = __ldg(a.pos + i);
        const int xs = tx * kTX - rc.y;  // first tile column, in the pattern's columns
        const int s = k % kStages;
        tcx::mbar_expect_tx(full + s, kStageBytes);
        tma_load_3d(stage_mem + (size_t)s * kStageBytes, &wmap, 2 * (xs & ~1), ty * kTY - rc.x, i, full + s);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < n && k < kStages; k++) issue(k);

    // kGroup stages per block barrier: patterns k .. k + kGroup - 1 added in list order (the
    // same additions as one stage at a time), then their stages are refilled together
    int k = 0;
    bool failed = false;
    for (; k < n; k += kGroup) {
        bool ok = true;
#pragma unroll
        for (int g = 0; g < kGroup; g++) {
            const int kk = k + g;
            if (kk >= n) break;
            const int s = kk % kStages;
            ok = tcx::mbar_wait(full + s, (uint32_t)((kk / kStages) & 1), spin_limit) && ok;
            // the window's column of this thread: one past the even start when the start is odd
            const int2 rc = __ldg(a.pos + __ldg(plan.tile_list + q0 + kk));
            const int col = (x - tx * kTX) + ((tx * kTX - rc.y) & 1);
            const float2 *stg = reinterpret_cast<const float2 *>(stage_mem + (size_t)s * kStageBytes);
#pragma unroll
            for (int j = 0; j < kNJ; j++) {
                const float2 v = stg[(threadIdx.x / kTX + kRowStep * j) * kBoxX + col];
                acc[j].x += v.x;
                acc[j].y += v.y;
            }
        }
        if (__syncthreads_or(!ok)) {  // every thread is done with the group's stages (or a wait gave up)
            failed = true;
            break;
        }
        if (threadIdx.x == 0 && k + kStages < n) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // reads before the next copies
            for (int g = 0; g < kGroup && k + kStages + g < n; g++) issue(k + kStages + g);
        }
    }
    if (failed) {
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            // copies issued and not consumed: k .. min(n, k + kStages) - 1; waited for with the
            // default limit (whatever the test limit), so that none outlives the CTA
            for (int kk = k; kk < n && kk < k + kStages; kk++)
                tcx::mbar_wait(full + kk % kStages, (uint32_t)((kk / kStages) & 1), tcx::kSpinLimit);
        }
        __syncthreads();
        return;
    }
    scatter_tail<kNT, kNJ, kRowStep>(a, acc, x, y0, b, lin, out, dy, ep, gp, part, psi, D, p2, red, tot);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

}  // namespace

size_t scatter_tma_map_bytes() { return sizeof(CUtensorMap); }

bool make_scatter_tma_map(void *map, const float2 *w, int P, int K)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || ((uintptr_t)w & 15) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * P, (cuuint64_t)P, (cuuint64_t)K};
    const cuuint64_t strides[2] = {(cuuint64_t)2 * P * sizeof(float), (cuuint64_t)2 * P * P * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxFloats, (cuuint32_t)kTY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                           const_cast<float2 *>(w), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t launch_scatter_tma(int P, const void *map, const PatternArgs &a, const ScatterPlan &plan, float2 *out,
                               int dy, const float2 *eta_prev, const float2 *g_prev, float2 *part,
                               const DevState *st, cudaStream_t s, const float2 *psi, const float *D, int *err,
                               long long spin_limit)
{
    const float p2 = (float)P * (float)P;
    const int nb = plan.ntile_x * plan.ntile_y;
    const size_t smem = (size_t)kStages * kStageBytes;
    const CUtensorMap &m = *static_cast<const CUtensorMap *>(map);
    cudaError_t e = cudaSuccess;
    switch (P) {
    case 64:
        e = cudaFuncSetAttribute(k_scatter_tma<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_scatter_tma<64><<<nb, kNT, smem, s>>>(a, plan, m, out, dy, eta_prev, g_prev, part, st, psi, D, p2, err,
                                                    spin_limit);
        break;
    case 128:
        e = cudaFuncSetAttribute(k_scatter_tma<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_scatter_tma<128><<<nb, kNT, smem, s>>>(a, plan, m, out, dy, eta_prev, g_prev, part, st, psi, D, p2, err,
                                                     spin_limit);
        break;
    case 256:
        e = cudaFuncSetAttribute(k_scatter_tma<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            k_scatter_tma<256><<<nb, kNT, smem, s>>>(a, plan, m, out, dy, eta_prev, g_prev, part, st, psi, D, p2, err,
                                                     spin_limit);
        break;
    default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace pty

// reduce.cuh -- deterministic block reductions.
//
// Every sum has a fixed shape (lanes combined in a fixed pattern inside a warp, then warps
// in index order), so results do not depend on scheduling: two runs give identical bits.
//
// The hot kernels sum in compensated single precision ("float-float"): a value is the
// unevaluated sum hi + lo of two floats, held in a float2 (x = hi, y = lo).  FP64 runs at
// 1/64 of the FP32 rate on this GPU (2 FP64 results per clock per SM against 128 FP32),
// so an FP64 butterfly over a block costs more than the arithmetic it sums.  Each
// float-float addition adds one rounding of at most about 2^-44 times the sum of the
// operands' magnitudes (Knuth's two-sum keeps the rounding error of the leading parts
// exactly; only the sum of the trailing parts and the final renormalisation round), well
// below the 2^-24 of the per-thread FP32 partial sums that enter it.  block_sum keeps the
// plain FP64 form for the few reductions outside the iteration.
#pragma once
#include <cuda_runtime.h>

namespace pty {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums NV values per thread over the block.  red: (NT/32) * NV doubles of shared memory.
// Thread v < NV receives the block total of value v in out[v] (shared memory, NV doubles)
// after the call; the call ends with a barrier.
template <int NT, int NV>
__device__ __forceinline__ void block_sum(const double (&v)[NV], double *red, double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) {
        double s = warp_sum(v[i]);
        if (lane == 0) red[warp * NV + i] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; w++) s += red[w * NV + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// ---- float-float ---------------------------------------------------------------------

// a + b = s + e exactly (Knuth's two-sum; round to nearest, no overflow).  The explicit
// round-to-nearest intrinsics keep the compiler from contracting or reordering the steps.
__device__ __forceinline__ float2 ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}

// (a.x + a.y) + (b.x + b.y) as a normalised pair (|lo| <= ulp(hi) / 2).
__device__ __forceinline__ float2 ff_add(float2 a, float2 b)
{
    const float2 s = ff_two_sum(a.x, b.x);
    const float t = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
    const float hi = __fadd_rn(s.x, t);  // |s.x| >= |t| unless both are tiny: fast two-sum
    return make_float2(hi, __fsub_rn(t, __fsub_rn(hi, s.x)));
}

// (s.x + s.y) + x: a float added to a running float-float sum.
__device__ __forceinline__ float2 ff_add_f(float2 s, float x)
{
    const float2 h = ff_two_sum(s.x, x);
    const float t = __fadd_rn(s.y, h.y);
    const float hi = __fadd_rn(h.x, t);
    return make_float2(hi, __fsub_rn(t, __fsub_rn(hi, h.x)));
}

__device__ __forceinline__ float2 ff_from(float a) { return make_float2(a, 0.0f); }
__host__ __device__ __forceinline__ double ff_value(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 shfl_xor_ff(float2 v, int o)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// Warp total of one value, in every lane.
__device__ __forceinline__ float2 warp_sum_ff(float2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = ff_add(v, shfl_xor_ff(v, o));
    return v;
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// Warp totals of NV values (NV a power of two, 2 <= NV <= 32) by recursive halving: at
// each step a lane keeps half of its live values and trades the other half with the lane
// that keeps the complement, so each step moves half as many values as the one before.
// Afterwards lane l holds the warp total of value l >> (5 - log2 NV) in x[0].
template <int NV>
__device__ __forceinline__ void warp_scatter_sum_ff(float2 (&x)[NV])
{
    constexpr int K = ilog2(NV);
    static_assert((1 << K) == NV && NV >= 2 && NV <= 32, "NV must be a power of two in [2, 32]");
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < K; s++) {
        const int o = 16 >> s, half = (NV >> s) / 2;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < half; j++) {
            const float2 keep = up ? x[j + half] : x[j];
            const float2 send = up ? x[j] : x[j + half];
            x[j] = ff_add(keep, shfl_xor_ff(send, o));
        }
    }
#pragma unroll
    for (int o = 16 >> K; o > 0; o >>= 1) x[0] = ff_add(x[0], shfl_xor_ff(x[0], o));
}

// First half of block_sum_ff: the warp totals of the NV values into red ((NT/32) * NV float2
// of shared memory).  No barrier.
template <int NT, int NV>
__device__ __forceinline__ void block_partials_ff(const float2 (&v)[NV], float2 *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (NV >= 2 && NV <= 32 && (NV & (NV - 1)) == 0) {
        float2 x[NV];
#pragma unroll
        for (int i = 0; i < NV; i++) x[i] = v[i];
        warp_scatter_sum_ff<NV>(x);
        constexpr int SH = 5 - ilog2(NV);
        if ((lane & ((1 << SH) - 1)) == 0) red[warp * NV + (lane >> SH)] = x[0];
    } else {
#pragma unroll
        for (int i = 0; i < NV; i++) {
            const float2 s = warp_sum_ff(v[i]);
            if (lane == 0) red[warp * NV + i] = s;
        }
    }
}

// Second half: called by warp 0 (all lanes) once the partials of every warp are visible;
// out[v] (shared memory) receives the block total of value v, written by lanes of warp 0
// (readable by warp 0 after __syncwarp).
template <int NT, int NV>
__device__ __forceinline__ void combine_partials_ff(const float2 *red, float2 *out)
{
    constexpr int NW = NT / 32;
    static_assert(NW <= 32, "at most 32 warps");
    static_assert(NV <= 32, "one value per lane of warp 0");
    const int lane = threadIdx.x & 31;
    if constexpr (NW <= 8) {  // few warps: thread v adds the partials of value v in order
        if (lane < NV) {
            float2 s = red[lane];
            for (int w = 1; w < NW; w++) s = ff_add(s, red[w * NV + lane]);
            out[lane] = s;
        }
    } else {  // many warps: one warp combines the partials as a tree
        float2 x[NV];
#pragma unroll
        for (int i = 0; i < NV; i++) x[i] = lane < NW ? red[lane * NV + i] : make_float2(0.f, 0.f);
        if constexpr (NV >= 2 && NV <= 32 && (NV & (NV - 1)) == 0) {
            warp_scatter_sum_ff<NV>(x);
            constexpr int SH = 5 - ilog2(NV);
            if ((lane & ((1 << SH) - 1)) == 0) out[lane >> SH] = x[0];
        } else {
#pragma unroll
            for (int i = 0; i < NV; i++) {
                const float2 s = warp_sum_ff(x[i]);
                if (lane == 0) out[i] = s;
            }
        }
    }
}

// Sums NV float-float values per thread over the block.  red: (NT/32) * NV float2 of shared
// memory; thread v < NV receives the block total of value v in out[v] (shared memory, NV
// float2) after the call; the call ends with a barrier.
template <int NT, int NV>
__device__ __forceinline__ void block_sum_ff(const float2 (&v)[NV], float2 *red, float2 *out)
{
    block_partials_ff<NT, NV>(v, red);
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) combine_partials_ff<NT, NV>(red, out);
    __syncthreads();
}

// The same for plain per-thread FP32 partial sums.
template <int NT, int NV>
__device__ __forceinline__ void block_sum_ff(const float (&v)[NV], float2 *red, float2 *out)
{
    float2 x[NV];
#pragma unroll
    for (int i = 0; i < NV; i++) x[i] = ff_from(v[i]);
    block_sum_ff<NT, NV>(x, red, out);
}

}  // namespace pty

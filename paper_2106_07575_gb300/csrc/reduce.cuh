// reduce.cuh -- deterministic block reductions in FP64.
//
// Every sum has a fixed shape (xor butterfly inside a warp, then warps in index order),
// so results do not depend on scheduling: two runs give identical bits.
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

}  // namespace pty

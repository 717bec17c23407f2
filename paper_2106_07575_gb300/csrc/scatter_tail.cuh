// scatter_tail.cuh -- the end of an object-tile scatter-add (both forms of it): with the
// accumulated gradient of the thread's kScNJ pixels, add the linear form's P^2 D psi term,
// write g, and form the tile's sums for the DIR stage (Eq. 6): ||g||^2, Re<eta_{m-1}, g -
// g_{m-1}> and (linear form) sum D |psi|^2, summed in float-float over the block.
#pragma once
#include "pty_internal.h"
#include "reduce.cuh"

namespace pty {

template <int NT, int NJ, int ROWSTEP>
__device__ __forceinline__ void scatter_tail(const PatternArgs &a, float2 (&acc)[NJ], int x, int y0, int b, bool lin,
                                             float2 *__restrict__ out, int dy, const float2 *__restrict__ ep,
                                             const float2 *__restrict__ gp, float2 *__restrict__ part,
                                             const float2 *__restrict__ psi, const float *__restrict__ D, float p2,
                                             float2 *red, float2 *tot)
{
    float gg = 0.f, den = 0.f, pd = 0.f;
    if (x < a.W) {
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            const int y = y0 + ROWSTEP * j;
            if (y < a.H) {
                const size_t o = (size_t)y * a.W + x;
                if (lin) {  // the |p|^2 psi terms of the linear form, summed over positions: P^2 D psi
                    const float2 pv = __ldg(psi + o);
                    const float dd = __ldg(D + o);
                    acc[j].x = fmaf(p2 * dd, pv.x, acc[j].x);
                    acc[j].y = fmaf(p2 * dd, pv.y, acc[j].y);
                    pd = fmaf(dd, fmaf(pv.x, pv.x, pv.y * pv.y), pd);
                }
                out[o] = acc[j];
                if (dy) {
                    const float2 e = __ldg(ep + o), g0 = __ldg(gp + o);
                    gg = fmaf(acc[j].x, acc[j].x, fmaf(acc[j].y, acc[j].y, gg));
                    den = fmaf(e.x, acc[j].x - g0.x, fmaf(e.y, acc[j].y - g0.y, den));
                }
            }
        }
    }
    if (dy) {
        float v[3] = {gg, den, pd};
        block_sum_ff<NT, 3>(v, red, tot);
        if (threadIdx.x < 3) part[3 * b + threadIdx.x] = tot[threadIdx.x];  // [ntiles][3]
    }
}

}  // namespace pty

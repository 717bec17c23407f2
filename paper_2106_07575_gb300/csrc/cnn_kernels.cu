// cnn_kernels.cu -- kernels of the learned initial guess: features, 3x3 convolutions
// (forward, backward-data, backward-weights), GELU, the bounded amplitude/phase head and
// its loss, Adam, and the probe-weighted stitching of predicted patches.
//
// Layouts: activations [B][C][P][P] FP32; weights BF16 [Cout][Cin][3][3] (FP32 masters
// elsewhere), biases FP32.  All sums that decide a result are taken in a fixed order, so
// every output is bitwise reproducible.
//
// Convolution tiling (k_conv): a CTA of 256 threads computes ROWS full image rows for all
// 32 output channels; thread (tx, cg, r) owns 8 consecutive pixels x 8 output channels (64
// FP32 accumulators).  Input channels are staged in chunks of 8 in shared memory, one row
// segment of 8 pixels padded by one float so that the 16-32 threads reading the same row
// hit distinct banks; weights are staged as [ci][tap][co] floats and read as float4 pairs.
// Per input channel a thread issues 30 + 18 shared loads for 576 FMAs.
#include <cuda_bf16.h>

#include <cmath>

#include "cnn_internal.h"
#include "reduce.cuh"

namespace pty {
namespace cnn {

namespace {

constexpr int NT = 256;
constexpr float kHalfPi = 1.57079632679489662f;
constexpr float kInvSqrt2Pi = 0.398942280401432678f;

__device__ __forceinline__ float gelu(float z) { return z * normcdff(z); }
__device__ __forceinline__ float gelu_grad(float z) { return normcdff(z) + z * kInvSqrt2Pi * expf(-0.5f * z * z); }
__device__ __forceinline__ float sigmoid(float z) { return 1.f / (1.f + expf(-z)); }

__global__ void k_features(int P, int B, const float *__restrict__ d, const int *__restrict__ idx,
                           float *__restrict__ x)
{
    const size_t n = (size_t)B * P * P;
    const int PP = P * P, h = P / 2;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / PP), r = (int)(i % PP);
        const int y = r / P, xx = r % P;
        const size_t src = idx ? (size_t)__ldg(idx + b) : (size_t)b;
        const float v = __ldg(d + src * PP + (size_t)((y + h) % P) * P + (xx + h) % P);
        x[i] = log1pf(sqrtf(fmaxf(v, 0.f)));
    }
}

// ---- 3x3 convolution, kC output channels ----
template <int P, int CIN>
struct ConvCfg {
    static constexpr int TX = P / 8;                 // threads along a row (8 px each)
    static constexpr int ROWS = NT / (TX * 4);       // output rows per CTA
    static constexpr int CC = CIN < 8 ? CIN : 8;     // input channels per chunk
    static constexpr int RS = (P + 2) + (P + 9) / 8 + 1;  // padded smem row: xs -> xs + xs / 8
    static constexpr int CH = (ROWS + 2) * RS;
};

template <int P, int CIN, bool BWD>
__global__ void __launch_bounds__(NT, 2)
    k_conv(const float *__restrict__ in, const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias,
           const float *__restrict__ zprev, float *__restrict__ zout, float *__restrict__ aout)
{
    using G = ConvCfg<P, CIN>;
    constexpr int TX = G::TX, ROWS = G::ROWS, CC = G::CC, RS = G::RS, CH = G::CH;
    static_assert(NT % (TX * 4) == 0 && P % ROWS == 0 && CIN % CC == 0, "conv tiling");
    __shared__ float s_in[CC * CH];
    __shared__ __align__(16) float s_w[CC * 9 * kC];
    const int tid = threadIdx.x;
    const int tx = tid % TX, cg = (tid / TX) % 4, r = tid / (TX * 4);
    constexpr int tiles = P / ROWS;
    const int b = blockIdx.x / tiles, y0 = (blockIdx.x % tiles) * ROWS;

    float acc[8][8];
#pragma unroll
    for (int c = 0; c < 8; c++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[c][j] = 0.f;

    for (int c0 = 0; c0 < CIN; c0 += CC) {
        __syncthreads();
        for (int e = tid; e < CC * (ROWS + 2) * (P + 2); e += NT) {
            const int xs = e % (P + 2), t = e / (P + 2);
            const int rr = t % (ROWS + 2), cc = t / (ROWS + 2);
            const int y = y0 - 1 + rr, x = xs - 1;
            float v = 0.f;
            if (y >= 0 && y < P && x >= 0 && x < P) v = __ldg(in + (((size_t)b * CIN + c0 + cc) * P + y) * P + x);
            s_in[cc * CH + rr * RS + xs + xs / 8] = v;
        }
        for (int e = tid; e < kC * CC * 9; e += NT) {
            const int co = e / (CC * 9), rem = e % (CC * 9);
            s_w[rem * kC + co] = __bfloat162float(w[((size_t)co * CIN + c0) * 9 + rem]);
        }
        __syncthreads();
#pragma unroll 2
        for (int cc = 0; cc < CC; cc++) {
#pragma unroll
            for (int dy = 0; dy < 3; dy++) {
                const float *row = s_in + cc * CH + (r + dy) * RS + 9 * tx;
                float v[10];
#pragma unroll
                for (int j = 0; j < 8; j++) v[j] = row[j];
                v[8] = row[9];
                v[9] = row[10];
#pragma unroll
                for (int dx = 0; dx < 3; dx++) {
                    const float4 *wp = reinterpret_cast<const float4 *>(s_w + (cc * 9 + dy * 3 + dx) * kC + 8 * cg);
                    const float4 wa = wp[0], wb = wp[1];
                    const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                    for (int c = 0; c < 8; c++)
#pragma unroll
                        for (int j = 0; j < 8; j++) acc[c][j] = fmaf(wv[c], v[j + dx], acc[c][j]);
                }
            }
        }
    }

    const int y = y0 + r, x0 = 8 * tx;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int co = 8 * cg + c;
        const size_t o = (((size_t)b * kC + co) * P + y) * P + x0;
        float4 *z4 = reinterpret_cast<float4 *>(zout + o);
        if (!BWD) {
            const float bb = __ldg(bias + co);
            float zz[8], aa[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                zz[j] = acc[c][j] + bb;
                aa[j] = gelu(zz[j]);
            }
            z4[0] = make_float4(zz[0], zz[1], zz[2], zz[3]);
            z4[1] = make_float4(zz[4], zz[5], zz[6], zz[7]);
            float4 *a4 = reinterpret_cast<float4 *>(aout + o);
            a4[0] = make_float4(aa[0], aa[1], aa[2], aa[3]);
            a4[1] = make_float4(aa[4], aa[5], aa[6], aa[7]);
        } else {
            const float4 *p4 = reinterpret_cast<const float4 *>(zprev + o);
            const float4 pa = __ldg(p4), pb = __ldg(p4 + 1);
            const float zp[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
            float oo[8];
#pragma unroll
            for (int j = 0; j < 8; j++) oo[j] = acc[c][j] * gelu_grad(zp[j]);
            z4[0] = make_float4(oo[0], oo[1], oo[2], oo[3]);
            z4[1] = make_float4(oo[4], oo[5], oo[6], oo[7]);
        }
    }
}

// ---- output layer: kC -> 2 channels; thread owns 8 consecutive pixels x 2 channels ----
template <int P>
struct HeadCfg {
    static constexpr int TX = P / 8;
    static constexpr int ROWS = NT / TX;
    static constexpr int CC = P >= 256 ? 2 : 4;
    static constexpr int RS = (P + 2) + (P + 9) / 8 + 1;
    static constexpr int CH = (ROWS + 2) * RS;
};

template <int P>
__global__ void __launch_bounds__(NT) k_conv_head(const float *__restrict__ in, const __nv_bfloat16 *__restrict__ w,
                                                  const float *__restrict__ bias, float *__restrict__ z)
{
    using G = HeadCfg<P>;
    constexpr int TX = G::TX, ROWS = G::ROWS, CC = G::CC, RS = G::RS, CH = G::CH;
    __shared__ float s_in[CC * CH];
    __shared__ __align__(8) float s_w[kC * 9 * 2];  // [ci][tap][co]
    const int tid = threadIdx.x, tx = tid % TX, r = tid / TX;
    constexpr int tiles = P / ROWS;
    const int b = blockIdx.x / tiles, y0 = (blockIdx.x % tiles) * ROWS;
    for (int e = tid; e < 2 * kC * 9; e += NT) {
        const int co = e / (kC * 9), rem = e % (kC * 9);
        s_w[rem * 2 + co] = __bfloat162float(w[e]);
    }
    float acc[2][8];
#pragma unroll
    for (int j = 0; j < 8; j++) acc[0][j] = acc[1][j] = 0.f;
    for (int c0 = 0; c0 < kC; c0 += CC) {
        __syncthreads();
        for (int e = tid; e < CC * (ROWS + 2) * (P + 2); e += NT) {
            const int xs = e % (P + 2), t = e / (P + 2);
            const int rr = t % (ROWS + 2), cc = t / (ROWS + 2);
            const int y = y0 - 1 + rr, x = xs - 1;
            float v = 0.f;
            if (y >= 0 && y < P && x >= 0 && x < P) v = __ldg(in + (((size_t)b * kC + c0 + cc) * P + y) * P + x);
            s_in[cc * CH + rr * RS + xs + xs / 8] = v;
        }
        __syncthreads();
        for (int cc = 0; cc < CC; cc++) {
#pragma unroll
            for (int dy = 0; dy < 3; dy++) {
                const float *row = s_in + cc * CH + (r + dy) * RS + 9 * tx;
                float v[10];
#pragma unroll
                for (int j = 0; j < 8; j++) v[j] = row[j];
                v[8] = row[9];
                v[9] = row[10];
#pragma unroll
                for (int dx = 0; dx < 3; dx++) {
                    const float2 ww = *reinterpret_cast<const float2 *>(s_w + ((c0 + cc) * 9 + dy * 3 + dx) * 2);
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        acc[0][j] = fmaf(ww.x, v[j + dx], acc[0][j]);
                        acc[1][j] = fmaf(ww.y, v[j + dx], acc[1][j]);
                    }
                }
            }
        }
    }
    const int y = y0 + r, x0 = 8 * tx;
#pragma unroll
    for (int co = 0; co < 2; co++) {
        const float bb = __ldg(bias + co);
        float4 *z4 = reinterpret_cast<float4 *>(z + (((size_t)b * 2 + co) * P + y) * P + x0);
        z4[0] = make_float4(acc[co][0] + bb, acc[co][1] + bb, acc[co][2] + bb, acc[co][3] + bb);
        z4[1] = make_float4(acc[co][4] + bb, acc[co][5] + bb, acc[co][6] + bb, acc[co][7] + bb);
    }
}

// ---- head and loss ----
__global__ void __launch_bounds__(NT) k_head_loss(int P, int B, const float *__restrict__ z, const int *__restrict__ idx,
                                                  const float2 *__restrict__ t, const float *__restrict__ w,
                                                  float inv_norm, float2 *__restrict__ o_out, float *__restrict__ dz,
                                                  double *__restrict__ part)
{
    __shared__ float2 red[NT / 32], tot[1];
    const size_t PP = (size_t)P * P, n = (size_t)B * PP;
    const size_t i = (size_t)blockIdx.x * NT + threadIdx.x;
    float l = 0.0f;
    if (i < n) {
        const size_t b = i / PP, px = i % PP;
        const float z0 = __ldg(z + (2 * b) * PP + px), z1 = __ldg(z + (2 * b + 1) * PP + px);
        const float s0 = sigmoid(z0), s1 = sigmoid(z1);
        const float amp = 0.8f + 0.2f * s0, ph = kHalfPi * s1;
        float sn, cs;
        sincosf(ph, &sn, &cs);
        const float2 o = make_float2(amp * cs, amp * sn);
        if (o_out) o_out[i] = o;
        if (t) {
            const size_t src = idx ? (size_t)__ldg(idx + b) : b;
            const float2 tt = __ldg(t + src * PP + px);
            const float rx = o.x - tt.x, ry = o.y - tt.y, ww = __ldg(w + px);
            l = ww * fmaf(rx, rx, ry * ry);
            const float g = 2.f * ww * inv_norm;
            const float damp = g * (rx * cs + ry * sn);
            const float dph = g * (ry * o.x - rx * o.y);
            dz[(2 * b) * PP + px] = damp * 0.2f * s0 * (1.f - s0);
            dz[(2 * b + 1) * PP + px] = dph * kHalfPi * s1 * (1.f - s1);
        }
    }
    if (part) {  // float-float block sum (FP64 runs at 1/64 of the FP32 rate)
        float v[1] = {l};
        block_sum_ff<NT, 1>(v, red, tot);
        if (threadIdx.x == 0) part[blockIdx.x] = ff_value(tot[0]);
    }
}

__global__ void k_loss_finalize(const double *__restrict__ part, int n, double inv_norm, double *__restrict__ loss)
{
    __shared__ double red[NT / 32], tot[1];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) s += part[i];
    double v[1] = {s};
    block_sum<NT, 1>(v, red, tot);
    if (threadIdx.x == 0) loss[0] = tot[0] * inv_norm;
}

// ---- weight gradient ----
// Thread (cog, ci, ph) accumulates dW[co][ci][tap] for the CG output channels of cog over
// the x-segment ph of every row of the CTA's band, with a sliding 3x3 input window.
// Phases of one (cog, ci) are adjacent lanes and are combined by a fixed xor butterfly.
constexpr int kWgRB = 16;   // rows per CTA
constexpr int kWgRCH = 2;   // rows per shared-memory chunk

template <int P, int CIN, int COUT, int CG>
struct WgCfg {
    static constexpr int NCOG = COUT / CG;
    static constexpr int NPH = NT / (NCOG * CIN);
    static constexpr int SEG = P / NPH;
    static constexpr int AW = (P + 2) + (P + 2) / SEG + 1;  // xs -> xs + xs / SEG
    static constexpr int ABASE = (kWgRCH + 2) * AW;
    // channel stride: odd when a warp holds 32 channels at one pixel; shifted by 8 banks
    // per channel when a warp holds 4 channels x 8 segments
    static constexpr int ASTR = CIN == 1 ? ABASE : (NPH == 1 ? (ABASE | 1) : ((ABASE + 31) / 32 * 32 + 8));
    static constexpr int DW = P + P / SEG;
    static constexpr int DSTR = kWgRCH * DW;
    static constexpr size_t SMEM = sizeof(float) * ((size_t)CIN * ASTR + (size_t)COUT * DSTR);
    static_assert(NT % (NCOG * CIN) == 0 && P % NPH == 0 && SEG >= 2, "wgrad tiling");
};

template <int P, int CIN, int COUT, int CG>
__global__ void __launch_bounds__(NT) k_wgrad(const float *__restrict__ a, const float *__restrict__ dz,
                                              float *__restrict__ part)
{
    using G = WgCfg<P, CIN, COUT, CG>;
    constexpr int NPH = G::NPH, SEG = G::SEG, AW = G::AW, ASTR = G::ASTR, DW = G::DW, DSTR = G::DSTR;
    constexpr int NPL = COUT * CIN * 9 + COUT;
    extern __shared__ float smem[];
    float *s_a = smem, *s_d = smem + (size_t)CIN * ASTR;
    const int tid = threadIdx.x;
    const int ph = tid % NPH, ci = (tid / NPH) % CIN, cog = tid / (NPH * CIN);
    constexpr int bands = P / kWgRB;
    const int b = blockIdx.x / bands, yb = (blockIdx.x % bands) * kWgRB;

    float acc[CG][9], bacc[CG];
#pragma unroll
    for (int c = 0; c < CG; c++) {
        bacc[c] = 0.f;
#pragma unroll
        for (int k = 0; k < 9; k++) acc[c][k] = 0.f;
    }

    for (int yc = 0; yc < kWgRB; yc += kWgRCH) {
        const int ylo = yb + yc;
        __syncthreads();
        for (int e = tid; e < CIN * (kWgRCH + 2) * (P + 2); e += NT) {
            const int xs = e % (P + 2), t = e / (P + 2);
            const int rr = t % (kWgRCH + 2), c = t / (kWgRCH + 2);
            const int y = ylo - 1 + rr, x = xs - 1;
            float v = 0.f;
            if (y >= 0 && y < P && x >= 0 && x < P) v = __ldg(a + (((size_t)b * CIN + c) * P + y) * P + x);
            s_a[c * ASTR + rr * AW + xs + xs / SEG] = v;
        }
        for (int e = tid; e < COUT * kWgRCH * P; e += NT) {
            const int x = e % P, t = e / P;
            const int rr = t % kWgRCH, c = t / kWgRCH;
            s_d[c * DSTR + rr * DW + x + x / SEG] = __ldg(dz + (((size_t)b * COUT + c) * P + ylo + rr) * P + x);
        }
        __syncthreads();
#pragma unroll 1
        for (int rr = 0; rr < kWgRCH; rr++) {
            const float *ar = s_a + ci * ASTR + rr * AW + ph * (SEG + 1);
            const float *dr = s_d + (cog * CG) * DSTR + rr * DW + ph * (SEG + 1);
            float win[3][3];
#pragma unroll
            for (int dy = 0; dy < 3; dy++) {
                win[dy][0] = ar[dy * AW + 0];
                win[dy][1] = ar[dy * AW + 1];
            }
#pragma unroll 4
            for (int i = 0; i < SEG; i++) {
                const int i2 = i + 2 + (i + 2) / SEG;
#pragma unroll
                for (int dy = 0; dy < 3; dy++) win[dy][2] = ar[dy * AW + i2];
#pragma unroll
                for (int c = 0; c < CG; c++) {
                    const float g = dr[c * DSTR + i];
                    bacc[c] += g;
#pragma unroll
                    for (int dy = 0; dy < 3; dy++)
#pragma unroll
                        for (int dx = 0; dx < 3; dx++) acc[c][dy * 3 + dx] = fmaf(g, win[dy][dx], acc[c][dy * 3 + dx]);
                }
#pragma unroll
                for (int dy = 0; dy < 3; dy++) {
                    win[dy][0] = win[dy][1];
                    win[dy][1] = win[dy][2];
                }
            }
        }
    }
    if (NPH > 1) {
#pragma unroll
        for (int c = 0; c < CG; c++) {
#pragma unroll
            for (int o = NPH / 2; o > 0; o >>= 1) {
                bacc[c] += __shfl_xor_sync(0xffffffffu, bacc[c], o);
#pragma unroll
                for (int k = 0; k < 9; k++) acc[c][k] += __shfl_xor_sync(0xffffffffu, acc[c][k], o);
            }
        }
    }
    if (ph == 0) {
        float *pb = part + (size_t)blockIdx.x * NPL;
#pragma unroll
        for (int c = 0; c < CG; c++) {
            const int co = cog * CG + c;
#pragma unroll
            for (int k = 0; k < 9; k++) pb[((size_t)co * CIN + ci) * 9 + k] = acc[c][k];
            if (ci == 0) pb[COUT * CIN * 9 + co] = bacc[c];
        }
    }
}

// grad[p] = sum over k of part[k][p] for 32 consecutive p per block: warp w adds the
// partials k = w, w + NW, ... (coalesced rows of 32), then warp 0 adds the NW warp sums in
// order w = 0 .. NW - 1.  Float-float throughout (FP64 runs at 1/64 of the FP32 rate); the
// order depends only on nblk.
__global__ void __launch_bounds__(NT) k_wreduce(const float *__restrict__ part, int nblk, int npl,
                                                float *__restrict__ grad)
{
    constexpr int NW = NT / 32;
    __shared__ float2 ws[NW][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    float2 s = make_float2(0.f, 0.f);
    if (p < npl) {
#pragma unroll 4
        for (int k = w; k < nblk; k += NW) s = ff_add_f(s, __ldg(part + (size_t)k * npl + p));
    }
    ws[w][lane] = s;
    __syncthreads();
    if (w == 0 && p < npl) {
        float2 t = ws[0][lane];
#pragma unroll
        for (int v = 1; v < NW; v++) t = ff_add(t, ws[v][lane]);
        grad[p] = t.x + t.y;
    }
}

// ---- Adam and the BF16 working copies ----
__global__ void k_adam(float *__restrict__ master, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        master[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

__global__ void k_refresh(const float *__restrict__ master, int cout, int cin, __nv_bfloat16 *__restrict__ w16,
                          __nv_bfloat16 *__restrict__ wt16)
{
    const int n = cout * cin * 9;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int co = i / (cin * 9), ci = (i / 9) % cin, tap = i % 9;
        const __nv_bfloat16 h = __float2bfloat16_rn(master[i]);
        w16[i] = h;
        if (wt16) wt16[((size_t)ci * cout + co) * 9 + (8 - tap)] = h;
    }
}

// ---- stitching ----
constexpr int kStTY = kTileY, kStTX = kTileX, kStNJ = kStTY * kStTX / NT;

template <int P>
__global__ void __launch_bounds__(NT) k_stitch_acc(PatternArgs a, ScatterPlan plan, const float2 *__restrict__ patches,
                                                   float2 *__restrict__ num, float *__restrict__ den,
                                                   float *__restrict__ tile_max)
{
    __shared__ float red[NT / 32];
    const int blk = blockIdx.x;
    const int ty = blk / plan.ntile_x, tx = blk % plan.ntile_x;
    const int x = tx * kStTX + (threadIdx.x % kStTX);
    const int y0 = ty * kStTY + threadIdx.x / kStTX;
    float2 acc[kStNJ];
    float wacc[kStNJ];
#pragma unroll
    for (int j = 0; j < kStNJ; j++) {
        acc[j] = make_float2(0.f, 0.f);
        wacc[j] = 0.f;
    }
    const int q0 = plan.tile_start[blk], q1 = plan.tile_start[blk + 1];
    for (int q = q0; q < q1; q++) {
        const int i = __ldg(plan.tile_list + q);
        const int2 rc = __ldg(a.pos + i);
        const int dx = x - rc.y;
        if (dx < 0 || dx >= P) continue;
        const float2 *pi = patches + (size_t)__ldg(a.perm + i) * P * P + dx;
        const float2 *pk = probe_of(a, i);
#pragma unroll
        for (int j = 0; j < kStNJ; j++) {
            const int yy = y0 + (NT / kStTX) * j - rc.x;
            if (yy >= 0 && yy < P) {
                const float2 p = __ldg(pk + yy * P + dx);
                const float w = p.x * p.x + p.y * p.y;
                const float2 o = __ldg(pi + yy * P);
                acc[j].x = fmaf(w, o.x, acc[j].x);
                acc[j].y = fmaf(w, o.y, acc[j].y);
                wacc[j] += w;
            }
        }
    }
    float mx = 0.f;
    if (x < a.W) {
#pragma unroll
        for (int j = 0; j < kStNJ; j++) {
            const int y = y0 + (NT / kStTX) * j;
            if (y < a.H) {
                const size_t o = (size_t)y * a.W + x;
                num[o] = acc[j];
                den[o] = wacc[j];
                mx = fmaxf(mx, wacc[j]);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int k = 0; k < NT / 32; k++) m = fmaxf(m, red[k]);
        tile_max[blk] = m;
    }
}

__global__ void k_max(const float *__restrict__ v, int n, float *__restrict__ out)
{
    __shared__ float red[NT / 32];
    float m = 0.f;
    for (int i = threadIdx.x; i < n; i += NT) m = fmaxf(m, v[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int k = 0; k < NT / 32; k++) r = fmaxf(r, red[k]);
        out[0] = r;
    }
}

__global__ void k_stitch_finish(size_t n, const float2 *__restrict__ num, const float *__restrict__ den, float floor_,
                                const float *__restrict__ dmax, float2 *__restrict__ out)
{
    const float f = floor_ * __ldg(dmax);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float dd = den[i];
        if (dd > 0.f) {
            const float2 u = num[i];
            const float inv = 1.f / (dd + f);
            out[i] = make_float2(u.x * inv, u.y * inv);
        } else {
            out[i] = make_float2(1.f, 0.f);
        }
    }
}

// part[block] = sum over the block's grid-stride share of |x|^2 w (x complex, w real, both
// may be offset views) or of plain floats (x NULL).
constexpr int kRedBlocks = 1024;

__global__ void __launch_bounds__(NT) k_partial_sums(const float2 *__restrict__ x, const float *__restrict__ w, size_t n,
                                                     double *__restrict__ part)
{
    __shared__ float2 red[NT / 32], tot[1];
    float2 s = make_float2(0.f, 0.f);  // float-float: FP64 runs at 1/64 of the FP32 rate
    for (size_t i = (size_t)blockIdx.x * NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
        if (x) {
            const float2 v = x[i];
            s = ff_add_f(s, fmaf(v.x, v.x, v.y * v.y) * w[i]);
        } else {
            s = ff_add_f(s, w[i]);
        }
    }
    float2 v[1] = {s};
    block_sum_ff<NT, 1>(v, red, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = ff_value(tot[0]);
}

__global__ void k_scale(float2 *__restrict__ x, size_t n, const double *__restrict__ num, const double *__restrict__ den,
                        double *__restrict__ c_out)
{
    const double c = den[0] > 0.0 ? sqrt(num[0] / den[0]) : 1.0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && c_out) c_out[0] = c;
    const float cf = (float)c;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = x[i];
        x[i] = make_float2(v.x * cf, v.y * cf);
    }
}

__global__ void k_fill_ones(float2 *x, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = make_float2(1.f, 0.f);
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + NT - 1) / NT, 152 * 16); }

template <int P>
cudaError_t conv_fwd_p(int cin, int B, const float *in, const __nv_bfloat16 *w, const float *bias, float *z, float *a,
                       cudaStream_t s)
{
    if (cin == 1) {
        k_conv<P, 1, false><<<B * (P / ConvCfg<P, 1>::ROWS), NT, 0, s>>>(in, w, bias, nullptr, z, a);
    } else if (cin == kC) {
        k_conv<P, kC, false><<<B * (P / ConvCfg<P, kC>::ROWS), NT, 0, s>>>(in, w, bias, nullptr, z, a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t conv_bwd_p(int cin, int B, const float *in, const __nv_bfloat16 *wt, const float *zprev, float *out,
                       cudaStream_t s)
{
    if (cin == 2) {
        k_conv<P, 2, true><<<B * (P / ConvCfg<P, 2>::ROWS), NT, 0, s>>>(in, wt, nullptr, zprev, out, nullptr);
    } else if (cin == kC) {
        k_conv<P, kC, true><<<B * (P / ConvCfg<P, kC>::ROWS), NT, 0, s>>>(in, wt, nullptr, zprev, out, nullptr);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int P, int CIN, int COUT, int CG>
cudaError_t wgrad_p(int B, const float *a, const float *dz, float *part, cudaStream_t s)
{
    using G = WgCfg<P, CIN, COUT, CG>;
    static bool attr_set = false;  // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad<P, CIN, COUT, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)G::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_wgrad<P, CIN, COUT, CG><<<B * (P / kWgRB), NT, G::SMEM, s>>>(a, dz, part);
    return cudaGetLastError();
}

template <int P>
cudaError_t wgrad_dispatch(int cin, int cout, int B, const float *a, const float *dz, float *part, cudaStream_t s)
{
    if (cin == kC && cout == kC) return wgrad_p<P, kC, kC, 4>(B, a, dz, part, s);
    if (cin == 1 && cout == kC) return wgrad_p<P, 1, kC, 4>(B, a, dz, part, s);
    if (cin == kC && cout == 2) return wgrad_p<P, kC, 2, 2>(B, a, dz, part, s);
    return cudaErrorInvalidValue;
}

}  // namespace

bool size_supported(int P) { return P == 64 || P == 128 || P == 256; }

cudaError_t launch_features(int P, int B, const float *d, const int *idx, float *x, cudaStream_t s)
{
    k_features<<<grid_for((size_t)B * P * P), NT, 0, s>>>(P, B, d, idx, x);
    return cudaGetLastError();
}

cudaError_t launch_conv_fwd(int P, int cin, int B, const float *in, const __nv_bfloat16 *w, const float *bias,
                            float *z, float *a, int *err, cudaStream_t s)
{
    if (err && conv_tc_on() && conv_tc_supported(P, cin))
        return launch_conv_tc(P, B, false, in, w, bias, nullptr, z, a, err, s);
    switch (P) {
    case 64: return conv_fwd_p<64>(cin, B, in, w, bias, z, a, s);
    case 128: return conv_fwd_p<128>(cin, B, in, w, bias, z, a, s);
    case 256: return conv_fwd_p<256>(cin, B, in, w, bias, z, a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_conv_bwd(int P, int cin, int B, const float *in, const __nv_bfloat16 *wt, const float *zprev,
                            float *out, int *err, cudaStream_t s)
{
    if (err && conv_tc_on() && conv_tc_supported(P, cin))
        return launch_conv_tc(P, B, true, in, wt, nullptr, zprev, out, nullptr, err, s);
    switch (P) {
    case 64: return conv_bwd_p<64>(cin, B, in, wt, zprev, out, s);
    case 128: return conv_bwd_p<128>(cin, B, in, wt, zprev, out, s);
    case 256: return conv_bwd_p<256>(cin, B, in, wt, zprev, out, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_conv_head(int P, int B, const float *in, const __nv_bfloat16 *w, const float *bias, float *z,
                             cudaStream_t s)
{
    switch (P) {
    case 64: k_conv_head<64><<<B * (64 / HeadCfg<64>::ROWS), NT, 0, s>>>(in, w, bias, z); break;
    case 128: k_conv_head<128><<<B * (128 / HeadCfg<128>::ROWS), NT, 0, s>>>(in, w, bias, z); break;
    case 256: k_conv_head<256><<<B * (256 / HeadCfg<256>::ROWS), NT, 0, s>>>(in, w, bias, z); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_head_loss(int P, int B, const float *z, const int *idx, const float2 *t, const float *w,
                             double inv_norm, float2 *o_out, float *dz, double *part, int *nparts, cudaStream_t s)
{
    const size_t n = (size_t)B * P * P;
    const int nb = (int)((n + NT - 1) / NT);
    k_head_loss<<<nb, NT, 0, s>>>(P, B, z, idx, t, w, (float)inv_norm, o_out, dz, t ? part : nullptr);
    if (nparts) *nparts = nb;
    return cudaGetLastError();
}

cudaError_t launch_loss_finalize(const double *part, int n, double inv_norm, double *loss, cudaStream_t s)
{
    k_loss_finalize<<<1, NT, 0, s>>>(part, n, inv_norm, loss);
    return cudaGetLastError();
}

int wgrad_blocks(int P, int B) { return B * (P / kWgRB); }

int wgrad_part_blocks(int P, int B)
{
    const int t = wgrad_tc_supported(P, kC, kC) ? wgrad_tc_blocks(P, B) : 0;
    return wgrad_blocks(P, B) > t ? wgrad_blocks(P, B) : t;
}

cudaError_t launch_wgrad(int P, int cin, int cout, int B, const float *a, const float *dz, float *part, float *grad,
                         int *err, cudaStream_t s)
{
    cudaError_t e;
    if (err && conv_tc_on() && wgrad_tc_supported(P, cin, cout)) {
        e = launch_wgrad_tc(P, B, a, dz, part, err, s);
        if (e != cudaSuccess) return e;
        const int npl = cout * cin * 9 + cout;
        k_wreduce<<<(npl + 31) / 32, NT, 0, s>>>(part, wgrad_tc_blocks(P, B), npl, grad);
        return cudaGetLastError();
    }
    switch (P) {
    case 64: e = wgrad_dispatch<64>(cin, cout, B, a, dz, part, s); break;
    case 128: e = wgrad_dispatch<128>(cin, cout, B, a, dz, part, s); break;
    case 256: e = wgrad_dispatch<256>(cin, cout, B, a, dz, part, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int npl = cout * cin * 9 + cout;
    k_wreduce<<<(npl + 31) / 32, NT, 0, s>>>(part, wgrad_blocks(P, B), npl, grad);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *master, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, cudaStream_t s)
{
    k_adam<<<grid_for((size_t)n), NT, 0, s>>>(master, m, v, g, n, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t launch_refresh(const float *master, int cout, int cin, __nv_bfloat16 *w16, __nv_bfloat16 *wt16,
                           cudaStream_t s)
{
    k_refresh<<<grid_for((size_t)cout * cin * 9), NT, 0, s>>>(master, cout, cin, w16, wt16);
    return cudaGetLastError();
}

cudaError_t launch_stitch(int P, const PatternArgs &a, const ScatterPlan &plan, const float2 *patches, float floor_,
                          float2 *num, float *den, float *tile_max, float *dmax, float2 *out, cudaStream_t s)
{
    if (plan.TY != kStTY || plan.TX != kStTX) return cudaErrorInvalidValue;
    const int nb = plan.ntile_x * plan.ntile_y;
    switch (P) {
    case 64: k_stitch_acc<64><<<nb, NT, 0, s>>>(a, plan, patches, num, den, tile_max); break;
    case 128: k_stitch_acc<128><<<nb, NT, 0, s>>>(a, plan, patches, num, den, tile_max); break;
    case 256: k_stitch_acc<256><<<nb, NT, 0, s>>>(a, plan, patches, num, den, tile_max); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_max<<<1, NT, 0, s>>>(tile_max, nb, dmax);
    const size_t n = (size_t)a.H * a.W;
    k_stitch_finish<<<grid_for(n), NT, 0, s>>>(n, num, den, floor_, dmax, out);
    return cudaGetLastError();
}

cudaError_t launch_sum_sq_weighted(const float2 *x, const float *w, size_t n, double *part, double *out, double scale,
                                   cudaStream_t s)
{
    k_partial_sums<<<kRedBlocks, NT, 0, s>>>(x, w, n, part);
    k_loss_finalize<<<1, NT, 0, s>>>(part, kRedBlocks, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_scale_to(float2 *x, size_t n, const double *num, const double *den, double *c_out, cudaStream_t s)
{
    k_scale<<<grid_for(n), NT, 0, s>>>(x, n, num, den, c_out);
    return cudaGetLastError();
}

cudaError_t launch_fill_ones(float2 *x, size_t n, cudaStream_t s)
{
    k_fill_ones<<<grid_for(n), NT, 0, s>>>(x, n);
    return cudaGetLastError();
}

}  // namespace cnn
}  // namespace pty

// fft_tile.cuh -- 2-D DFT of one P x P complex exit wave held in shared memory, by one CTA
// or by a thread-block cluster of CS = P / R CTAs.
//
// This is the F of Eq. 1 (and F^H of Eq. 3) in the paper: the far-field transform of one
// exit wave.  Each 1-D transform of length P = R1 * R2 (R1 = 16, R2 = P/16) is split
// Cooley-Tukey style into two in-place passes over the lines of a buffer:
//   stride pass: radix-16 DFT over the elements n2 + R2*n1 (n1 = 0..15), then the
//                twiddle W_P^{n2 k1}, written back to the same slots;
//   block pass : radix-R2 DFT over the contiguous block n2 + R2*k1 (n2 = 0..R2-1),
//                written back to the same slots.
// Forward (stride, block) leaves frequency k1 + R1*k2 in slot k2 + R2*k1 ("permuted"
// order); the inverse runs (block, stride) with conjugate twiddles applied before the
// radix-16 step and takes the permuted order back to natural order.  Both passes are in
// place: a thread keeps one line segment in registers at a time and a barrier separates
// passes.
//
// Layout.  CTA c of a cluster owns the R rows [cR, cR+R) during the row passes ("row
// slab", row stride P+1) and the R columns [cR, cR+R) during the column passes ("column
// slab", row stride R+1).  The change of slab is an all-to-all through distributed shared
// memory (exchange_*).  With R = P the two layouts coincide and no exchange happens.
// Lines are mapped to consecutive threads in both layouts, which keeps every warp access
// free of shared-memory bank conflicts.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

namespace pty {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}

// cos(2 pi m / 16), m in [0, 16): the 16th roots of unity (exact decimal expansions of
// cos(pi/8), sin(pi/8) and sqrt(2)/2 rounded to float).
__host__ __device__ constexpr float cos16(int m)
{
    return m == 0    ? 1.0f
           : m == 1  ? 0.923879532511286756f
           : m == 2  ? 0.707106781186547524f
           : m == 3  ? 0.382683432365089772f
           : m == 4  ? 0.0f
           : m == 5  ? -0.382683432365089772f
           : m == 6  ? -0.707106781186547524f
           : m == 7  ? -0.923879532511286756f
           : m == 8  ? -1.0f
           : m == 9  ? -0.923879532511286756f
           : m == 10 ? -0.707106781186547524f
           : m == 11 ? -0.382683432365089772f
           : m == 12 ? 0.0f
           : m == 13 ? 0.382683432365089772f
           : m == 14 ? 0.707106781186547524f
                     : 0.923879532511286756f;
}

// a * exp(SIGN * 2 pi i m / 16) for m known at compile time after unrolling.
template <int SIGN>
__device__ __forceinline__ float2 rot16(float2 a, int m)
{
    m &= 15;
    if (m == 0) return a;
    if (m == 4) return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    if (m == 8) return make_float2(-a.x, -a.y);
    if (m == 12) return SIGN < 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    const float c = cos16(m), s = (SIGN < 0 ? -1.0f : 1.0f) * cos16((m + 12) & 15);
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}

template <int SIGN>
__device__ __forceinline__ void dft2(float2 &a, float2 &b)
{
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

// X[k] = sum_n x[n] exp(SIGN 2 pi i n k / 4)
template <int SIGN>
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3)
{
    float2 a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = csub(x1, x3);
    float2 dw = SIGN < 0 ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);  // d * (SIGN i)
    x0 = cadd(a, c);
    x2 = csub(a, c);
    x1 = cadd(b, dw);
    x3 = csub(b, dw);
}

// In-register DFT of N in {4, 8, 16} points, natural order in and out.
template <int N, int SIGN>
__device__ __forceinline__ void dft_reg(float2 (&x)[N])
{
    if constexpr (N == 4) {
        dft4<SIGN>(x[0], x[1], x[2], x[3]);
    } else if constexpr (N == 8) {
        // n = n2 + 4 n1 (n1 < 2): radix-2 over n1, twiddle W8^{n2 k1}, radix-4 over n2
#pragma unroll
        for (int n2 = 0; n2 < 4; n2++) dft2<SIGN>(x[n2], x[n2 + 4]);
#pragma unroll
        for (int n2 = 1; n2 < 4; n2++) x[n2 + 4] = rot16<SIGN>(x[n2 + 4], 2 * n2);
        dft4<SIGN>(x[0], x[1], x[2], x[3]);
        dft4<SIGN>(x[4], x[5], x[6], x[7]);
        // slot k2 + 4 k1 holds X[k1 + 2 k2]
        float2 y[8];
#pragma unroll
        for (int k1 = 0; k1 < 2; k1++)
#pragma unroll
            for (int k2 = 0; k2 < 4; k2++) y[k1 + 2 * k2] = x[k2 + 4 * k1];
#pragma unroll
        for (int i = 0; i < 8; i++) x[i] = y[i];
    } else if constexpr (N == 16) {
        // n = n2 + 4 n1: radix-4 over n1, twiddle W16^{n2 k1}, radix-4 over n2
#pragma unroll
        for (int n2 = 0; n2 < 4; n2++) dft4<SIGN>(x[n2], x[n2 + 4], x[n2 + 8], x[n2 + 12]);
#pragma unroll
        for (int k1 = 1; k1 < 4; k1++)
#pragma unroll
            for (int n2 = 1; n2 < 4; n2++) x[n2 + 4 * k1] = rot16<SIGN>(x[n2 + 4 * k1], n2 * k1);
#pragma unroll
        for (int k1 = 0; k1 < 4; k1++) dft4<SIGN>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
        float2 y[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; k1++)
#pragma unroll
            for (int k2 = 0; k2 < 4; k2++) y[k1 + 4 * k2] = x[k2 + 4 * k1];
#pragma unroll
        for (int i = 0; i < 16; i++) x[i] = y[i];
    }
}

// Slot order of one transform of length P.
template <int P>
struct Tile {
    static constexpr int R1 = 16;
    static constexpr int R2 = P / 16;
    static constexpr int LD = P + 1;  // row stride of the single-CTA tile (R = P)
    static constexpr int ELEMS = P * LD;
    // natural frequency held by slot q after a forward transform
    static __device__ __forceinline__ int nat(int q) { return q / R2 + R1 * (q % R2); }
    // slot holding natural frequency k
    static __device__ __forceinline__ int slot(int k) { return k / R1 + R2 * (k % R1); }
};

// Geometry of the slab decomposition: CS = P / R CTAs per pattern.
template <int P, int R>
struct Slab {
    static_assert(P % R == 0, "R must divide P");
    static constexpr int CS = P / R;
    static constexpr int LDA = P + 1;  // row slab: R rows x P columns
    static constexpr int LDB = R + 1;  // column slab: P rows x R columns
    static constexpr int ELEMS = (R * LDA > P * LDB) ? R * LDA : P * LDB;
    static constexpr int PER_CTA = P * R;  // values owned by one CTA
};

// Stride pass over NLINES lines of length P; element e of line l at buf[l * LS + e * ES].
template <int P, int NT, int NLINES, int LS, int ES, int SIGN>
__device__ __forceinline__ void pass_stride(float2 *buf, const float2 *tw)
{
    constexpr int R1 = Tile<P>::R1, R2 = Tile<P>::R2;
    for (int t = threadIdx.x; t < NLINES * R2; t += NT) {
        const int line = t % NLINES, n2 = t / NLINES;
        float2 *b = buf + line * LS + n2 * ES;
        float2 x[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; n1++) x[n1] = b[(R2 * n1) * ES];
        if constexpr (SIGN < 0) {
            dft_reg<R1, -1>(x);
#pragma unroll
            for (int k1 = 1; k1 < R1; k1++) x[k1] = cmul(x[k1], tw[(n2 * k1) & (P - 1)]);
        } else {
#pragma unroll
            for (int k1 = 1; k1 < R1; k1++) x[k1] = cmulc(x[k1], tw[(n2 * k1) & (P - 1)]);
            dft_reg<R1, +1>(x);
        }
#pragma unroll
        for (int n1 = 0; n1 < R1; n1++) b[(R2 * n1) * ES] = x[n1];
    }
}

// Block pass (either direction) over NLINES lines.
template <int P, int NT, int NLINES, int LS, int ES, int SIGN>
__device__ __forceinline__ void pass_block(float2 *buf)
{
    constexpr int R1 = Tile<P>::R1, R2 = Tile<P>::R2;
    for (int t = threadIdx.x; t < NLINES * R1; t += NT) {
        const int line = t % NLINES, k1 = t / NLINES;
        float2 *b = buf + line * LS + (R2 * k1) * ES;
        float2 x[R2];
#pragma unroll
        for (int j = 0; j < R2; j++) x[j] = b[j * ES];
        dft_reg<R2, SIGN>(x);
#pragma unroll
        for (int j = 0; j < R2; j++) b[j * ES] = x[j];
    }
}

// Row passes over the R rows of a row slab; caller syncs before; ends with a barrier.
template <int P, int R, int NT, int SIGN>
__device__ __forceinline__ void rows_fft(float2 *buf, const float2 *tw)
{
    constexpr int LDA = Slab<P, R>::LDA;
    if constexpr (SIGN < 0) {
        pass_stride<P, NT, R, LDA, 1, -1>(buf, tw);
        __syncthreads();
        pass_block<P, NT, R, LDA, 1, -1>(buf);
    } else {
        pass_block<P, NT, R, LDA, 1, +1>(buf);
        __syncthreads();
        pass_stride<P, NT, R, LDA, 1, +1>(buf, tw);
    }
    __syncthreads();
}

// Warp groups of the single-CTA 128 x 128 tile with 1024 threads.  Both column passes give
// thread t the column t % 128, so the 8 warps w with w % 4 = g own the columns 32 g .. + 31
// in both; the row stride step (row_item) gives warp w rows of the block 32 (w / 8) .. + 31,
// and pass_block_rows_grouped keeps that block.  Between the two passes of one dimension only
// the 8 warps of a group exchange values, so they meet at a named barrier of 256 threads
// (ids 1 .. 4) and the groups drift apart; the change of dimension keeps the full barrier.
// Used by the inverse transform (the GRAD pass); in the forward transform of the LS pass the
// full barriers measured faster.
template <int P, int R, int NT>
__device__ __forceinline__ constexpr bool grouped_tile()
{
    return P == 128 && R == P && NT == 1024;
}


__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 256;" ::"r"(g + 1) : "memory"); }
__device__ __forceinline__ void col_group_sync() { group_sync((threadIdx.x >> 5) & 3); }
__device__ __forceinline__ void row_group_sync() { group_sync(threadIdx.x >> 8); }

// Block pass over the rows of a single-CTA 128 x 128 tile (row stride P + 1), warp w taking
// rows 32 (w / 8) + lane and k1 = w % 8 + 8 ii: the rows of its row-step group.  Lanes read
// 32 consecutive rows at one column: no bank conflicts.
template <int P, int NT, int SIGN>
__device__ __forceinline__ void pass_block_rows_grouped(float2 *buf)
{
    constexpr int R2 = Tile<P>::R2, LDA = P + 1;
    static_assert(grouped_tile<P, P, NT>(), "128 x 128 tile, 1024 threads");
    const int w = threadIdx.x >> 5, row = 32 * (w >> 3) + (threadIdx.x & 31);
#pragma unroll 1
    for (int ii = 0; ii < 2; ii++) {
        float2 *b = buf + row * LDA + R2 * ((w & 7) + 8 * ii);
        float2 x[R2];
#pragma unroll
        for (int j = 0; j < R2; j++) x[j] = b[j];
        dft_reg<R2, SIGN>(x);
#pragma unroll
        for (int j = 0; j < R2; j++) b[j] = x[j];
    }
}

// Column passes over the R columns of a column slab; caller syncs before; ends with a barrier.
template <int P, int R, int NT, int SIGN>
__device__ __forceinline__ void cols_fft(float2 *buf, const float2 *tw)
{
    constexpr int LDB = Slab<P, R>::LDB;
    if constexpr (SIGN < 0) {
        pass_stride<P, NT, R, 1, LDB, -1>(buf, tw);
        __syncthreads();
        pass_block<P, NT, R, 1, LDB, -1>(buf);
    } else {
        pass_block<P, NT, R, 1, LDB, +1>(buf);
        if constexpr (grouped_tile<P, R, NT>()) col_group_sync();
        else __syncthreads();
        pass_stride<P, NT, R, 1, LDB, +1>(buf, tw);
    }
    __syncthreads();
}

// Items per thread of a single-CTA block pass over the P columns (P * R1 items).
template <int P, int NT>
constexpr int block_items()
{
    return P * Tile<P>::R1 / NT;
}

// The column block pass of the inverse transform of a single-CTA tile whose slots outside a
// mask hold no value (their contents are ignored and read as zero): mw[q] holds, from bit
// 0, the mask bits of the R2 elements of the thread's q-th item (column t % P, rows R2 k1 ..
// R2 k1 + R2 - 1, k1 = t / P, t = threadIdx.x + q NT).  The same results as zeroing those
// slots first.
template <int P, int NT>
__device__ __forceinline__ void pass_block_cols_masked(float2 *buf, const unsigned (&mw)[block_items<P, NT>()])
{
    constexpr int R2 = Tile<P>::R2, LDB = P + 1;
#pragma unroll
    for (int q = 0; q < block_items<P, NT>(); q++) {
        const int t = threadIdx.x + q * NT, line = t % P, k1 = t / P;
        float2 *b = buf + line + (R2 * k1) * LDB;
        float2 x[R2];
#pragma unroll
        for (int j = 0; j < R2; j++) x[j] = (mw[q] >> j) & 1u ? b[j * LDB] : make_float2(0.f, 0.f);
        dft_reg<R2, +1>(x);
#pragma unroll
        for (int j = 0; j < R2; j++) b[j * LDB] = x[j];
    }
}

// Row slab -> column slab across the cluster (all CTAs of the cluster call it).
// Every value is read into registers, the cluster synchronises (all reads done, the
// buffers are free), every value is stored into its owner's buffer, the cluster
// synchronises again (all stores visible).
template <int P, int R, int NT>
__device__ __forceinline__ void exchange_to_cols(float2 *buf)
{
    if constexpr (P != R) {
        namespace cg = cooperative_groups;
        constexpr int LDA = Slab<P, R>::LDA, LDB = Slab<P, R>::LDB, N = P * R / NT;
        cg::cluster_group cl = cg::this_cluster();
        const int c = (int)cl.block_rank();
        float2 v[N];
#pragma unroll
        for (int k = 0; k < N; k++) {
            const int j = threadIdx.x + NT * k, rl = j / P, qx = j % P;
            v[k] = buf[rl * LDA + qx];
        }
        cl.sync();
#pragma unroll
        for (int k = 0; k < N; k++) {
            const int j = threadIdx.x + NT * k, rl = j / P, qx = j % P;
            float2 *dst = cl.map_shared_rank(buf, qx / R);
            dst[(c * R + rl) * LDB + (qx % R)] = v[k];
        }
        cl.sync();
    }
}

// Column slab -> row slab across the cluster.
template <int P, int R, int NT>
__device__ __forceinline__ void exchange_to_rows(float2 *buf)
{
    if constexpr (P != R) {
        namespace cg = cooperative_groups;
        constexpr int LDA = Slab<P, R>::LDA, LDB = Slab<P, R>::LDB, N = P * R / NT;
        cg::cluster_group cl = cg::this_cluster();
        const int c = (int)cl.block_rank();
        float2 v[N];
#pragma unroll
        for (int k = 0; k < N; k++) {
            const int j = threadIdx.x + NT * k, r = j / R, xl = j % R;
            v[k] = buf[r * LDB + xl];
        }
        cl.sync();
#pragma unroll
        for (int k = 0; k < N; k++) {
            const int j = threadIdx.x + NT * k, r = j / R, xl = j % R;
            float2 *dst = cl.map_shared_rank(buf, r / R);
            dst[(r % R) * LDA + (c * R + xl)] = v[k];
        }
        cl.sync();
    }
}

// Unnormalised forward 2-D DFT: natural order in (row slab), permuted order out (column slab).
template <int P, int R, int NT>
__device__ __forceinline__ void fft2_fwd(float2 *buf, const float2 *tw)
{
    rows_fft<P, R, NT, -1>(buf, tw);
    exchange_to_cols<P, R, NT>(buf);
    cols_fft<P, R, NT, -1>(buf, tw);
}

// Unnormalised inverse 2-D DFT: permuted order in (column slab), natural order out (row slab).
template <int P, int R, int NT>
__device__ __forceinline__ void fft2_inv(float2 *buf, const float2 *tw)
{
    cols_fft<P, R, NT, +1>(buf, tw);
    exchange_to_rows<P, R, NT>(buf);
    rows_fft<P, R, NT, +1>(buf, tw);
}

// ---------------------------------------------------------------------------------------
// Single-CTA transforms whose row stride step exchanges with registers (R = P): the forward
// transform's first step takes the exit wave from a loader, the inverse transform's last step
// hands its natural-order rows to a storer, so neither the gather nor the adjoint's emit
// makes a pass of its own through shared memory.
//
// Work item (row, n2) of a row stride step: 16 elements n2 + R2 n1 of one row.  Warp item vw
// holds the rows b + R2 j (j < 32 / R2), b = vw % R2 + 32 (vw / R2), lane l the row
// b + R2 (l / R2) and n2 = l % R2: with the tile's row stride P + 1 the 16 lanes of a
// half-warp touch 16 distinct bank pairs, and a global access of a warp covers 32 / R2 runs
// of R2 consecutive complex values.  A thread's items are vw = warp + ii NT / 32.
template <int P>
__device__ __forceinline__ void row_item(int vw, int lane, int &row, int &n2)
{
    constexpr int R2 = Tile<P>::R2;
    row = (vw % R2) + 32 * (vw / R2) + R2 * (lane / R2);
    n2 = lane % R2;
}

// Twiddles of the row stride step in item order: tw2[k1 R2 + n2] = W_P^(n2 k1) (lanes of a
// warp read consecutive entries).
template <int P, int NT>
__device__ __forceinline__ void load_row_twiddles(float2 *tw2, const float2 *__restrict__ g_tw)
{
    constexpr int R2 = Tile<P>::R2;
    for (int m = threadIdx.x; m < 16 * R2; m += NT) tw2[m] = g_tw[((m % R2) * (m / R2)) & (P - 1)];
}

// Forward: ld(ii, row, n2, x) fills x[n1] = the exit wave at (row, n2 + R2 n1); the tile
// then holds what pass_stride<-1> over the rows would have written.
template <int P, int NT, typename LD>
__device__ __forceinline__ void rows_stride_fwd_in(float2 *buf, const float2 *tw2, LD ld)
{
    constexpr int R1 = Tile<P>::R1, R2 = Tile<P>::R2, LDA = P + 1, NVW = P * R2 / 32;
    static_assert(NVW % (NT / 32) == 0, "whole items per thread");
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int ii = 0; ii < NVW / (NT / 32); ii++) {
        int row, n2;
        row_item<P>((threadIdx.x >> 5) + ii * (NT / 32), lane, row, n2);
        float2 x[R1];
        ld(ii, row, n2, x);
        dft_reg<R1, -1>(x);
#pragma unroll
        for (int k1 = 1; k1 < R1; k1++) x[k1] = cmul(x[k1], tw2[k1 * R2 + n2]);
        float2 *b = buf + row * LDA + n2;
#pragma unroll
        for (int n1 = 0; n1 < R1; n1++) b[R2 * n1] = x[n1];
    }
}

// Inverse, the last step: reads what pass_stride<+1> over the rows would read and hands
// st(ii, row, n2, x) the results x[n1] = row element n2 + R2 n1 (natural order).
template <int P, int NT, typename ST>
__device__ __forceinline__ void rows_stride_inv_out(const float2 *buf, const float2 *tw2, ST st)
{
    constexpr int R1 = Tile<P>::R1, R2 = Tile<P>::R2, LDA = P + 1, NVW = P * R2 / 32;
    static_assert(NVW % (NT / 32) == 0, "whole items per thread");
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int ii = 0; ii < NVW / (NT / 32); ii++) {
        int row, n2;
        row_item<P>((threadIdx.x >> 5) + ii * (NT / 32), lane, row, n2);
        const float2 *b = buf + row * LDA + n2;
        float2 x[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; n1++) x[n1] = b[R2 * n1];
#pragma unroll
        for (int k1 = 1; k1 < R1; k1++) x[k1] = cmulc(x[k1], tw2[k1 * R2 + n2]);
        dft_reg<R1, +1>(x);
        st(ii, row, n2, x);
    }
}

// Unnormalised forward 2-D DFT of one tile, the first step from ld (see rows_stride_fwd_in);
// permuted order out, ends with a barrier.  The caller has synchronised buf's earlier use.
template <int P, int NT, typename LD>
__device__ __forceinline__ void fft2_fwd_in(float2 *buf, const float2 *tw, const float2 *tw2, LD ld)
{
    rows_stride_fwd_in<P, NT>(buf, tw2, ld);
    __syncthreads();
    pass_block<P, NT, P, P + 1, 1, -1>(buf);
    __syncthreads();
    cols_fft<P, P, NT, -1>(buf, tw);
}

// Unnormalised inverse 2-D DFT of one tile (permuted order in), the natural-order rows of
// the result handed to st (see rows_stride_inv_out).  No barrier at the end.  With mw, only
// the masked slots of the input are read (pass_block_cols_masked).
template <int P, int NT, typename ST>
__device__ __forceinline__ void fft2_inv_out(float2 *buf, const float2 *tw, const float2 *tw2, ST st,
                                             const unsigned (*mw)[block_items<P, NT>()] = nullptr)
{
    if (mw) {
        pass_block_cols_masked<P, NT>(buf, *mw);
        if constexpr (grouped_tile<P, P, NT>()) col_group_sync();
        else __syncthreads();
        pass_stride<P, NT, P, 1, P + 1, +1>(buf, tw);
        __syncthreads();
    } else {
        cols_fft<P, P, NT, +1>(buf, tw);
    }
    if constexpr (grouped_tile<P, P, NT>()) {
        pass_block_rows_grouped<P, NT, +1>(buf);
        row_group_sync();
    } else {
        pass_block<P, NT, P, P + 1, 1, +1>(buf);
        __syncthreads();
    }
    rows_stride_inv_out<P, NT>(buf, tw2, st);
}

// Single-CTA forms (R = P), kept for callers that hold the whole tile.
template <int P, int NT>
__device__ __forceinline__ void fft2_fwd(float2 *tile, const float2 *tw)
{
    fft2_fwd<P, P, NT>(tile, tw);
}
template <int P, int NT>
__device__ __forceinline__ void fft2_inv(float2 *tile, const float2 *tw)
{
    fft2_inv<P, P, NT>(tile, tw);
}

}  // namespace pty

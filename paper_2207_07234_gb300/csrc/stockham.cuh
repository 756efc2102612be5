// stockham.cuh -- batched mixed-radix (4, and one 2 when log2 N is odd)
// Stockham FFT in shared memory: natural order in, natural order out, one
// __syncthreads() per stage.  Sequence b of the batch lives at buf + b*N (or
// b*(N + N/4) in the padded layout).  Spans, batch size and block size are
// compile-time constants, so every stage's index arithmetic folds and its loop
// unrolls.
//
// Twiddles come from a staged table (host-built, N entries): the radix-4 stage of
// span p reads tw[(p - P0) + q p + k] = W_N^{(q+1) k N/(4p)} for q = 0, 1, 2 and
// k < p, where W_N = exp(-2 pi i / N) and P0 = 1 when log2 N is even, 2 when it is
// odd (the spans are P0, 4 P0, 16 P0, ...).  Lanes with consecutive k then read
// consecutive words: a linear table W_N^j read at stride N/(4p) would put up to
// sixteen lanes of a warp on one shared-memory bank.
#pragma once

#include "common.cuh"

namespace pdhg {

template <int LOG2N>
struct StageTw {
    static constexpr int P0 = (LOG2N & 1) ? 2 : 1;
    // first entry of the block of span p
    __host__ __device__ static constexpr int off(int p) { return p - P0; }
};

template <bool INV>
__device__ __forceinline__ float2 twmul(float2 x, float2 w) { return INV ? cmulconj(x, w) : cmul(x, w); }

// Shared-memory index with 4 float2 of padding after every 16: for N = 1024 this
// makes every access of the middle radix-4 stages (spans 4, 16, 64) free of bank
// conflicts (the span-4 writes, 64 bytes apart per lane, otherwise hit 4 ways).
__device__ __forceinline__ int padx(int j) { return j + 4 * (j >> 4); }

// Layouts (PAD): 0 plain, sequence stride N; 1 padded within a sequence (padx),
// stride N + N/4; 2 as 1 with stride N + N/4 + 4 -- the extra 4 puts the same
// index of consecutive sequences 4 banks apart, so lanes that read one index of
// 4 sequences (the real-FFT split of 4 rows) do not collide.
template <int PAD>
__device__ __forceinline__ int sidx(int j) { return PAD ? padx(j) : j; }

template <int LOG2N, int PAD>
struct SeqLayout {
    static constexpr int N = 1 << LOG2N;
    static constexpr int PN = PAD == 0 ? N : (PAD == 1 ? N + N / 4 : N + N / 4 + 4);
};

// The radix-2 stage, always first (span 1, so no twiddles): outputs 2i, 2i+1.
template <int LOG2N, int BATCH, int NTHR, int PAD>
__device__ __forceinline__ void stage_r2_first(const float2 *a, float2 *b) {
    constexpr int N = 1 << LOG2N, Q = N >> 1, W = BATCH * Q, ITERS = (W + NTHR - 1) / NTHR;
    constexpr int PN = SeqLayout<LOG2N, PAD>::PN;
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int idx = threadIdx.x + it * NTHR;
        if (W % NTHR != 0 && idx >= W) break;
        const int s = idx >> (LOG2N - 1), i = idx & (Q - 1);
        const float2 *src = a + s * PN;
        float2 *dst = b + s * PN;
        const float2 x0 = src[sidx<PAD>(i)], x1 = src[sidx<PAD>(i + Q)];
        dst[sidx<PAD>(2 * i)] = cadd(x0, x1);
        dst[sidx<PAD>(2 * i + 1)] = csub(x0, x1);
    }
}

// One radix-4 stage with span P (the product of the radices of earlier stages).
template <int LOG2N, bool INV, int P, int BATCH, int NTHR, int PAD>
__device__ __forceinline__ void stage_r4(const float2 *a, float2 *b, const float2 *tw) {
    constexpr int N = 1 << LOG2N, Q = N >> 2, W = BATCH * Q, ITERS = (W + NTHR - 1) / NTHR;
    constexpr int PN = SeqLayout<LOG2N, PAD>::PN;
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int idx = threadIdx.x + it * NTHR;
        if (W % NTHR != 0 && idx >= W) break;
        const int s = idx >> (LOG2N - 2), i = idx & (Q - 1);
        const float2 *src = a + s * PN;
        float2 *dst = b + s * PN;
        const int k = i & (P - 1);
        float2 x0 = src[sidx<PAD>(i)];
        float2 x1 = src[sidx<PAD>(i + Q)], x2 = src[sidx<PAD>(i + 2 * Q)], x3 = src[sidx<PAD>(i + 3 * Q)];
        if (P > 1) {
            const float2 *tp = tw + StageTw<LOG2N>::off(P) + k;
            x1 = twmul<INV>(x1, tp[0]);
            x2 = twmul<INV>(x2, tp[P]);
            x3 = twmul<INV>(x3, tp[2 * P]);
        }
        const float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = csub(x1, x3);
        // forward: y1 = t1 - i t3, y3 = t1 + i t3; inverse: swapped
        const float2 mi = make_float2(t3.y, -t3.x);      // -i * t3
        const float2 y1 = INV ? csub(t1, mi) : cadd(t1, mi);
        const float2 y3 = INV ? cadd(t1, mi) : csub(t1, mi);
        const int j = ((i - k) << 2) + k;
        dst[sidx<PAD>(j)] = cadd(t0, t2);
        dst[sidx<PAD>(j + P)] = y1;
        dst[sidx<PAD>(j + 2 * P)] = csub(t0, t2);
        dst[sidx<PAD>(j + 3 * P)] = y3;
    }
}

// Radix-4 stages with spans PFROM, 4 PFROM, ... below PTO; returns the buffer
// holding the result.  Ends with __syncthreads() (when it runs any stage).
template <int LOG2N, bool INV, int PFROM, int PTO, int BATCH, int NTHR, int PAD>
__device__ __forceinline__ float2 *stockham_r4_range(float2 *a, float2 *b, const float2 *tw) {
    if constexpr (PFROM >= PTO) {
        return a;
    } else {
        stage_r4<LOG2N, INV, PFROM, BATCH, NTHR, PAD>(a, b, tw);
        __syncthreads();
        return stockham_r4_range<LOG2N, INV, PFROM * 4, PTO, BATCH, NTHR, PAD>(b, a, tw);
    }
}

// 4-point DFT of (x0, x1, x2, x3) in registers (forward: W_4 = -i).
template <bool INV>
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
    const float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = csub(x1, x3);
    const float2 mi = make_float2(t3.y, -t3.x);
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = INV ? csub(t1, mi) : cadd(t1, mi);
    x3 = INV ? cadd(t1, mi) : csub(t1, mi);
}

// Full transform of BATCH sequences by NTHR threads; data starts in a, b is
// scratch; returns the buffer holding the result.  Ends with __syncthreads().
template <int LOG2N, bool INV, int BATCH, int NTHR, int PAD = 0>
__device__ __forceinline__ float2 *stockham(float2 *a, float2 *b, const float2 *tw) {
    if constexpr (LOG2N & 1) {
        stage_r2_first<LOG2N, BATCH, NTHR, PAD>(a, b);
        __syncthreads();
        return stockham_r4_range<LOG2N, INV, 2, (1 << LOG2N), BATCH, NTHR, PAD>(b, a, tw);
    } else {
        return stockham_r4_range<LOG2N, INV, 1, (1 << LOG2N), BATCH, NTHR, PAD>(a, b, tw);
    }
}

}  // namespace pdhg

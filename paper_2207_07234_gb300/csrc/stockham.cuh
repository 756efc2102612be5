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

// ---------------------------------------------------------------------------
// Radix-8 Stockham: one leading radix-2 or radix-4 stage when log2 N is not a
// multiple of 3, then radix-8 stages of span P0, 8 P0, ... (P0 = 2^(log2 N mod 3)),
// so 512 points take 3 shared-memory passes instead of 5.
//
// Twiddles (host-built, N entries): the radix-8 stage of span p reads
// tw8[(p - P0) + (q - 1) p + k] = W_N^{q k N/(8p)} for q = 1..7, k < p.
//
// Layout: sequence stride N + N/8 + 4; inside a sequence, element j of the buffer
// written by a stage sits at j + c (j >> 4), with c = 1 after a span-1 stage, 2
// after a span-2..8 stage and 0 after the last stage (span >= 16).  The writes of
// span-1 stages (stride 8 or 4 or 2 per lane) and of span-2..8 stages (groups of
// lanes 16..64 elements apart) then hit 16 distinct banks per 16 lanes, and the
// reads (consecutive lanes at offsets that are multiples of 16) stay contiguous.
// Input and output use c = 0.
// ---------------------------------------------------------------------------
template <int LOG2N>
struct R8 {
    static constexpr int N = 1 << LOG2N;
    static constexpr int R0 = LOG2N % 3;              // leading radix 2^R0 (none when 0)
    static constexpr int P0 = 1 << R0;                // span of the first radix-8 stage
    static constexpr int PN = N + N / 8 + 4;          // sequence stride
};

template <int C>
__device__ __forceinline__ int padc(int j) { return C ? j + C * (j >> 4) : j; }

// 8-point DFT in registers (forward: W_8 = exp(-i pi/4)), natural order in and out:
// two 4-point DFTs of the even and odd inputs, combined with W_8^r.
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
    dft4<INV>(x[0], x[2], x[4], x[6]);        // E_r -> x[2r]
    dft4<INV>(x[1], x[3], x[5], x[7]);        // O_r -> x[2r+1]
    constexpr float h = 0.70710678118654752f;
    const float2 o1 = x[3], o2 = x[5], o3 = x[7];
    float2 t1, t2, t3;                         // W_8^{+-r} O_r
    if (!INV) {
        t1 = make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
        t2 = make_float2(o2.y, -o2.x);
        t3 = make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    } else {
        t1 = make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y));
        t2 = make_float2(-o2.y, o2.x);
        t3 = make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y));
    }
    const float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6], t0 = x[1];
    x[0] = cadd(e0, t0); x[4] = csub(e0, t0);
    x[1] = cadd(e1, t1); x[5] = csub(e1, t1);
    x[2] = cadd(e2, t2); x[6] = csub(e2, t2);
    x[3] = cadd(e3, t3); x[7] = csub(e3, t3);
}

// Leading radix-2^R0 stage (span 1, no twiddles): reads c = 0, writes c = 1.
template <int LOG2N, bool INV, int BATCH, int NTHR>
__device__ __forceinline__ void stage_r8_lead(const float2 *a, float2 *b) {
    constexpr int N = 1 << LOG2N, R = 1 << R8<LOG2N>::R0, Q = N / R, W = BATCH * Q;
    constexpr int ITERS = (W + NTHR - 1) / NTHR, PN = R8<LOG2N>::PN, LQ = LOG2N - R8<LOG2N>::R0;
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int idx = threadIdx.x + it * NTHR;
        if (W % NTHR != 0 && idx >= W) break;
        const int s = idx >> LQ, i = idx & (Q - 1);
        const float2 *src = a + s * PN;
        float2 *dst = b + s * PN;
        if constexpr (R == 2) {
            const float2 x0 = src[i], x1 = src[i + Q];
            dst[padc<1>(2 * i)] = cadd(x0, x1);
            dst[padc<1>(2 * i + 1)] = csub(x0, x1);
        } else {
            float2 x0 = src[i], x1 = src[i + Q], x2 = src[i + 2 * Q], x3 = src[i + 3 * Q];
            dft4<INV>(x0, x1, x2, x3);
            dst[padc<1>(4 * i)] = x0;
            dst[padc<1>(4 * i + 1)] = x1;
            dst[padc<1>(4 * i + 2)] = x2;
            dst[padc<1>(4 * i + 3)] = x3;
        }
    }
}

// One radix-8 stage of span P.  TW0 is the span whose block starts the twiddle
// table (the span of the first radix-8 stage, unless a custom plan says otherwise).
template <int LOG2N, bool INV, int P, int CIN, int COUT, int BATCH, int NTHR, int TW0 = R8<LOG2N>::P0>
__device__ __forceinline__ void stage_r8(const float2 *a, float2 *b, const float2 *tw) {
    constexpr int N = 1 << LOG2N, Q = N >> 3, W = BATCH * Q, ITERS = (W + NTHR - 1) / NTHR;
    constexpr int PN = R8<LOG2N>::PN;
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int idx = threadIdx.x + it * NTHR;
        if (W % NTHR != 0 && idx >= W) break;
        const int s = idx >> (LOG2N - 3), i = idx & (Q - 1);
        const float2 *src = a + s * PN;
        float2 *dst = b + s * PN;
        const int k = i & (P - 1);
        float2 x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = src[padc<CIN>(i + q * Q)];
        if (P > 1) {
            const float2 *tp = tw + (P - TW0) + k;
#pragma unroll
            for (int q = 1; q < 8; ++q) x[q] = twmul<INV>(x[q], tp[(q - 1) * P]);
        }
        dft8<INV>(x);
        const int j = ((i - k) << 3) + k;
#pragma unroll
        for (int r = 0; r < 8; ++r) dst[padc<COUT>(j + r * P)] = x[r];
    }
}

template <int LOG2N, bool INV, int P, int CIN, int BATCH, int NTHR>
__device__ __forceinline__ float2 *stockham8_range(float2 *a, float2 *b, const float2 *tw) {
    if constexpr (P >= (1 << LOG2N)) {
        return a;
    } else {
        constexpr int COUT = 8 * P >= (1 << LOG2N) ? 0 : (P == 1 ? 1 : 2);
        stage_r8<LOG2N, INV, P, CIN, COUT, BATCH, NTHR>(a, b, tw);
        __syncthreads();
        return stockham8_range<LOG2N, INV, 8 * P, COUT, BATCH, NTHR>(b, a, tw);
    }
}

// Full transform of BATCH sequences (stride R8<LOG2N>::PN, c = 0 layout) by NTHR
// threads; data starts in a, b is scratch; returns the buffer holding the result
// (c = 0 layout).  Ends with __syncthreads().
template <int LOG2N, bool INV, int BATCH, int NTHR>
__device__ __forceinline__ float2 *stockham8(float2 *a, float2 *b, const float2 *tw8) {
    if constexpr (R8<LOG2N>::R0 == 0) {
        return stockham8_range<LOG2N, INV, 1, 0, BATCH, NTHR>(a, b, tw8);
    } else {
        stage_r8_lead<LOG2N, INV, BATCH, NTHR>(a, b);
        __syncthreads();
        return stockham8_range<LOG2N, INV, R8<LOG2N>::P0, 1, BATCH, NTHR>(b, a, tw8);
    }
}

}  // namespace pdhg

// stockham.cuh -- batched mixed-radix (4, and one 2 when log2 N is odd)
// Stockham FFT in shared memory: natural order in, natural order out, one
// __syncthreads() per stage.  Sequence b of the batch lives at buf + b*N.
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
    static __device__ __forceinline__ int off(int p) { return p - P0; }
};

template <bool INV>
__device__ __forceinline__ float2 twmul(float2 x, float2 w) { return INV ? cmulconj(x, w) : cmul(x, w); }

// The radix-2 stage, always first (span 1, so no twiddles): outputs 2i, 2i+1.
template <int LOG2N>
__device__ __forceinline__ void stage_r2_first(const float2 *a, float2 *b, int batch) {
    constexpr int N = 1 << LOG2N, Q = N >> 1;
    for (int idx = threadIdx.x; idx < batch * Q; idx += blockDim.x) {
        int s = idx >> (LOG2N - 1), i = idx & (Q - 1);
        const float2 *src = a + s * N;
        float2 *dst = b + s * N;
        float2 x0 = src[i], x1 = src[i + Q];
        dst[2 * i] = cadd(x0, x1);
        dst[2 * i + 1] = csub(x0, x1);
    }
}

// One radix-4 stage with span p.
template <int LOG2N, bool INV>
__device__ __forceinline__ void stage_r4(const float2 *a, float2 *b, int batch, int p, const float2 *tw) {
    constexpr int N = 1 << LOG2N, Q = N >> 2;
    for (int idx = threadIdx.x; idx < batch * Q; idx += blockDim.x) {
        int s = idx >> (LOG2N - 2), i = idx & (Q - 1);
        const float2 *src = a + s * N;
        float2 *dst = b + s * N;
        int k = i & (p - 1);
        float2 x0 = src[i];
        float2 x1 = src[i + Q], x2 = src[i + 2 * Q], x3 = src[i + 3 * Q];
        if (p > 1) {
            const float2 *tp = tw + StageTw<LOG2N>::off(p) + k;
            x1 = twmul<INV>(x1, tp[0]);
            x2 = twmul<INV>(x2, tp[p]);
            x3 = twmul<INV>(x3, tp[2 * p]);
        }
        float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = csub(x1, x3);
        // forward: y1 = t1 - i t3, y3 = t1 + i t3; inverse: swapped
        float2 mi = make_float2(t3.y, -t3.x);      // -i * t3
        float2 y1 = INV ? csub(t1, mi) : cadd(t1, mi);
        float2 y3 = INV ? cadd(t1, mi) : csub(t1, mi);
        int j = ((i - k) << 2) + k;
        dst[j] = cadd(t0, t2);
        dst[j + p] = y1;
        dst[j + 2 * p] = csub(t0, t2);
        dst[j + 3 * p] = y3;
    }
}

// Shared-memory index with 4 float2 of padding after every 16: for N = 1024 this
// makes every access of the middle radix-4 stages (spans 4, 16, 64) free of bank
// conflicts (the span-4 writes, 64 bytes apart per lane, otherwise hit 4 ways).
__device__ __forceinline__ int padx(int j) { return j + 4 * (j >> 4); }

// Radix-4 stage with span p on padded buffers (sequence s at buf + s * padN).
template <int LOG2N, bool INV>
__device__ __forceinline__ void stage_r4_pad(const float2 *a, float2 *b, int batch, int p, const float2 *tw) {
    constexpr int N = 1 << LOG2N, Q = N >> 2, PN = N + N / 4;
    for (int idx = threadIdx.x; idx < batch * Q; idx += blockDim.x) {
        int s = idx >> (LOG2N - 2), i = idx & (Q - 1);
        const float2 *src = a + s * PN;
        float2 *dst = b + s * PN;
        int k = i & (p - 1);
        const float2 *tp = tw + StageTw<LOG2N>::off(p) + k;
        float2 x0 = src[padx(i)];
        float2 x1 = twmul<INV>(src[padx(i + Q)], tp[0]);
        float2 x2 = twmul<INV>(src[padx(i + 2 * Q)], tp[p]);
        float2 x3 = twmul<INV>(src[padx(i + 3 * Q)], tp[2 * p]);
        float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = csub(x1, x3);
        float2 mi = make_float2(t3.y, -t3.x);
        float2 y1 = INV ? csub(t1, mi) : cadd(t1, mi);
        float2 y3 = INV ? cadd(t1, mi) : csub(t1, mi);
        int j = ((i - k) << 2) + k;
        dst[padx(j)] = cadd(t0, t2);
        dst[padx(j + p)] = y1;
        dst[padx(j + 2 * p)] = csub(t0, t2);
        dst[padx(j + 3 * p)] = y3;
    }
}

template <int LOG2N, bool INV>
__device__ float2 *stockham_r4_range_pad(float2 *a, float2 *b, int batch, const float2 *tw, int p_from, int p_to) {
    for (int p = p_from; p < p_to; p <<= 2) {
        stage_r4_pad<LOG2N, INV>(a, b, batch, p, tw);
        __syncthreads();
        float2 *t = a; a = b; b = t;
    }
    return a;
}

// Radix-4 stages with span p in [p_from, p_to) only (p_from a power of 4 times the
// first span); returns the buffer holding the result.  Ends with __syncthreads().
template <int LOG2N, bool INV>
__device__ float2 *stockham_r4_range(float2 *a, float2 *b, int batch, const float2 *tw, int p_from, int p_to) {
    for (int p = p_from; p < p_to; p <<= 2) {
        stage_r4<LOG2N, INV>(a, b, batch, p, tw);
        __syncthreads();
        float2 *t = a; a = b; b = t;
    }
    return a;
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

// Full transform; data starts in a, b is scratch; returns the buffer holding
// the result.  Ends with __syncthreads().
template <int LOG2N, bool INV>
__device__ float2 *stockham(float2 *a, float2 *b, int batch, const float2 *tw) {
    int p = 1;
    if (LOG2N & 1) {
        stage_r2_first<LOG2N>(a, b, batch);
        __syncthreads();
        float2 *t = a; a = b; b = t;
        p = 2;
    }
    for (; p < (1 << LOG2N); p <<= 2) {
        stage_r4<LOG2N, INV>(a, b, batch, p, tw);
        __syncthreads();
        float2 *t = a; a = b; b = t;
    }
    return a;
}

}  // namespace pdhg

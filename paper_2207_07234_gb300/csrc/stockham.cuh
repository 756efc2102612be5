// stockham.cuh -- batched mixed-radix (4, and one 2 when log2 N is odd)
// Stockham FFT in shared memory: natural order in, natural order out, one
// __syncthreads() per stage.  Sequence b of the batch lives at buf + b*N.
// tw[j] = W_N^j = exp(-2 pi i j / N) for j < N (host-computed table).
#pragma once

#include "common.cuh"

namespace pdhg {

// tw may point to global or shared memory: plain (generic) load.
template <bool INV>
__device__ __forceinline__ float2 twid(const float2 *tw, int j) {
    float2 w = tw[j];
    if (INV) w.y = -w.y;
    return w;
}

// One radix-2 stage with span p (product of the radices of earlier stages).
template <int LOG2N, bool INV>
__device__ __forceinline__ void stage_r2(const float2 *a, float2 *b, int batch, int p, const float2 *tw) {
    constexpr int N = 1 << LOG2N, Q = N >> 1;
    for (int idx = threadIdx.x; idx < batch * Q; idx += blockDim.x) {
        int s = idx >> (LOG2N - 1), i = idx & (Q - 1);
        const float2 *src = a + s * N;
        float2 *dst = b + s * N;
        int k = i & (p - 1);
        float2 x0 = src[i], x1 = cmul(src[i + Q], twid<INV>(tw, k * (N / (2 * p))));
        int j = ((i - k) << 1) + k;
        dst[j] = cadd(x0, x1);
        dst[j + p] = csub(x0, x1);
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
        int st = k * (N / (4 * p));
        float2 x0 = src[i];
        float2 x1 = src[i + Q], x2 = src[i + 2 * Q], x3 = src[i + 3 * Q];
        if (p > 1) {
            x1 = cmul(x1, twid<INV>(tw, st));
            x2 = cmul(x2, twid<INV>(tw, 2 * st));
            x3 = cmul(x3, twid<INV>(tw, 3 * st));
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
        stage_r2<LOG2N, INV>(a, b, batch, 1, tw);
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

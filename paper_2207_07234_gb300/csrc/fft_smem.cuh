// fft_smem.cuh -- block-cooperative radix-2 FFTs in shared memory.
//
// The x-transform of a real line of length N uses a complex FFT of length
// M = N/2 on the packed samples z_n = x_{2n} + i x_{2n+1} and the standard
// even/odd split; the y-transform (2D) is a complex FFT of length ny.  Both
// are unnormalised; the inverse scalings are folded into the dual step.
// Twiddles W_N^k = exp(-2 pi i k / N) come from tables computed on the host
// in double precision.
#pragma once

#include "common.cuh"

namespace pdhg {

__device__ __forceinline__ int bitrev(int i, int log2n) {
    return log2n == 0 ? 0 : (int)(__brev((unsigned)i) >> (32 - log2n));
}

// In-place decimation-in-time radix-2 FFT of `batch` sequences of length
// n = 2^log2n held in shared memory in bit-reversed order.  Element i of
// sequence c lives at z[c*cs + i*is]: contiguous sequences (is = 1) or
// interleaved ones (cs = 1, is = batch; then consecutive threads take consecutive
// sequences at the same element, so a warp's accesses stay contiguous).
// tw[j*tws] = W_n^j (j < n/2); inverse: conjugate twiddles.  Stages run in pairs
// in registers (the elements b, b + hs, b + 2 hs, b + 3 hs of one group through
// stages s and s+1), halving the shared-memory passes and barriers; an odd last
// stage runs alone.  Ends with __syncthreads().
template <typename C>
__device__ void fft_radix2(C *z, int log2n, int batch, int cs, int is, const C *__restrict__ tw,
                           int tws, bool inverse) {
    const bool inter = is != 1;
    const bool pow2b = (batch & (batch - 1)) == 0;
    const int lb = __ffs(batch) - 1;
    // thread index t -> (sequence c, group g) with lq = log2(groups per sequence)
    auto split = [&](int t, int lq, int &c, int &g) {
        if (!inter) {
            c = t >> lq;
            g = t & ((1 << lq) - 1);
        } else if (pow2b) {
            c = t & (batch - 1);
            g = t >> lb;
        } else {
            g = t / batch;
            c = t - g * batch;
        }
    };
    int s = 0;
    for (; s + 1 < log2n; s += 2) {
        const int hs = 1 << s, lq = log2n - 2;
        for (int t = threadIdx.x; t < (batch << lq); t += blockDim.x) {
            int c, g;
            split(t, lq, c, g);
            const int pos = g & (hs - 1);
            const int b = ((g >> s) << (s + 2)) + pos;
            C w1 = tw[(pos << (log2n - s - 1)) * tws];
            C wa = tw[(pos << (log2n - s - 2)) * tws], wb = tw[((pos + hs) << (log2n - s - 2)) * tws];
            if (inverse) { w1.y = -w1.y; wa.y = -wa.y; wb.y = -wb.y; }
            C *zc = z + c * cs;
            const C a0 = zc[b * is], a1 = zc[(b + hs) * is], a2 = zc[(b + 2 * hs) * is], a3 = zc[(b + 3 * hs) * is];
            const C t1 = cmul(w1, a1), t3 = cmul(w1, a3);
            const C c0 = cadd(a0, t1), c1 = csub(a0, t1), c2 = cadd(a2, t3), c3 = csub(a2, t3);
            const C u2 = cmul(wa, c2), u3 = cmul(wb, c3);
            zc[b * is] = cadd(c0, u2);
            zc[(b + 2 * hs) * is] = csub(c0, u2);
            zc[(b + hs) * is] = cadd(c1, u3);
            zc[(b + 3 * hs) * is] = csub(c1, u3);
        }
        __syncthreads();
    }
    if (s < log2n) {
        const int hs = 1 << s, lq = log2n - 1;
        for (int t = threadIdx.x; t < (batch << lq); t += blockDim.x) {
            int c, k;
            split(t, lq, c, k);
            const int pos = k & (hs - 1);
            const int i0 = ((k >> s) << (s + 1)) + pos;
            C w = tw[(pos << (log2n - s - 1)) * tws];
            if (inverse) w.y = -w.y;
            C *zc = z + c * cs;
            const C tb = cmul(w, zc[(i0 + hs) * is]);
            const C ta = zc[i0 * is];
            zc[i0 * is] = cadd(ta, tb);
            zc[(i0 + hs) * is] = csub(ta, tb);
        }
        __syncthreads();
    }
}

// Layout of the Bluestein work buffer (length n = 2^log2n): element p sits at
// p ^ (((p >> 4) ^ (p >> (log2n - 4))) & 15), an XOR within each aligned group of 16
// (no extra memory).  The first term spreads the stride-8 accesses of the first stage
// group over all banks; the second, the top 4 bits of p, spreads the bit-reversed
// accesses (a warp's lanes n/32 apart) of the input scatter and the pointwise pass.  A
// half-warp then meets at most 2 distinct elements per bank where the plain layout
// gave up to 16 (every access pattern enumerated for n = 2^9 .. 2^13).
__device__ __forceinline__ int blu_swz(int p, int log2n) {
    return p ^ (((p >> 4) ^ (p >> (log2n - 4))) & 15);
}

// The same in-place DIT transform for one sequence of length n = 2^log2n, held in
// the swizzled layout of blu_swz, with twiddles grouped by stage: stage s (half-span hs = 2^s) reads tw[(hs - 1) + pos]
// = W_n^{pos n / (2 hs)}, so a warp's lanes read consecutive entries.  Stages run
// in threes: the elements b + j hs (j = 0..7) of one group pass through stage s
// (pairs (j, j+1), j even, twiddle W_{2hs}^pos), stage s+1 (pairs (j, j+2),
// twiddles W_{4hs}^pos for j = 0, 4 and W_{4hs}^{pos+hs} for j = 1, 5) and stage s+2
// (pairs (j, j+4), twiddle W_{8hs}^{pos + j hs}) in registers, which cuts the
// shared-memory passes and barriers to a third; one or two leftover stages run as
// a pair or alone.
template <typename C>
__device__ void fft_radix2_staged(C *z, int log2n, const C *__restrict__ tw, bool inverse) {
    const int n = 1 << log2n;
    int s = 0;
    for (; s + 2 < log2n; s += 3) {
        const int hs = 1 << s;
        for (int g = threadIdx.x; g < (n >> 3); g += blockDim.x) {
            const int pos = g & (hs - 1);
            const int b = ((g >> s) << (s + 3)) + pos;
            C w1 = tw[(hs - 1) + pos], wa = tw[(2 * hs - 1) + pos], wb = tw[(2 * hs - 1) + pos + hs];
            C wc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) wc[j] = tw[(4 * hs - 1) + pos + j * hs];
            if (inverse) {
                w1.y = -w1.y; wa.y = -wa.y; wb.y = -wb.y;
#pragma unroll
                for (int j = 0; j < 4; ++j) wc[j].y = -wc[j].y;
            }
            C a[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = z[blu_swz(b + j * hs, log2n)];
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                const C t = cmul(w1, a[j + 1]);
                a[j + 1] = csub(a[j], t);
                a[j] = cadd(a[j], t);
            }
#pragma unroll
            for (int j0 = 0; j0 < 8; j0 += 4) {
                const C t0 = cmul(wa, a[j0 + 2]), t1 = cmul(wb, a[j0 + 3]);
                a[j0 + 2] = csub(a[j0], t0);
                a[j0] = cadd(a[j0], t0);
                a[j0 + 3] = csub(a[j0 + 1], t1);
                a[j0 + 1] = cadd(a[j0 + 1], t1);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const C t = cmul(wc[j], a[j + 4]);
                a[j + 4] = csub(a[j], t);
                a[j] = cadd(a[j], t);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) z[blu_swz(b + j * hs, log2n)] = a[j];
        }
        __syncthreads();
    }
    if (s + 1 < log2n) {                    // two leftover stages: one pair
        const int hs = 1 << s;
        for (int g = threadIdx.x; g < (n >> 2); g += blockDim.x) {
            const int pos = g & (hs - 1);
            const int b = ((g >> s) << (s + 2)) + pos;
            C w1 = tw[(hs - 1) + pos], wa = tw[(2 * hs - 1) + pos], wb = tw[(2 * hs - 1) + pos + hs];
            if (inverse) { w1.y = -w1.y; wa.y = -wa.y; wb.y = -wb.y; }
            C a0 = z[blu_swz(b, log2n)], a1 = z[blu_swz(b + hs, log2n)], a2 = z[blu_swz(b + 2 * hs, log2n)],
              a3 = z[blu_swz(b + 3 * hs, log2n)];
            const C t1 = cmul(w1, a1), t3 = cmul(w1, a3);
            const C c0 = cadd(a0, t1), c1 = csub(a0, t1), c2 = cadd(a2, t3), c3 = csub(a2, t3);
            const C u2 = cmul(wa, c2), u3 = cmul(wb, c3);
            z[blu_swz(b, log2n)] = cadd(c0, u2);
            z[blu_swz(b + 2 * hs, log2n)] = csub(c0, u2);
            z[blu_swz(b + hs, log2n)] = cadd(c1, u3);
            z[blu_swz(b + 3 * hs, log2n)] = csub(c1, u3);
        }
        __syncthreads();
        s += 2;
    }
    if (s < log2n) {                        // one leftover stage
        const int hs = 1 << s;
        for (int k = threadIdx.x; k < (n >> 1); k += blockDim.x) {
            const int pos = k & (hs - 1);
            const int i0 = ((k >> s) << (s + 1)) + pos;
            C w = tw[(hs - 1) + pos];
            if (inverse) w.y = -w.y;
            const C tb = cmul(w, z[blu_swz(i0 + hs, log2n)]);
            const C ta = z[blu_swz(i0, log2n)];
            z[blu_swz(i0, log2n)] = cadd(ta, tb);
            z[blu_swz(i0 + hs, log2n)] = csub(ta, tb);
        }
        __syncthreads();
    }
}

// Real-FFT split: given Z = FFT_M(z) (natural order, length M) produce
// X_k = E_k + W_N^k O_k for k = 0..M, with E_k = (Z_k + conj Z_{M-k})/2 and
// O_k = (Z_k - conj Z_{M-k})/(2i).  twN[k] = W_N^k, k = 0..M.
template <typename C>
__device__ __forceinline__ C rfft_split_vals(C zk, C zm, int k, const C *__restrict__ twN) {
    C e, a, o;
    e.x = 0.5f * (zk.x + zm.x);
    e.y = 0.5f * (zk.y - zm.y);
    a.x = zk.x - zm.x;
    a.y = zk.y + zm.y;        // a = Z_k - conj(Z_{M-k})
    o.x = 0.5f * a.y;         // a / (2i) = -i a / 2
    o.y = -0.5f * a.x;
    return cadd(e, cmul(twN[k], o));
}

// Both outputs of the pair (k, M-k) from the same two inputs: with t = W_N^k O_k,
// X_k = E_k + t and X_{M-k} = conj(E_k - t) (E_{M-k} = conj E_k, O_{M-k} = conj O_k and
// W_N^{M-k} = -conj W_N^k).  k = 0 gives X_0 and X_M.
template <typename C>
__device__ __forceinline__ void rfft_split_pair(C zk, C zm, C w, C &xk, C &xm) {
    C e, a, o;
    e.x = 0.5f * (zk.x + zm.x);
    e.y = 0.5f * (zk.y - zm.y);
    a.x = zk.x - zm.x;
    a.y = zk.y + zm.y;
    o.x = 0.5f * a.y;
    o.y = -0.5f * a.x;
    const C t = cmul(w, o);
    xk = cadd(e, t);
    xm.x = e.x - t.x;
    xm.y = t.y - e.y;
}

template <typename C>
__device__ __forceinline__ C rfft_split(const C *Z, int M, int k, const C *__restrict__ twN) {
    return rfft_split_vals(Z[k == M ? 0 : k], Z[k == 0 ? 0 : M - k], k, twN);
}

// Inverse split: Z_k = E_k + i O_k for k = 0..M-1, E_k = (X_k + conj X_{M-k})/2,
// O_k = (X_k - conj X_{M-k}) conj(W_N^k) / 2.
template <typename C>
__device__ __forceinline__ C irfft_merge(C xk, C xm, C w) {
    C e, a, o, r;
    e.x = 0.5f * (xk.x + xm.x);
    e.y = 0.5f * (xk.y - xm.y);
    a.x = 0.5f * (xk.x - xm.x);
    a.y = 0.5f * (xk.y + xm.y);
    o = cmulconj(a, w);
    r.x = e.x - o.y;          // e + i o
    r.y = e.y + o.x;
    return r;
}

}  // namespace pdhg

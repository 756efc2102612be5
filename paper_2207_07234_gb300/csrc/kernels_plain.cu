// kernels_plain.cu -- one kernel per stage of Algorithm 1 (Sec. 3.3), for every
// scheme of the library, in float or double.  This is the general path (and
// the float64 comparator): each stage streams the space-time fields through
// HBM once.  The fused path for large 2D problems lives in kernels_fused2d.cu.
//
// Stages of one iteration n:
//   k_primal        u^l <- u^l - tau_u (J(u)^T phit)^l, l >= 1; u^0 row and
//                   lambda, lambdat (Algorithm 1 steps 1 and the lambda update)
//   k_residual_rfft R^l(u^n) and its forward real FFT along x
//   k_fft_y         2D: complex FFT along y (forward, and later inverse)
//   k_tsolve        (T_t + kappa h_t^2) z = r per Fourier mode (Thomas, closed-form pivots;
//                   k_tsolve_rtab: 1D handles with a pivot table, deeper prefetch)
//   k_dual_irfft    inverse FFT along x, phi <- phi + tau_phi z, phit = 2 phi^n - phi^{n-1}
// plus k_check / k_reduce for Res (Eq. 2.12).
#include <algorithm>

#include "plain.h"
#include "fft_smem.cuh"

namespace pdhg {

// ---------------------------------------------------------------------------
// time part of (J^T psi)^l = sum_m coef(m, l) psi^m  (summation by parts, Sec. 3.1)
// psi points at the value of slice 0 for this dof; slice stride S.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T time_T(const Params<T> &P, const T *psi, int64_t S, int l) {
    T t = T(0);
    if (l >= 1) t += coef_new(P, l - 1) * psi[(int64_t)(l - 1) * S];
    if (l <= P.nt - 1) t += coef_cur(P, l) * psi[(int64_t)l * S];
    if (l + 1 <= P.nt - 1) t += coef_old(P, l + 1) * psi[(int64_t)(l + 1) * S];
    return t;
}

// ---------------------------------------------------------------------------
// primal step (Algorithm 1, step 1; linearised at u^{n-1} as in Eq. 2.11)
// ---------------------------------------------------------------------------
// Each kernel body below is a __device__ function of its block coordinates, so
// that the batched path (kernels_batch.cu) runs the same code per instance.
template <typename T>
__device__ __forceinline__ void primal_block(const Params<T> &P, T *__restrict__ u, const T *__restrict__ phit,
                                             T *__restrict__ lam, T *__restrict__ lamt, const T *__restrict__ u0,
                                             int bx, int l) {
    const int64_t S = P.S, nU = (int64_t)(P.nt + 1) * S;
    if (is_dg(P.space)) {
        const int N = P.nx, nm = P.lines;
        const int k = bx * blockDim.x + threadIdx.x;
        if (k >= N) return;
        T c[3] = {0, 0, 0}, g[3] = {0, 0, 0};
        T *ul = u + (int64_t)l * S;
        for (int m = 0; m < nm; ++m) {
            c[m] = ul[m * N + k];
            g[m] = time_T(P, phit + m * N + k, S, l);
        }
        if (l >= 1) {
            const T *ps = phit + (int64_t)(l - 1) * S;
            int km = wrapm(k, N), kp = wrapp(k, N);
            T pl[3] = {0, 0, 0}, pc[3] = {0, 0, 0}, pr[3] = {0, 0, 0}, d[3];
            for (int m = 0; m < nm; ++m) {
                pl[m] = ps[m * N + km]; pc[m] = ps[m * N + k]; pr[m] = ps[m * N + kp];
            }
            dgx_DT(P, c, pl, pc, pr, d);
            for (int m = 0; m < nm; ++m)
                u[dbg_idx(P, (int64_t)l * S + m * N + k, nU, 101)] = c[m] - P.tau_u * (g[m] + d[m]);
        } else if (P.init == INIT_LAMBDA) {
            for (int m = 0; m < nm; ++m) {
                const int64_t i = dbg_idx(P, (int64_t)m * N + k, S, 102);
                T un = c[m] - P.tau_u0 * (P.ht * g[m] + lamt[i]);
                u[i] = un;
                T r0 = un - u0[i];
                T ln = lam[i] + P.tau_lambda * r0;
                lam[i] = ln;
                lamt[i] = ln + P.tau_lambda * r0;
            }
        }
        return;
    }
    const int64_t i = (int64_t)bx * blockDim.x + threadIdx.x;
    if (i >= S) return;
    // one slice < 2^31 dofs: 32-bit division, none in 1D (S == nx)
    const int ii = (int)i, y = P.S == P.nx ? 0 : ii / P.nx, x = ii - y * P.nx;
    T *ul = u + (int64_t)l * S;
    T c = ul[i];
    T g = time_T(P, phit + i, S, l);
    if (l >= 1) {
        const T cl = P.ulin ? P.ulin[(int64_t)l * S + i] : c;     // linearisation point
        g += fd_DT(P, cl, phit + (int64_t)(l - 1) * S, y, x);
        T un = c - P.tau_u * g;
        if (l == P.nt && P.tshift) {          // proximal step of |v - tshift|^2 / h_t
            const T k = T(2) * P.tau_u * P.inv_ht;
            un = (un + k * P.tshift[i]) / (T(1) + k);
        }
        u[dbg_idx(P, (int64_t)l * S + i, nU, 103)] = un;
    } else if (P.init == INIT_LAMBDA) {
        T un = c - P.tau_u0 * (P.ht * g + lamt[i]);
        u[dbg_idx(P, i, nU, 104)] = un;
        T r0 = un - u0[i];
        T ln = lam[i] + P.tau_lambda * r0;
        lam[i] = ln;
        lamt[i] = ln + P.tau_lambda * r0;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_primal(Params<T> P, T *__restrict__ u, const T *__restrict__ phit,
                                                T *__restrict__ lam, T *__restrict__ lamt,
                                                const T *__restrict__ u0) {
    primal_block(P, u, phit, lam, lamt, u0, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// residual R^l(u^n) and forward real FFT along x.  One block per (l, line);
// DG: one block per l holding the three mode planes.
// spec layout: [l][line][kx], kx = 0..nx/2 (complex).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T time_R(const Params<T> &P, const T *u, int64_t S, int l) {
    // time part of R^l at this dof; u points at slice 0 of the dof
    T r = coef_new(P, l) * u[(int64_t)(l + 1) * S] + coef_cur(P, l) * u[(int64_t)l * S];
    if (l >= 1 && P.time == BDF2) r += coef_old(P, l) * u[(int64_t)(l - 1) * S];
    return r;
}

// Bluestein core on z (length L, shared memory, blu_swz layout): on entry
// z[bitrev(n)] = a_n; on exit z_k = L conj((a * b)_k), the circular convolution
// with the chirp filter b, via FFT(a), the product with FFT(b), and a second
// forward FFT of its conjugate.
template <typename T>
__device__ __forceinline__ void bluestein_core(const Params<T> &P, typename Cplx<T>::type *z) {
    typedef typename Cplx<T>::type C;
    const int lgL = P.blu_log2L, L = 1 << lgL;
    const C *tw = (const C *)P.blu_tw, *bh = (const C *)P.blu_b;
    fft_radix2_staged(z, lgL, tw, false);
    for (int i = threadIdx.x; i < L; i += blockDim.x) {       // Y = conj(A B^), bit-reversed in place
        const int j = bitrev(i, lgL);
        if (i > j) continue;
        const int si = blu_swz(i, lgL), sj = blu_swz(j, lgL);
        const C a = cconj(cmul(z[si], bh[i])), b = cconj(cmul(z[sj], bh[j]));
        z[sj] = a;
        z[si] = b;
    }
    __syncthreads();
    fft_radix2_staged(z, lgL, tw, false);
}

template <typename T>
__device__ __forceinline__ void residual_rfft_block(const Params<T> &P, const T *__restrict__ u,
                                                    typename Cplx<T>::type *__restrict__ spec,
                                                    const typename Cplx<T>::type *__restrict__ twx, int line, int l) {
    typedef typename Cplx<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *z = reinterpret_cast<C *>(smem_raw);      // line: row y (FD); 0 for DG
    const int N = P.nx, M = N >> 1;
    const int lg = P.log2m;
    const int64_t S = P.S, nX = (int64_t)P.nt * P.lines * P.nkx;     // spectrum extent (complex)
    T *zr = reinterpret_cast<T *>(z);
    if (is_dg(P.space)) {
        const int nm = P.lines;
        const T *un = u + (int64_t)(l + 1) * S;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            int jm = wrapm(j, N), jp = wrapp(j, N);
            T c[3] = {0, 0, 0}, lft[3] = {0, 0, 0}, rgt[3] = {0, 0, 0}, d[3];
            for (int m = 0; m < nm; ++m) {
                c[m] = un[m * N + j]; lft[m] = un[m * N + jm]; rgt[m] = un[m * N + jp];
            }
            dgx_D(P, c, lft, rgt, d);
            int pos = bitrev(j >> 1, lg) * 2 + (j & 1);
            for (int m = 0; m < nm; ++m) zr[m * N + pos] = d[m] + time_R(P, u + m * N + j, S, l);
        }
        __syncthreads();
        fft_radix2(z, lg, nm, M, 1, twx, 2, false);
        for (int t = threadIdx.x; t < nm * (M + 1); t += blockDim.x) {
            int m = t / (M + 1), k = t - m * (M + 1);
            spec[dbg_idx(P, ((int64_t)l * nm + m) * P.nkx + k, nX, 111)] = rfft_split(z + m * M, M, k, twx);
        }
        return;
    }
    const T *un = u + (int64_t)(l + 1) * S;
    const int64_t row = (int64_t)line * N;
    if (P.blu_log2L) {
        // Two real rows per complex transform: the block of an even slice l takes
        // w_n = R^l_n + i R^{l+1}_n (R^{l+1} = 0 past the last slice); the block of an
        // odd slice has nothing to do.  DFT(w)_k = conj(c_k) (a * b)_k with
        // a_n = w_n conj(c_n); then X_k = (W_k + conj W_{N-k}) / 2 and
        // Y_k = (W_k - conj W_{N-k}) / (2i) are the spectra of the two rows.
        if (l & 1) return;
        const bool two = l + 1 < P.nt;
        const int lgL = P.blu_log2L, L = 1 << lgL;
        const C *cc = (const C *)P.blu_c;
        const T *un2 = u + (int64_t)(l + 2) * S;
        for (int x = threadIdx.x; x < L; x += blockDim.x) {
            C v = mk<C, T>(T(0), T(0));
            if (x < N) {
                const T r = (P.ulin ? fd_D_jvp(P, P.ulin + (int64_t)(l + 1) * S, un, line, x) : fd_D(P, un, line, x)) +
                            time_R(P, u + row + x, S, l);
                T r2 = T(0);
                if (two)
                    r2 = (P.ulin ? fd_D_jvp(P, P.ulin + (int64_t)(l + 2) * S, un2, line, x) : fd_D(P, un2, line, x)) +
                         time_R(P, u + row + x, S, l + 1);
                v = cmulconj(mk<C, T>(r, r2), cc[x]);
            }
            z[blu_swz(bitrev(x, lgL), lgL)] = v;
        }
        __syncthreads();
        bluestein_core(P, z);
        // z_k = L conj((a * b)_k): W_k = conj(c_k z_k) / L
        const int64_t o1 = ((int64_t)l * P.lines + line) * P.nkx, o2 = ((int64_t)(l + 1) * P.lines + line) * P.nkx;
        const T h = T(0.5) / T(L);
        for (int k = threadIdx.x; k < P.nkx; k += blockDim.x) {
            const int km = k == 0 ? 0 : N - k;
            const C wk = cconj(cmul(cc[k], z[blu_swz(k, lgL)])), wm = cmul(cc[km], z[blu_swz(km, lgL)]);     // W_k L, conj(W_{N-k}) L
            spec[dbg_idx(P, o1 + k, nX, 112)] = cscale(cadd(wk, wm), h);
            if (two) {
                const C d = csub(wk, wm);                                      // (W_k - conj W_{N-k}) L
                spec[dbg_idx(P, o2 + k, nX, 113)] = cscale(mk<C, T>(d.y, -d.x), h);   // / (2i)
            }
        }
        return;
    }
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        T r = (P.ulin ? fd_D_jvp(P, P.ulin + (int64_t)(l + 1) * S, un, line, x) : fd_D(P, un, line, x)) +
              time_R(P, u + row + x, S, l);
        zr[bitrev(x >> 1, lg) * 2 + (x & 1)] = r;
    }
    __syncthreads();
    fft_radix2(z, lg, 1, M, 1, twx, 2, false);
    const int64_t o = ((int64_t)l * P.lines + line) * P.nkx;
    for (int k = threadIdx.x; k <= M; k += blockDim.x) spec[dbg_idx(P, o + k, nX, 114)] = rfft_split(z, M, k, twx);
}

template <typename T>
__global__ void __launch_bounds__(256) k_residual_rfft(Params<T> P, const T *__restrict__ u,
                                                       typename Cplx<T>::type *__restrict__ spec,
                                                       const typename Cplx<T>::type *__restrict__ twx) {
    residual_rfft_block(P, u, spec, twx, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// complex FFT along y (2D), in place on spec[l][y][kx], CB columns per block
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fft_y(Params<T> P, typename Cplx<T>::type *__restrict__ spec,
                                               const typename Cplx<T>::type *__restrict__ twy, int CB,
                                               int inverse) {
    typedef typename Cplx<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *z = reinterpret_cast<C *>(smem_raw);
    const int l = blockIdx.y;
    const int k0 = blockIdx.x * CB;
    const int cb = min(CB, P.nkx - k0);
    const int ny = P.ny, lg = P.log2ny;
    C *base = spec + (int64_t)l * ny * P.nkx + k0;
    for (int t = threadIdx.x; t < ny * cb; t += blockDim.x) {
        int y = t / cb, c = t - y * cb;
        z[bitrev(y, lg) * cb + c] = base[(int64_t)y * P.nkx + c];
    }
    __syncthreads();
    fft_radix2(z, lg, cb, 1, cb, twy, 1, inverse != 0);
    const int64_t off = (int64_t)l * ny * P.nkx + k0, nX = (int64_t)P.nt * ny * P.nkx;
    for (int t = threadIdx.x; t < ny * cb; t += blockDim.x) {
        int y = t / cb, c = t - y * cb;
        spec[dbg_idx(P, off + (int64_t)y * P.nkx + c, nX, 121)] = z[y * cb + c];
    }
}

// ---------------------------------------------------------------------------
// tridiagonal solve in t per Fourier mode:  (T_t + s) z = r,  s = kappa h_t^2,
// T_t = tridiag(-1; 1,2,...,2; -1).  With cosh(theta) = 1 + s/2 the LU pivots
// are d_l = cosh((l+3/2) theta) / cosh((l+1/2) theta), so
//   rho_l = 1/d_l = e^{-theta} (1 + w_l) / (1 + q w_l),  w_l = e^{-(2l+1) theta}, q = e^{-2 theta}.
// Forward: y_0 = r_0, y_l = r_l + rho_{l-1} y_{l-1};  backward: z_{nt-1} = rho y,
// z_l = rho_l (y_l + z_{l+1}).  The h_t^2 factor of the right-hand side is
// applied in the dual step.  DG: per kx the 3x3 block K_x = V diag(lam) V^H is
// diagonalised first (theta per eigenvalue), and transformed back at the end.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float expT(float x) { return expf(x); }
__device__ __forceinline__ double expT(double x) { return exp(x); }

// Past x = (2l+1) theta = 17 (float) or 37 (double), w = e^{-x} is below half an ulp
// of 1, so 1 + w and 1 + q w round to 1 and the pivot is exactly e^{-theta}: the same
// value with no exponential and no division (most steps of most modes).
template <typename T> struct RhoCut;
template <> struct RhoCut<float> { static constexpr float x = 17.f; };
template <> struct RhoCut<double> { static constexpr double x = 37.0; };

template <typename T>
__device__ __forceinline__ T rho_of(T theta, T emt, T q, int l) {
    const T x = (T)(2 * l + 1) * theta;
    if (x > RhoCut<T>::x) return emt;
    T w = expT(-x);
    return emt * (T(1) + w) / (T(1) + q * w);
}

// (K + s) z = r along t for one mode with the exact time operator (PDHG_FLAG_EXACT_TIME_PRECOND):
// K + s = L D L^T with the host's factors fac[3][nt][nmodes] at mode id m (1/d_l, e_l =
// L_{l,l-1}, f_l = L_{l,l-2}); forward y_l = r_l - e_l y_{l-1} - f_l y_{l-2} (stored), then
// z_l = y_l / d_l - e_{l+1} z_{l+1} - f_{l+2} z_{l+2}.  s points at slice 0 of the mode, stride st.
// Both sweeps load TU slices (right-hand sides and factors) ahead of the recurrence.
// Debug builds check every access against the spectrum (s = spec + base, nX elements)
// and the factor table (3 nt nmodes).
template <typename T, typename C>
__device__ __forceinline__ void tsolve_exact(const Params<T> &P, C *s, int64_t base, int64_t nX, int64_t st,
                                             const T *__restrict__ fac, int64_t nmodes, int64_t m, int nt) {
    constexpr int TU = 4;
    const int64_t ts = (int64_t)nt * nmodes, nF = 3 * ts;
    auto si = [&](int64_t off, int code) { return dbg_idx(P, base + off, nX, code) - base; };
    auto fi = [&](int64_t off, int code) { return dbg_idx(P, off, nF, code); };
    C y1 = s[si(0, 140)], y2 = mk<C, T>(T(0), T(0));
    int l = 1;
    for (; l < nt; l += TU) {
        const int nb = min(TU, nt - l);
        C r[TU];
        T e[TU], f[TU];
#pragma unroll
        for (int j = 0; j < TU; ++j)
            if (j < nb) {
                r[j] = s[si((int64_t)(l + j) * st, 140)];
                e[j] = fac[fi(ts + (int64_t)(l + j) * nmodes + m, 141)];
                f[j] = fac[fi(2 * ts + (int64_t)(l + j) * nmodes + m, 141)];
            }
#pragma unroll
        for (int j = 0; j < TU; ++j)
            if (j < nb) {
                const C y = csub(r[j], cadd(cscale(y1, e[j]), cscale(y2, f[j])));
                s[si((int64_t)(l + j) * st, 142)] = y;
                y2 = y1;
                y1 = y;
            }
    }
    C z1 = mk<C, T>(T(0), T(0)), z2 = z1;
    for (l = nt - 1; l >= 0; l -= TU) {
        const int nb = min(TU, l + 1);
        C y[TU];
        T d[TU], e1[TU], f2[TU];
#pragma unroll
        for (int j = 0; j < TU; ++j)
            if (j < nb) {
                const int k = l - j;
                y[j] = k == nt - 1 ? y1 : s[si((int64_t)k * st, 140)];
                d[j] = fac[fi((int64_t)k * nmodes + m, 141)];
                e1[j] = k + 1 < nt ? fac[fi(ts + (int64_t)(k + 1) * nmodes + m, 141)] : T(0);
                f2[j] = k + 2 < nt ? fac[fi(2 * ts + (int64_t)(k + 2) * nmodes + m, 141)] : T(0);
            }
#pragma unroll
        for (int j = 0; j < TU; ++j)
            if (j < nb) {
                const C z = csub(cscale(y[j], d[j]), cadd(cscale(z1, e1[j]), cscale(z2, f2[j])));
                s[si((int64_t)(l - j) * st, 142)] = z;
                z2 = z1;
                z1 = z;
            }
    }
}

// TUR: slices in flight per sweep on the pivot-table path (1D finite differences).  The
// batch kernels keep 8 (16 raised the persistent kernel's registers past one block per
// multiprocessor); the single-instance t-solve of a 1D problem, about a thousand mode
// columns on a few multiprocessors and bound by load latency, takes 16.  The arithmetic,
// and so every value, is the same for any depth.
template <typename T, int TUR = 8>
__device__ __forceinline__ void tsolve_block(const Params<T> &P, typename Cplx<T>::type *__restrict__ spec,
                                             const T *__restrict__ theta_tab,
                                             const typename Cplx<T>::type *__restrict__ V, int bx) {
    typedef typename Cplx<T>::type C;
    const int nt = P.nt;
    if (is_dg(P.space)) {
        const int nm = P.lines;
        const int k = bx * blockDim.x + threadIdx.x;
        if (k >= P.nkx) return;
        const int64_t ls = nm * (int64_t)P.nkx;      // slice stride
        C v[9];
        for (int i = 0; i < 9; ++i) v[i] = V[(int64_t)k * 9 + i];   // v[m*3+i] = V_{m,i}
        if (P.tfac) {
            // w = V^H r in place, the exact time operator per eigen-index (mode id k nm + i), z = V w
            for (int l = 0; l < nt; ++l) {
                C r[3], w[3];
                for (int m = 0; m < nm; ++m) r[m] = spec[dbg_idx(P, l * ls + m * P.nkx + k, nt * ls, 143)];
                for (int i = 0; i < nm; ++i) {
                    C acc = mk<C, T>(T(0), T(0));
                    for (int m = 0; m < nm; ++m) acc = cadd(acc, cmulconj(r[m], v[m * 3 + i]));
                    w[i] = acc;
                }
                for (int i = 0; i < nm; ++i) spec[dbg_idx(P, l * ls + i * P.nkx + k, nt * ls, 143)] = w[i];
            }
            for (int i = 0; i < nm; ++i)
                tsolve_exact<T, C>(P, spec + i * P.nkx + k, i * P.nkx + k, nt * ls, ls, P.tfac, (int64_t)P.nkx * nm,
                                   (int64_t)k * nm + i, nt);
            for (int l = 0; l < nt; ++l) {
                C w[3], zz[3];
                for (int i = 0; i < nm; ++i) w[i] = spec[dbg_idx(P, l * ls + i * P.nkx + k, nt * ls, 143)];
                for (int m = 0; m < nm; ++m) {
                    C acc = mk<C, T>(T(0), T(0));
                    for (int i = 0; i < nm; ++i) acc = cadd(acc, cmul(v[m * 3 + i], w[i]));
                    zz[m] = acc;
                }
                for (int m = 0; m < nm; ++m) spec[dbg_idx(P, l * ls + m * P.nkx + k, nt * ls, 143)] = zz[m];
            }
            return;
        }
        T th[3], emt[3], q[3];
        for (int i = 0; i < nm; ++i) {
            th[i] = theta_tab[k * nm + i]; emt[i] = expT(-th[i]); q[i] = emt[i] * emt[i];
        }
        C yv[3];
        for (int l = 0; l < nt; ++l) {
            C r[3], w[3];
            for (int m = 0; m < nm; ++m) r[m] = spec[l * ls + m * P.nkx + k];
            for (int i = 0; i < nm; ++i) {                // w = V^H r
                C acc = mk<C, T>(T(0), T(0));
                for (int m = 0; m < nm; ++m) acc = cadd(acc, cmulconj(r[m], v[m * 3 + i]));
                w[i] = acc;
            }
            for (int i = 0; i < nm; ++i) {
                if (l > 0) w[i] = cadd(w[i], cscale(yv[i], rho_of(th[i], emt[i], q[i], l - 1)));
                yv[i] = w[i];
                spec[dbg_idx(P, l * ls + i * P.nkx + k, nt * ls, 131)] = w[i];
            }
        }
        C zv[3];
        for (int l = nt - 1; l >= 0; --l) {
            C zz[3];
            for (int i = 0; i < nm; ++i) {
                C yl = spec[l * ls + i * P.nkx + k];
                if (l < nt - 1) yl = cadd(yl, zv[i]);
                zv[i] = cscale(yl, rho_of(th[i], emt[i], q[i], l));
            }
            for (int m = 0; m < nm; ++m) {                // z = V w
                C acc = mk<C, T>(T(0), T(0));
                for (int i = 0; i < nm; ++i) acc = cadd(acc, cmul(v[m * 3 + i], zv[i]));
                zz[m] = acc;
            }
            for (int m = 0; m < nm; ++m) spec[dbg_idx(P, l * ls + m * P.nkx + k, nt * ls, 132)] = zz[m];
        }
        return;
    }
    const int64_t modes = (int64_t)P.lines * P.nkx;
    const int64_t col = (int64_t)bx * blockDim.x + threadIdx.x;
    if (col >= modes) return;
    if (P.tfac) {
        tsolve_exact<T, C>(P, spec + col, col, (int64_t)nt * modes, modes, P.tfac, modes, col, nt);
        return;
    }
    if (sizeof(T) == 4 && P.t64) {
        // the recurrence in float64 (PDHG_FLAG_T_SOLVE_FP64): pivots and the running y, z
        // in double; each stored y_l and z_l is rounded to the field's precision once
        const double th = (double)theta_tab[col];
        const double emt = exp(-th), q = emt * emt;
        const int64_t nS = (int64_t)nt * modes;
        auto si = [&](int l) { return dbg_idx(P, col + (int64_t)l * modes, nS, 144); };
        double yr = (double)spec[si(0)].x, yi = (double)spec[si(0)].y;
        for (int l = 1; l < nt; ++l) {
            const C r = spec[si(l)];
            const double rh = rho_of<double>(th, emt, q, l - 1);
            yr = (double)r.x + rh * yr;
            yi = (double)r.y + rh * yi;
            spec[si(l)] = mk<C, T>((T)yr, (T)yi);
        }
        const double rl = rho_of<double>(th, emt, q, nt - 1);
        double zr = rl * yr, zi = rl * yi;
        spec[si(nt - 1)] = mk<C, T>((T)zr, (T)zi);
        for (int l = nt - 2; l >= 0; --l) {
            const C yl = spec[si(l)];
            const double rh = rho_of<double>(th, emt, q, l);
            zr = rh * ((double)yl.x + zr);
            zi = rh * ((double)yl.y + zi);
            spec[si(l)] = mk<C, T>((T)zr, (T)zi);
        }
        return;
    }
    const int64_t nX = (int64_t)nt * modes;
    if (P.rtab) {
        // pivots from the handle's [nt][modes] table (the values rho_of gives), loaded with
        // the right-hand sides, TU slices ahead
        constexpr int TU = TUR;
        const T *rt = P.rtab;
        C y = spec[dbg_idx(P, col, nX, 135)];
        int l = 1;
        for (; l + TU <= nt; l += TU) {
            C r[TU];
            T rh[TU];
#pragma unroll
            for (int j = 0; j < TU; ++j) {
                r[j] = spec[dbg_idx(P, col + (int64_t)(l + j) * modes, nX, 135)];
                rh[j] = rt[dbg_idx(P, col + (int64_t)(l + j - 1) * modes, nX, 136)];
            }
#pragma unroll
            for (int j = 0; j < TU; ++j) {
                y = cadd(r[j], cscale(y, rh[j]));
                spec[dbg_idx(P, col + (int64_t)(l + j) * modes, nX, 135)] = y;
            }
        }
        for (; l < nt; ++l) {
            const int64_t i = dbg_idx(P, col + (int64_t)l * modes, nX, 135);
            y = cadd(spec[i], cscale(y, rt[dbg_idx(P, col + (int64_t)(l - 1) * modes, nX, 136)]));
            spec[i] = y;
        }
        C z = cscale(y, rt[dbg_idx(P, col + (int64_t)(nt - 1) * modes, nX, 136)]);
        spec[dbg_idx(P, col + (int64_t)(nt - 1) * modes, nX, 137)] = z;
        l = nt - 2;
        for (; l - TU + 1 >= 0; l -= TU) {
            C r[TU];
            T rh[TU];
#pragma unroll
            for (int j = 0; j < TU; ++j) {
                r[j] = spec[dbg_idx(P, col + (int64_t)(l - j) * modes, nX, 137)];
                rh[j] = rt[dbg_idx(P, col + (int64_t)(l - j) * modes, nX, 136)];
            }
#pragma unroll
            for (int j = 0; j < TU; ++j) {
                z = cscale(cadd(r[j], z), rh[j]);
                spec[dbg_idx(P, col + (int64_t)(l - j) * modes, nX, 137)] = z;
            }
        }
        for (; l >= 0; --l) {
            const int64_t i = dbg_idx(P, col + (int64_t)l * modes, nX, 137);
            z = cscale(cadd(spec[i], z), rt[dbg_idx(P, col + (int64_t)l * modes, nX, 136)]);
            spec[i] = z;
        }
        return;
    }
    const T th = theta_tab[col];
    const T emt = expT(-th), q = emt * emt;
    // the right-hand sides do not depend on the recurrence: each sweep loads TU slices
    // ahead into registers, so a thread has TU loads in flight instead of one (the sweeps
    // of 1D problems, a few modes per multiprocessor, are bound by that latency)
    constexpr int TU = 8;
    C y = spec[dbg_idx(P, col, nX, 133)];
    int l = 1;
    for (; l + TU <= nt; l += TU) {
        C r[TU];
#pragma unroll
        for (int j = 0; j < TU; ++j) r[j] = spec[dbg_idx(P, col + (int64_t)(l + j) * modes, nX, 133)];
#pragma unroll
        for (int j = 0; j < TU; ++j) {
            y = cadd(r[j], cscale(y, rho_of(th, emt, q, l + j - 1)));
            spec[dbg_idx(P, col + (int64_t)(l + j) * modes, nX, 133)] = y;
        }
    }
    for (; l < nt; ++l) {
        const int64_t i = dbg_idx(P, col + (int64_t)l * modes, nX, 133);
        y = cadd(spec[i], cscale(y, rho_of(th, emt, q, l - 1)));
        spec[i] = y;
    }
    C z = cscale(y, rho_of(th, emt, q, nt - 1));
    spec[dbg_idx(P, col + (int64_t)(nt - 1) * modes, nX, 134)] = z;
    l = nt - 2;
    for (; l - TU + 1 >= 0; l -= TU) {
        C r[TU];
#pragma unroll
        for (int j = 0; j < TU; ++j) r[j] = spec[dbg_idx(P, col + (int64_t)(l - j) * modes, nX, 134)];
#pragma unroll
        for (int j = 0; j < TU; ++j) {
            z = cscale(cadd(r[j], z), rho_of(th, emt, q, l - j));
            spec[dbg_idx(P, col + (int64_t)(l - j) * modes, nX, 134)] = z;
        }
    }
    for (; l >= 0; --l) {
        const int64_t i = dbg_idx(P, col + (int64_t)l * modes, nX, 134);
        z = cscale(cadd(spec[i], z), rho_of(th, emt, q, l));
        spec[i] = z;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rho_table(const T *__restrict__ theta_tab, int64_t modes, int nt,
                                                   T *__restrict__ tab) {
    const int64_t n = (int64_t)nt * modes;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / modes);
        const T th = theta_tab[i - (int64_t)l * modes];
        const T emt = expT(-th), q = emt * emt;
        tab[i] = rho_of(th, emt, q, l);
    }
}

template <typename T>
cudaError_t launch_rho_table(const T *theta, int64_t modes, int nt, T *tab, cudaStream_t s) {
    const int64_t n = (int64_t)nt * modes;
    const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    k_rho_table<T><<<g, 256, 0, s>>>(theta, modes, nt, tab);
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(128) k_tsolve(Params<T> P, typename Cplx<T>::type *__restrict__ spec,
                                                const T *__restrict__ theta_tab,
                                                const typename Cplx<T>::type *__restrict__ V) {
    tsolve_block(P, spec, theta_tab, V, blockIdx.x);
}

// the same for a handle with a pivot table (1D finite differences): 16 slices in flight
template <typename T>
__global__ void __launch_bounds__(128) k_tsolve_rtab(Params<T> P, typename Cplx<T>::type *__restrict__ spec,
                                                     const T *__restrict__ theta_tab,
                                                     const typename Cplx<T>::type *__restrict__ V) {
    tsolve_block<T, 16>(P, spec, theta_tab, V, blockIdx.x);
}

// ---------------------------------------------------------------------------
// inverse real FFT along x + dual step + extrapolation:
//   z = K_d^{-1} R,  phi^n = phi^{n-1} + tau_phi z,  phit = phi^n + tau_phi z
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void dual_irfft_block(const Params<T> &P, const typename Cplx<T>::type *__restrict__ spec,
                                                 T *__restrict__ phi, T *__restrict__ phit,
                                                 const typename Cplx<T>::type *__restrict__ twx, int bx, int l) {
    typedef typename Cplx<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *z = reinterpret_cast<C *>(smem_raw);
    const int N = P.nx, M = N >> 1, lg = P.log2m;
    const int nl = is_dg(P.space) ? P.lines : 1;
    const int line0 = is_dg(P.space) ? 0 : bx;
    if (P.blu_log2L) {
        // Two rows per transform (even slice l with l+1): W = Z^l + i Z^{l+1}, the
        // Hermitian extensions of the two half spectra; IDFT(W) = x^l + i x^{l+1}, and
        // IDFT(W)_n = c_n z_n / (L nx) after the core on a_k = conj(W_k c_k).
        if (l & 1) return;
        const bool two = l + 1 < P.nt;
        const int lgL = P.blu_log2L, L = 1 << lgL;
        const C *cc = (const C *)P.blu_c;
        const C *X = spec + ((int64_t)l * P.lines + line0) * P.nkx;
        const C *Y = spec + ((int64_t)(l + 1) * P.lines + line0) * P.nkx;
        for (int k = threadIdx.x; k < L; k += blockDim.x) {
            C v = mk<C, T>(T(0), T(0));
            if (k < N) {
                const C Zk = k < P.nkx ? X[k] : cconj(X[N - k]);
                C Wk = Zk;
                if (two) {
                    const C Vk = k < P.nkx ? Y[k] : cconj(Y[N - k]);
                    Wk = mk<C, T>(Zk.x - Vk.y, Zk.y + Vk.x);                      // Z + i V
                }
                v = cconj(cmul(Wk, cc[k]));
            }
            z[blu_swz(bitrev(k, lgL), lgL)] = v;
        }
        __syncthreads();
        bluestein_core(P, z);
        const T sc = P.blu_scale / (T(L) * T(N));
        const int64_t off = (int64_t)l * P.S + (int64_t)line0 * N;
        const int64_t nF = (int64_t)P.nt * P.S;
        for (int x = threadIdx.x; x < N; x += blockDim.x) {
            const C w = cmul(cc[x], z[blu_swz(x, lgL)]);
            const T dz = sc * w.x;
            const int64_t i = dbg_idx(P, off + x, nF, 141);
            const T pn = phi[i] + dz;
            phi[i] = pn;
            phit[i] = pn + dz;
            if (two) {
                const T dz2 = sc * w.y;
                const int64_t i2 = dbg_idx(P, off + x + P.S, nF, 142);
                const T pn2 = phi[i2] + dz2;
                phi[i2] = pn2;
                phit[i2] = pn2 + dz2;
            }
        }
        return;
    }
    for (int t = threadIdx.x; t < nl * M; t += blockDim.x) {
        int m = t / M, k = t - m * M;
        const C *X = spec + ((int64_t)l * P.lines + line0 + m) * P.nkx;
        z[m * M + bitrev(k, lg)] = irfft_merge(X[k], X[M - k], twx[k]);
    }
    __syncthreads();
    fft_radix2(z, lg, nl, M, 1, twx, 2, true);
    const T *zr = reinterpret_cast<const T *>(z);
    const int64_t off = (int64_t)l * P.S + (int64_t)line0 * N;
    for (int t = threadIdx.x; t < nl * N; t += blockDim.x) {
        int m = t / N, x = t - m * N;
        T dz = P.dual_scale * zr[m * N + x];
        const int64_t i = dbg_idx(P, off + (int64_t)m * N + x, (int64_t)P.nt * P.S, 143);
        T pn = phi[i] + dz;
        phi[i] = pn;
        phit[i] = pn + dz;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_dual_irfft(Params<T> P, const typename Cplx<T>::type *__restrict__ spec,
                                                    T *__restrict__ phi, T *__restrict__ phit,
                                                    const typename Cplx<T>::type *__restrict__ twx) {
    dual_irfft_block(P, spec, phi, phit, twx, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// float64 state with the preconditioner applied in float32 (the float64 phase of
// the mixed solve; finite differences, x-length a power of two): R^l is formed in
// float64 and rounded to float32 for the x-transform, and the float32 result of
// the inverse transform is added to the float64 phi.  K_d^{-1} only shapes the
// iteration (Sec. 3.3), so the rounding moves the iterates, never the fixed point
// R(u*) = 0: the stopping test on Res (float64) decides as before.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_residual_rfft_p32(Params<double> P, const double *__restrict__ u,
                                                           float2 *__restrict__ spec,
                                                           const float2 *__restrict__ twx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *z = reinterpret_cast<float2 *>(smem_raw);
    float *zr = reinterpret_cast<float *>(z);
    const int line = blockIdx.x, l = blockIdx.y;
    const int N = P.nx, M = N >> 1, lg = P.log2m;
    const int64_t S = P.S;
    const double *un = u + (int64_t)(l + 1) * S;
    const int64_t row = (int64_t)line * N;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        const double r = fd_D(P, un, line, x) + time_R(P, u + row + x, S, l);
        zr[bitrev(x >> 1, lg) * 2 + (x & 1)] = (float)r;
    }
    __syncthreads();
    fft_radix2(z, lg, 1, M, 1, twx, 2, false);
    const int64_t o = ((int64_t)l * P.lines + line) * P.nkx, nX = (int64_t)P.nt * P.lines * P.nkx;
    for (int k = threadIdx.x; k <= M; k += blockDim.x) spec[dbg_idx(P, o + k, nX, 145)] = rfft_split(z, M, k, twx);
}

__global__ void __launch_bounds__(256) k_dual_irfft_p32(Params<double> P, const float2 *__restrict__ spec,
                                                        double *__restrict__ phi, double *__restrict__ phit,
                                                        const float2 *__restrict__ twx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *z = reinterpret_cast<float2 *>(smem_raw);
    const int line = blockIdx.x, l = blockIdx.y;
    const int N = P.nx, M = N >> 1, lg = P.log2m;
    const float2 *X = spec + ((int64_t)l * P.lines + line) * P.nkx;
    for (int k = threadIdx.x; k < M; k += blockDim.x) z[bitrev(k, lg)] = irfft_merge(X[k], X[M - k], twx[k]);
    __syncthreads();
    fft_radix2(z, lg, 1, M, 1, twx, 2, true);
    const float *zr = reinterpret_cast<const float *>(z);
    const int64_t off = (int64_t)l * P.S + (int64_t)line * N;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        const double dz = P.dual_scale * (double)zr[x];
        const int64_t i = dbg_idx(P, off + x, (int64_t)P.nt * P.S, 146);
        const double pn = phi[i] + dz;
        phi[i] = pn;
        phit[i] = pn + dz;
    }
}

// ---------------------------------------------------------------------------
// residual norms (Eq. 2.12): the six sums of common.cuh::block_sum6, per block
// ---------------------------------------------------------------------------
// One thread accumulates many units of one slice (grid-stride over units) into
// acc (type A).  check_block folds float32 partial sums of at most 16 units into
// float64 accumulators (GB300's float64 adds would otherwise bound this kernel), so
// each partial carries a relative rounding error below 16 x 2^-24 ~ 1e-6; float64
// fields accumulate in float64 throughout.
template <typename T, typename A>
__device__ __forceinline__ void check_unit(const Params<T> &P, const T *__restrict__ u, const T *__restrict__ phi,
                                           const T *__restrict__ lam, const T *__restrict__ u0, int l, int64_t unit,
                                           A acc[6]) {
    const int64_t S = P.S;
    if (is_dg(P.space)) {
        const int N = P.nx, nm = P.lines;
        const int k = (int)unit;
        const int km = wrapm(k, N), kp = wrapp(k, N);
        if (l < P.nt) {
            const T *un = u + (int64_t)(l + 1) * S;
            T c[3] = {0, 0, 0}, lf[3] = {0, 0, 0}, rg[3] = {0, 0, 0}, d[3];
            for (int m = 0; m < nm; ++m) { c[m] = un[m * N + k]; lf[m] = un[m * N + km]; rg[m] = un[m * N + kp]; }
            dgx_D(P, c, lf, rg, d);
            for (int m = 0; m < nm; ++m) {
                double r = (double)(d[m] + time_R(P, u + m * N + k, S, l));
                acc[0] += (A)(r * r);
                acc[2] += (A)((double)phi[(int64_t)l * S + m * N + k] * r);
            }
        }
        T c[3] = {0, 0, 0};
        for (int m = 0; m < nm; ++m) c[m] = u[(int64_t)l * S + m * N + k];
        if (l >= 1) {
            const T *ps = phi + (int64_t)(l - 1) * S;
            T pl[3] = {0, 0, 0}, pc[3] = {0, 0, 0}, pr[3] = {0, 0, 0}, d[3];
            for (int m = 0; m < nm; ++m) { pl[m] = ps[m * N + km]; pc[m] = ps[m * N + k]; pr[m] = ps[m * N + kp]; }
            dgx_DT(P, c, pl, pc, pr, d);
            for (int m = 0; m < nm; ++m) {
                double g = (double)(d[m] + time_T(P, phi + m * N + k, S, l));
                acc[1] += (A)(g * g);
            }
        } else {
            for (int m = 0; m < nm; ++m) {
                const double r0 = (double)c[m] - (double)u0[m * N + k];
                acc[3] += (A)(r0 * r0);
                if (P.init == INIT_LAMBDA) {
                    const double g0 = (double)P.ht * (double)time_T(P, phi + m * N + k, S, 0) + (double)lam[m * N + k];
                    acc[4] += (A)(g0 * g0);
                    acc[5] += (A)((double)lam[m * N + k] * r0);
                }
            }
        }
        return;
    }
    const int64_t i = unit;
    // one slice < 2^31 dofs: 32-bit division, none in 1D (S == nx)
    const int ii = (int)i, y = P.S == P.nx ? 0 : ii / P.nx, x = ii - y * P.nx;
    if (l < P.nt) {
        const T *un = u + (int64_t)(l + 1) * S;
        const T d = P.ulin ? fd_D_jvp(P, P.ulin + (int64_t)(l + 1) * S, un, y, x) : fd_D(P, un, y, x);
        const T r = d + time_R(P, u + i, S, l);
        acc[0] += (A)(r * r);
        acc[2] += (A)(phi[(int64_t)l * S + i] * r);
    }
    const T c = u[(int64_t)l * S + i];
    if (l >= 1) {
        const T cl = P.ulin ? P.ulin[(int64_t)l * S + i] : c;
        T g = fd_DT(P, cl, phi + (int64_t)(l - 1) * S, y, x) + time_T(P, phi + i, S, l);
        if (l == P.nt && P.tshift) g += T(2) * (c - P.tshift[i]) * P.inv_ht;
        acc[1] += (A)(g * g);
    } else {
        const double r0 = (double)c - (double)u0[i];
        acc[3] += (A)(r0 * r0);
        if (P.init == INIT_LAMBDA) {
            const double g0 = (double)P.ht * (double)time_T(P, phi + i, S, 0) + (double)lam[i];
            acc[4] += (A)(g0 * g0);
            acc[5] += (A)((double)lam[i] * r0);
        }
    }
}

// block bx of gx for slice row l; partial sums at partials[(l gx + bx) * 6]
template <typename T>
__device__ __forceinline__ void check_block(const Params<T> &P, const T *__restrict__ u, const T *__restrict__ phi,
                                            const T *__restrict__ lam, const T *__restrict__ u0,
                                            double *__restrict__ partials, int bx, int l, int gx) {
    const int64_t units = is_dg(P.space) ? P.nx : P.S;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if constexpr (sizeof(T) == 4) {
        float part[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int cnt = 0;
#pragma unroll 4
        for (int64_t unit = (int64_t)bx * blockDim.x + threadIdx.x; unit < units; unit += (int64_t)gx * blockDim.x) {
            check_unit<T, float>(P, u, phi, lam, u0, l, unit, part);
            if (++cnt == 16) {
                for (int k = 0; k < 6; ++k) { acc[k] += (double)part[k]; part[k] = 0.f; }
                cnt = 0;
            }
        }
        for (int k = 0; k < 6; ++k) acc[k] += (double)part[k];
    } else {
#pragma unroll 4
        for (int64_t unit = (int64_t)bx * blockDim.x + threadIdx.x; unit < units; unit += (int64_t)gx * blockDim.x)
            check_unit<T, double>(P, u, phi, lam, u0, l, unit, acc);
    }
    block_sum6(acc, partials + ((int64_t)l * gx + bx) * 6);
}

template <typename T>
__global__ void __launch_bounds__(256) k_check(Params<T> P, const T *__restrict__ u, const T *__restrict__ phi,
                                               const T *__restrict__ lam, const T *__restrict__ u0,
                                               double *__restrict__ partials) {
    check_block(P, u, phi, lam, u0, partials, blockIdx.x, blockIdx.y, gridDim.x);
}

__global__ void __launch_bounds__(256) k_reduce6(const double *__restrict__ partials, int64_t nblocks,
                                                 double *__restrict__ out) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 6; ++k) acc[k] += partials[b * 6 + k];
    block_sum6(acc, out);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_primal(const Params<T> &P, T *u, const T *phit, T *lam, T *lamt, const T *u0, cudaStream_t s) {
    int64_t units = is_dg(P.space) ? P.nx : P.S;
    dim3 grid((unsigned)((units + 255) / 256), (unsigned)(P.nt + 1));
    k_primal<T><<<grid, 256, 0, s>>>(P, u, phit, lam, lamt, u0);
    return cudaGetLastError();
}

template <typename T>
size_t smem_rows(const Params<T> &P) {
    if (P.blu_log2L) return ((size_t)1 << P.blu_log2L) * sizeof(typename Cplx<T>::type);
    int nl = is_dg(P.space) ? P.lines : 1;
    return (size_t)nl * (P.nx / 2) * sizeof(typename Cplx<T>::type);
}

template <typename T>
cudaError_t launch_residual_rfft(const Params<T> &P, const T *u, void *spec, const void *twx, cudaStream_t s) {
    typedef typename Cplx<T>::type C;
    size_t sm = smem_rows(P);
    int nlines = is_dg(P.space) ? 1 : P.lines;
    dim3 grid((unsigned)nlines, (unsigned)P.nt);
    k_residual_rfft<T><<<grid, 256, sm, s>>>(P, u, (C *)spec, (const C *)twx);
    return cudaGetLastError();
}

template <typename T>
int fft_y_cols(const Params<T> &P) {
    return sizeof(T) == 4 ? 8 : 4;
}

template <typename T>
cudaError_t launch_fft_y(const Params<T> &P, void *spec, const void *twy, int inverse, cudaStream_t s) {
    typedef typename Cplx<T>::type C;
    int CB = fft_y_cols(P);
    size_t sm = (size_t)P.ny * CB * sizeof(C);
    dim3 grid((unsigned)((P.nkx + CB - 1) / CB), (unsigned)P.nt);
    k_fft_y<T><<<grid, 256, sm, s>>>(P, (C *)spec, (const C *)twy, CB, inverse);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tsolve(const Params<T> &P, void *spec, const T *theta, const void *V, cudaStream_t s) {
    typedef typename Cplx<T>::type C;
    int64_t cols = is_dg(P.space) ? P.nkx : (int64_t)P.lines * P.nkx;
    if (P.rtab)
        k_tsolve_rtab<T><<<(unsigned)((cols + 127) / 128), 128, 0, s>>>(P, (C *)spec, theta, (const C *)V);
    else
        k_tsolve<T><<<(unsigned)((cols + 127) / 128), 128, 0, s>>>(P, (C *)spec, theta, (const C *)V);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dual_irfft(const Params<T> &P, const void *spec, T *phi, T *phit, const void *twx, cudaStream_t s) {
    typedef typename Cplx<T>::type C;
    size_t sm = smem_rows(P);
    int nlines = is_dg(P.space) ? 1 : P.lines;
    dim3 grid((unsigned)nlines, (unsigned)P.nt);
    k_dual_irfft<T><<<grid, 256, sm, s>>>(P, (const C *)spec, phi, phit, (const C *)twx);
    return cudaGetLastError();
}

// blocks per slice of the residual check (check_blocks_per_row)
template <typename T>
static int64_t check_grid_x(const Params<T> &P) {
    return check_blocks_per_row(is_dg(P.space) ? P.nx : P.S, P.nt);
}

cudaError_t launch_residual_rfft_p32(const Params<double> &P, const double *u, void *spec, const void *twx32,
                                     cudaStream_t s) {
    const dim3 grid((unsigned)P.lines, (unsigned)P.nt);
    k_residual_rfft_p32<<<grid, 256, (size_t)(P.nx / 2) * sizeof(float2), s>>>(P, u, (float2 *)spec,
                                                                                (const float2 *)twx32);
    return cudaGetLastError();
}

cudaError_t launch_dual_irfft_p32(const Params<double> &P, const void *spec, double *phi, double *phit,
                                  const void *twx32, cudaStream_t s) {
    const dim3 grid((unsigned)P.lines, (unsigned)P.nt);
    k_dual_irfft_p32<<<grid, 256, (size_t)(P.nx / 2) * sizeof(float2), s>>>(P, (const float2 *)spec, phi, phit,
                                                                             (const float2 *)twx32);
    return cudaGetLastError();
}

cudaError_t launch_reduce6(const double *partials, int64_t nblocks, double *out, cudaStream_t s) {
    k_reduce6<<<1, 256, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

template <typename T>
int64_t check_blocks(const Params<T> &P) {
    return check_grid_x(P) * (int64_t)(P.nt + 1);
}

template <typename T>
cudaError_t launch_check(const Params<T> &P, const T *u, const T *phi, const T *lam, const T *u0,
                         double *partials, double *out, cudaStream_t s, int slices) {
    // blocks per slice row: the usual check_grid_x; a launch over fewer rows may use
    // the blocks (and partial records) of the rows it skips
    const int rows = slices > 0 ? slices : P.nt + 1;
    const int64_t units = is_dg(P.space) ? P.nx : P.S;
    const int64_t gx = std::min<int64_t>(check_grid_x(P) * (int64_t)(P.nt + 1) / rows, (units + 255) / 256);
    dim3 grid((unsigned)std::max<int64_t>(gx, check_grid_x(P)), (unsigned)rows);
    k_check<T><<<grid, 256, 0, s>>>(P, u, phi, lam, u0, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce6<<<1, 256, 0, s>>>(partials, (int64_t)grid.x * grid.y, out);
    return cudaGetLastError();
}

// sum_l <phi^l, Lap_h u^{l+1}> in float64 (FD; 2D: both directions).  The viscous
// term of D is -nu Lap_h u, so dR^l/dnu = -Lap_h u^{l+1}.
template <typename T>
__global__ void __launch_bounds__(256) k_phi_lap(Params<T> P, const T *__restrict__ u, const T *__restrict__ phi,
                                                 double *__restrict__ partials) {
    const int l = blockIdx.y;
    const int64_t S = P.S;
    const T *ul = u + (int64_t)(l + 1) * S;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        // one slice < 2^31 dofs: 32-bit division, none in 1D (S == nx)
        const int ii = (int)i, y = P.S == P.nx ? 0 : ii / P.nx, x = ii - y * P.nx;
        const int64_t r = (int64_t)y * P.nx;
        const T c = ul[i];
        T lap = (ul[r + wrapp(x, P.nx)] - T(2) * c + ul[r + wrapm(x, P.nx)]) * P.inv_hx * P.inv_hx;
        if (P.dims == 2)
            lap += (ul[(int64_t)wrapp(y, P.ny) * P.nx + x] - T(2) * c + ul[(int64_t)wrapm(y, P.ny) * P.nx + x]) *
                   P.inv_hy * P.inv_hy;
        acc[0] += (double)phi[(int64_t)l * S + i] * (double)lap;
    }
    block_sum6(acc, partials + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 6);
}

template <typename T>
cudaError_t launch_phi_lap(const Params<T> &P, const T *u, const T *phi, double *partials, double *out,
                           cudaStream_t s) {
    dim3 grid((unsigned)check_grid_x(P), (unsigned)P.nt);
    k_phi_lap<T><<<grid, 256, 0, s>>>(P, u, phi, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce6<<<1, 256, 0, s>>>(partials, (int64_t)grid.x * grid.y, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched launches: many 1D instances per launch.  Every block looks up its
// (instance, block coordinates) in a table and runs the same block function as
// the single-instance kernels above; tables list active instances only,
// largest first.
// ---------------------------------------------------------------------------
// The instance's record (its Params and pointers) copied to shared memory by the block,
// so that the per-block code reads its coefficients there and not through global memory.
template <typename T>
__device__ __forceinline__ const BatchInst<T> &batch_inst_shared(const BatchInst<T> *I, int inst) {
    static_assert(sizeof(BatchInst<T>) % 8 == 0, "8-byte words");
    constexpr int NW = (int)(sizeof(BatchInst<T>) / 8);
    __shared__ uint64_t rec[NW];
    const uint64_t *src = reinterpret_cast<const uint64_t *>(I + inst);
    for (int w = threadIdx.x; w < NW; w += blockDim.x) rec[w] = src[w];
    __syncthreads();
    return *reinterpret_cast<const BatchInst<T> *>(rec);
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_primal(const BatchInst<T> *__restrict__ I, const BatchEntry *__restrict__ tab) {
    const BatchEntry e = tab[blockIdx.x];
    const BatchInst<T> &b = batch_inst_shared(I, e.inst);
    for (int k = 0; k < max(e.pad, 1); ++k) primal_block(b.P, b.u, b.phit, b.lam, b.lamt, b.u0, e.bx, e.l + k);
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_residual_rfft(const BatchInst<T> *__restrict__ I,
                                                         const BatchEntry *__restrict__ tab) {
    typedef typename Cplx<T>::type C;
    const BatchEntry e = tab[blockIdx.x];
    const BatchInst<T> &b = batch_inst_shared(I, e.inst);
    residual_rfft_block(b.P, b.u, (C *)b.spec, (const C *)b.twx, e.bx, e.l);
}

template <typename T>
__global__ void __launch_bounds__(128) k_b_tsolve(const BatchInst<T> *__restrict__ I, const BatchEntry *__restrict__ tab) {
    typedef typename Cplx<T>::type C;
    const BatchEntry e = tab[blockIdx.x];
    const BatchInst<T> &b = batch_inst_shared(I, e.inst);
    tsolve_block(b.P, (C *)b.spec, b.theta, (const C *)b.V, e.bx);
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_dual_irfft(const BatchInst<T> *__restrict__ I,
                                                      const BatchEntry *__restrict__ tab) {
    typedef typename Cplx<T>::type C;
    const BatchEntry e = tab[blockIdx.x];
    const BatchInst<T> &b = batch_inst_shared(I, e.inst);
    dual_irfft_block(b.P, (const C *)b.spec, b.phi, b.phit, (const C *)b.twx, e.bx, e.l);
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_check(const BatchInst<T> *__restrict__ I, const BatchEntry *__restrict__ tab,
                                                 double *__restrict__ partials) {
    const BatchEntry e = tab[blockIdx.x];
    const BatchInst<T> &b = I[e.inst];
    check_block(b.P, b.u, b.phi, b.lam, b.u0, partials + b.part_off * 6, e.bx, e.l, b.gx);
}

// one block per listed instance: the sum of its (nt+1) * gx partial records
template <typename T>
__global__ void __launch_bounds__(256) k_b_reduce(const BatchInst<T> *__restrict__ I, const int32_t *__restrict__ list,
                                                  const double *__restrict__ partials, double *__restrict__ out) {
    const int inst = list[blockIdx.x];
    const BatchInst<T> &b = I[inst];
    const int64_t n = (int64_t)(b.P.nt + 1) * b.gx;
    const double *p = partials + b.part_off * 6;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x)
        for (int j = 0; j < 6; ++j) acc[j] += p[k * 6 + j];
    block_sum6(acc, out + (int64_t)inst * 6);
}

// ---------------------------------------------------------------------------
// One batched iteration in a single persistent launch.  Blocks take work items from
// a queue (atomic counter cnt[0]) in the queue's order: every instance's primal items,
// then its residual + x-FFT rows, its t-solve columns and its inverse x-FFT + dual rows,
// stage after stage, the instances with most cells first within a stage.  An item of
// stage s > 0 starts once all stage s-1 items of its instance are finished (counter
// cnt[1 + 4 inst + s-1] = need[4 inst + s-1]); it only waits on items that earlier
// dequeues have handed to running blocks, and all blocks are resident (cooperative
// launch), so every wait ends.  Each wait is bounded by wait_ns of %globaltimer (0:
// gives up at once); a block that gives up sets *err and leaves, and so do the blocks
// that then wait on it.  A queue entry covers `pad >> 2` consecutive row items (the
// tiles chosen per size class) and stage `pad & 3`.  Completion: every thread fences
// its writes, the block synchronises, one thread counts the item; the waiting thread
// fences after it sees the count, then its block synchronises (the pattern of a grid
// barrier).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t batch_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__global__ void __launch_bounds__(256, 3) k_b_persistent(const BatchInst<T> *__restrict__ I,
                                                      const BatchEntry *__restrict__ q, int64_t nq,
                                                      const int32_t *__restrict__ need, unsigned int *cnt, int *err,
                                                      uint64_t wait_ns) {
    typedef typename Cplx<T>::type C;
    __shared__ int64_t s_item;
    __shared__ int s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(cnt, 1u);
        __syncthreads();
        const int64_t it = s_item;
        if (it >= nq) return;
        const BatchEntry e = q[it];
        const int stage = e.pad & 3, span = max(e.pad >> 2, 1), inst = e.inst;
        if (threadIdx.x == 0) {
            int ok = 1;
            if (stage > 0) {
                const unsigned int target = (unsigned int)need[4 * inst + stage - 1];
                volatile unsigned int *c = cnt + 1 + 4 * inst + stage - 1;
                if (wait_ns == 0) {
                    ok = 0;
                } else if (*c < target) {
                    const uint64_t t0 = batch_ns();
                    while (*c < target)
                        if (batch_ns() - t0 > wait_ns) { ok = 0; break; }
                }
                __threadfence();
            }
            if (!ok) atomicExch(err, 1);
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        const BatchInst<T> &b = batch_inst_shared(I, inst);
        for (int k = 0; k < span; ++k) {
            switch (stage) {
            case 0: primal_block(b.P, b.u, b.phit, b.lam, b.lamt, b.u0, e.bx, e.l + k); break;
            case 1:
                residual_rfft_block(b.P, b.u, (C *)b.spec, (const C *)b.twx, e.bx,
                                    e.l + k * (b.P.blu_log2L ? 2 : 1));
                break;
            case 2: tsolve_block(b.P, (C *)b.spec, b.theta, (const C *)b.V, e.bx + k); break;
            default:
                dual_irfft_block(b.P, (const C *)b.spec, b.phi, b.phit, (const C *)b.twx, e.bx,
                                 e.l + k * (b.P.blu_log2L ? 2 : 1));
                break;
            }
            __syncthreads();
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(cnt + 1 + 4 * inst + stage, 1u);
    }
}

template <typename T>
cudaError_t launch_batch_persistent(const BatchInst<T> *I, const BatchEntry *q, int64_t nq, const int32_t *need,
                                    unsigned int *cnt, int *err, uint64_t wait_ns, int grid, size_t smem,
                                    cudaStream_t s) {
    void *args[] = {(void *)&I, (void *)&q, (void *)&nq, (void *)&need, (void *)&cnt, (void *)&err, (void *)&wait_ns};
    return cudaLaunchCooperativeKernel((const void *)k_b_persistent<T>, dim3((unsigned)grid), dim3(256), args, smem, s);
}

template <typename T>
cudaError_t batch_persistent_occupancy(size_t smem, int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_b_persistent<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_b_persistent<T>, 256, smem);
    return e;
}

template <typename T>
cudaError_t launch_batch(int kind, const BatchInst<T> *I, const BatchEntry *tab, int64_t nblocks, size_t smem,
                         const int32_t *list, double *partials, double *out, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    const unsigned g = (unsigned)nblocks;
    switch (kind) {
    case BATCH_PRIMAL: k_b_primal<T><<<g, 256, 0, s>>>(I, tab); break;
    case BATCH_RESIDUAL: k_b_residual_rfft<T><<<g, 256, smem, s>>>(I, tab); break;
    case BATCH_TSOLVE: k_b_tsolve<T><<<g, 128, 0, s>>>(I, tab); break;
    case BATCH_DUAL: k_b_dual_irfft<T><<<g, 256, smem, s>>>(I, tab); break;
    case BATCH_CHECK: k_b_check<T><<<g, 256, 0, s>>>(I, tab, partials); break;
    case BATCH_REDUCE: k_b_reduce<T><<<g, 256, 0, s>>>(I, list, partials, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t init_plain_attributes() {
    const int mx = 200 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_residual_rfft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft_y<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dual_irfft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_residual_rfft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_b_dual_irfft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
}

#define PDHG_INSTANTIATE(T)                                                                                   \
    template cudaError_t launch_primal<T>(const Params<T> &, T *, const T *, T *, T *, const T *, cudaStream_t); \
    template cudaError_t launch_residual_rfft<T>(const Params<T> &, const T *, void *, const void *, cudaStream_t); \
    template cudaError_t launch_fft_y<T>(const Params<T> &, void *, const void *, int, cudaStream_t);          \
    template cudaError_t launch_tsolve<T>(const Params<T> &, void *, const T *, const void *, cudaStream_t);   \
    template cudaError_t launch_rho_table<T>(const T *, int64_t, int, T *, cudaStream_t);                     \
    template cudaError_t launch_dual_irfft<T>(const Params<T> &, const void *, T *, T *, const void *, cudaStream_t); \
    template int64_t check_blocks<T>(const Params<T> &);                                                      \
    template cudaError_t init_plain_attributes<T>();                                                      \
    template cudaError_t launch_check<T>(const Params<T> &, const T *, const T *, const T *, const T *, double *, \
                                         double *, cudaStream_t, int);                                        \
    template cudaError_t launch_phi_lap<T>(const Params<T> &, const T *, const T *, double *, double *, cudaStream_t); \
    template cudaError_t launch_batch<T>(int, const BatchInst<T> *, const BatchEntry *, int64_t, size_t,        \
                                         const int32_t *, double *, double *, cudaStream_t);                     \
    template cudaError_t launch_batch_persistent<T>(const BatchInst<T> *, const BatchEntry *, int64_t,          \
                                                    const int32_t *, unsigned int *, int *, uint64_t, int, size_t, \
                                                    cudaStream_t);                                              \
    template cudaError_t batch_persistent_occupancy<T>(size_t, int *);

PDHG_INSTANTIATE(float)
PDHG_INSTANTIATE(double)

}  // namespace pdhg

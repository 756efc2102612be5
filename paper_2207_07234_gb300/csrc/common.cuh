// common.cuh -- parameters, complex helpers and the spatial stencils of the
// implicit schemes, shared by every kernel of the library.
//
// Notation follows the paper: u^l is time slice l (l = 0..nt), R^l the
// equation of slice l (l = 0..nt-1, Sec. 3.1), phi^l its multiplier, phit the
// extrapolated multiplier, lambda the multiplier of the initial row (Sec. 3.3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdhg {

enum Space { FD_UPWIND = 0, FD_LF = 1, DG_P2_LF = 2, DG_P1_UPWIND = 3, DG_P1_LF = 4 };
enum Time { BE = 0, BDF2 = 1 };
enum Init { INIT_LAMBDA = 0, INIT_PINNED = 1 };

template <typename T> struct Cplx;
template <> struct Cplx<float> { typedef float2 type; };
template <> struct Cplx<double> { typedef double2 type; };

template <typename C, typename T>
__host__ __device__ __forceinline__ C mk(T re, T im) { C c; c.x = re; c.y = im; return c; }
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C>
__device__ __forceinline__ C cmulconj(C a, C b) {   // a * conj(b)
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename C, typename T>
__device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
template <typename C>
__device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// Everything a kernel needs to evaluate the scheme, passed by value.
template <typename T>
struct Params {
    int32_t dims, space, time, init;
    int32_t nx, ny, nt;     // nx: points (FD) or cells (DG)
    int32_t log2m;          // log2(nx/2): length of the packed complex x-FFT
    int32_t log2ny;         // 2D only
    int64_t S;              // dofs per slice
    int32_t nkx;            // nx/2 + 1
    int32_t lines;          // x-lines per slice: 1 (1D FD), ny (2D), modes per cell (DG: 3 or 2)
    T alpha, beta, nu, lf_a;
    T ht, inv_ht, inv_hx, inv_hy;
    T tau_u, tau_u0, tau_phi, tau_lambda;
    T dual_scale;           // tau_phi * h_t^2 / (nx/2 * ny): folds FFT and Thomas scalings
    const T *gamma_half;    // 1D FD, nullable
    // Bluestein x-transform (1D FD, nx not a power of two): DFT of length nx as a
    // chirp convolution through radix-2 FFTs of length L = 2^blu_log2L >= 2 nx - 1
    int32_t blu_log2L = 0;      // 0: the packed power-of-two transform
    T blu_scale = T(0);         // tau_phi h_t^2 (the Bluestein inverse is normalised)
    const void *blu_tw = nullptr;   // stage-grouped W_L: entry (2^s - 1) + pos = W_L^{pos L / 2^{s+1}}
    const void *blu_c = nullptr;    // chirp c_n = exp(i pi n^2 / nx), n < nx
    const void *blu_b = nullptr;    // FFT_L of b: b_m = c_|m| for |m| < nx (indices mod L), else 0
    // adjoint mode (FD, plain path): the state is a perturbation v of the solution
    // u*, the residual is J(u*) v and the transposes are taken at u*; the last
    // slice carries the objective |v - tshift|^2 (tshift = target - u*^nt).
    const T *ulin = nullptr;     // u*, [nt+1][S]; nullptr: forward mode
    const T *tshift = nullptr;   // [S]; nullptr: no terminal objective
    int *dbg = nullptr;          // debug builds: site code of the first out-of-range index
    // exact time operator (PDHG_FLAG_EXACT_TIME_PRECOND): per mode the LDL^T factors of
    // h_t^2 D_t D_t^T + s as [3][nt][modes] (1/d_l, e_l, f_l); nullptr: T_t (closed form)
    const T *tfac = nullptr;
    // float32 fields with the t-solve recurrence in float64 (PDHG_FLAG_T_SOLVE_FP64)
    int32_t t64 = 0;
    // t-solve pivots rho_l per mode as [nt][modes] (1D finite differences); nullptr: evaluated
    const T *rtab = nullptr;
};

// Debug builds (-DPDHG_DEBUG): the global indices of the instrumented kernels are checked
// against their buffer's extent n; the first violation records its site code in *P.dbg
// (read at the next residual check) and the access goes to element 0 instead, so nothing
// outside the buffer is touched.  Release builds: the index itself.
template <typename T>
__device__ __forceinline__ int64_t dbg_idx(const Params<T> &P, int64_t i, int64_t n, int code) {
#ifdef PDHG_DEBUG
    if (i < 0 || i >= n) {
        if (P.dbg) atomicCAS(P.dbg, 0, code);
        return 0;
    }
#else
    (void)P; (void)n; (void)code;
#endif
    return i;
}

template <typename T>
__device__ __forceinline__ T flux(const Params<T> &P, T v) { return v * (P.alpha * v + P.beta); }
template <typename T>
__device__ __forceinline__ T dflux(const Params<T> &P, T v) { return T(2) * P.alpha * v + P.beta; }

__device__ __forceinline__ int wrapm(int j, int n) { return j == 0 ? n - 1 : j - 1; }
__device__ __forceinline__ int wrapp(int j, int n) { return j == n - 1 ? 0 : j + 1; }

// ---------------------------------------------------------------------------
// Time stencils (Sec. 3.1).  R^m has the time part sum_l coef(m,l) u^l:
//   BE, and BDF2 for m = 0 (a BE start):  u^{m+1}/h_t - u^m/h_t
//   BDF2, m >= 1:  1.5 u^{m+1}/h_t - 2 u^m/h_t + 0.5 u^{m-1}/h_t
// Summation by parts gives the time part of (J^T psi)^l = sum_m coef(m,l) psi^m.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T coef_new(const Params<T> &P, int m) {        // coef(m, m+1)
    return (P.time == BE || m == 0) ? P.inv_ht : T(1.5) * P.inv_ht;
}
template <typename T>
__device__ __forceinline__ T coef_cur(const Params<T> &P, int m) {        // coef(m, m)
    return (P.time == BE || m == 0) ? -P.inv_ht : T(-2) * P.inv_ht;
}
template <typename T>
__device__ __forceinline__ T coef_old(const Params<T> &P, int m) {        // coef(m, m-1)
    return (P.time == BE || m == 0) ? T(0) : T(0.5) * P.inv_ht;
}

// ---------------------------------------------------------------------------
// Finite differences (Sec. 3.2.1, 3.2.2).  Interface flux F_{j+1/2}:
//   upwind: f(v_j);  Lax-Friedrichs: (f(v_j)+f(v_{j+1}))/2 - a/2 (v_{j+1}-v_j).
// D(v)_j = (F_{j+1/2} - F_{j-1/2})/h - nu (v_{j+1}-2v_j+v_{j-1})/h^2 - Lap_gamma(v)_j.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T fd_face(const Params<T> &P, T vl, T vr) {
    if (P.space == FD_UPWIND) return flux(P, vl);
    return T(0.5) * (flux(P, vl) + flux(P, vr)) - T(0.5) * P.lf_a * (vr - vl);
}

// one direction of D at a point: neighbours vm, v, vp; inv_h = 1/h
template <typename T>
__device__ __forceinline__ T fd_dir(const Params<T> &P, T vm, T v, T vp, T inv_h) {
    T out = (fd_face(P, v, vp) - fd_face(P, vm, v)) * inv_h;
    if (P.nu != T(0)) out -= P.nu * (vp - T(2) * v + vm) * inv_h * inv_h;
    return out;
}

// transpose of one direction at a point: u-value v, multipliers pm, p, pp
// g_j = (psi_j - psi_{j+1})/h;  upwind: f'(v) g_j;
// LF: (f'(v)+a)/2 g_j + (f'(v)-a)/2 g_{j-1};  viscous term is symmetric.
template <typename T>
__device__ __forceinline__ T fd_dir_T(const Params<T> &P, T v, T pm, T p, T pp, T inv_h) {
    T g0 = (p - pp) * inv_h;
    T gm = (pm - p) * inv_h;
    T df = dflux(P, v);
    T out;
    if (P.space == FD_UPWIND) out = df * g0;
    else out = T(0.5) * (df + P.lf_a) * g0 + T(0.5) * (df - P.lf_a) * gm;
    if (P.nu != T(0)) out -= P.nu * (pp - T(2) * p + pm) * inv_h * inv_h;
    return out;
}

// variable-coefficient Laplacian term of D (1D): -[g_j (v_{j+1}-v_j) - g_{j-1}(v_j - v_{j-1})]/h^2
template <typename T>
__device__ __forceinline__ T fd_gamma(const Params<T> &P, int j, int jm, T vm, T v, T vp) {
    return -(P.gamma_half[j] * (vp - v) - P.gamma_half[jm] * (v - vm)) * P.inv_hx * P.inv_hx;
}

// D(v) at point (y, x) of a slice v (1D: y = 0)
template <typename T>
__device__ __forceinline__ T fd_D(const Params<T> &P, const T *__restrict__ v, int y, int x) {
    const int nx = P.nx;
    const T *row = v + (int64_t)y * nx;
    int xm = wrapm(x, nx), xp = wrapp(x, nx);
    T c = row[x];
    T vm = row[xm], vp = row[xp];
    T out = fd_dir(P, vm, c, vp, P.inv_hx);
    if (P.dims == 2) {
        int ym = wrapm(y, P.ny), yp = wrapp(y, P.ny);
        out += fd_dir(P, v[(int64_t)ym * nx + x], c, v[(int64_t)yp * nx + x], P.inv_hy);
    } else if (P.gamma_half) {
        out += fd_gamma(P, x, xm, vm, c, vp);
    }
    return out;
}

// derivative of one direction of D at u (values um, u, up) along w (wm, w, wp)
template <typename T>
__device__ __forceinline__ T fd_dir_jvp(const Params<T> &P, T um, T u, T up, T wm, T w, T wp, T inv_h) {
    T fr, fl;                                   // derivatives of F_{j+1/2}, F_{j-1/2}
    if (P.space == FD_UPWIND) {
        fr = dflux(P, u) * w;
        fl = dflux(P, um) * wm;
    } else {
        fr = T(0.5) * (dflux(P, u) * w + dflux(P, up) * wp) - T(0.5) * P.lf_a * (wp - w);
        fl = T(0.5) * (dflux(P, um) * wm + dflux(P, u) * w) - T(0.5) * P.lf_a * (w - wm);
    }
    T out = (fr - fl) * inv_h;
    if (P.nu != T(0)) out -= P.nu * (wp - T(2) * w + wm) * inv_h * inv_h;
    return out;
}

// D'(u) w at point (y, x) of slices u, w
template <typename T>
__device__ __forceinline__ T fd_D_jvp(const Params<T> &P, const T *__restrict__ u, const T *__restrict__ w, int y,
                                      int x) {
    const int nx = P.nx;
    const int64_t r = (int64_t)y * nx;
    int xm = wrapm(x, nx), xp = wrapp(x, nx);
    T out = fd_dir_jvp(P, u[r + xm], u[r + x], u[r + xp], w[r + xm], w[r + x], w[r + xp], P.inv_hx);
    if (P.dims == 2) {
        const int64_t rm = (int64_t)wrapm(y, P.ny) * nx, rp = (int64_t)wrapp(y, P.ny) * nx;
        out += fd_dir_jvp(P, u[rm + x], u[r + x], u[rp + x], w[rm + x], w[r + x], w[rp + x], P.inv_hy);
    } else if (P.gamma_half) {
        out += fd_gamma(P, x, xm, w[r + xm], w[r + x], w[r + xp]);
    }
    return out;
}

// D'(v)^T psi at point (y, x): v pointwise, psi with halo
template <typename T>
__device__ __forceinline__ T fd_DT(const Params<T> &P, T v, const T *__restrict__ psi, int y, int x) {
    const int nx = P.nx;
    const T *row = psi + (int64_t)y * nx;
    int xm = wrapm(x, nx), xp = wrapp(x, nx);
    T p = row[x], pm = row[xm], pp = row[xp];
    T out = fd_dir_T(P, v, pm, p, pp, P.inv_hx);
    if (P.dims == 2) {
        int ym = wrapm(y, P.ny), yp = wrapp(y, P.ny);
        out += fd_dir_T(P, v, psi[(int64_t)ym * nx + x], p, psi[(int64_t)yp * nx + x], P.inv_hy);
    } else if (P.gamma_half) {
        out += fd_gamma(P, x, xm, pm, p, pp);
    }
    return out;
}

// ---------------------------------------------------------------------------
// DG P2, modal Legendre basis P0, P1, P2 on cells of width h, global
// Lax-Friedrichs interface flux; the residual carries the inverse mass matrix
// diag((2m+1)/h) (as in Eq. 3.5):
//   D_m = -(2m+1)/h [ int f(u_h) P_m' dxi - Fh_{j+1/2} + (-1)^m Fh_{j-1/2} ],
// volume integral by 3-point Gauss-Legendre (exact for quadratic f on P2).
// ---------------------------------------------------------------------------
struct Gauss3 {
    // nodes -sqrt(3/5), 0, sqrt(3/5); weights 5/9, 8/9, 5/9
    static constexpr double x = 0.77459666924148337704;   // sqrt(0.6)
    static constexpr double w0 = 5.0 / 9.0, w1 = 8.0 / 9.0;
};

template <typename T>
__device__ __forceinline__ T dg_face(const Params<T> &P, T ul, T ur) {
    return T(0.5) * (flux(P, ul) + flux(P, ur)) - T(0.5) * P.lf_a * (ur - ul);
}

// D for one cell: c = cell j's modes, l = cell j-1, r = cell j+1
template <typename T>
__device__ __forceinline__ void dg_D(const Params<T> &P, const T c[3], const T l[3], const T r[3], T out[3]) {
    const T gx = T(Gauss3::x), w0 = T(Gauss3::w0), w1 = T(Gauss3::w1);
    // u at the Gauss nodes: P2(+-gx) = 0.4, P2(0) = -0.5
    T qm = c[0] - gx * c[1] + T(0.4) * c[2];
    T q0 = c[0] - T(0.5) * c[2];
    T qp = c[0] + gx * c[1] + T(0.4) * c[2];
    T fm = flux(P, qm), f0 = flux(P, q0), fp = flux(P, qp);
    T vol1 = w0 * (fm + fp) + w1 * f0;                // P1' = 1
    T vol2 = T(3) * gx * w0 * (fp - fm);              // P2' = 3 xi (xi = 0 term vanishes)
    T uR = c[0] + c[1] + c[2];
    T uL = c[0] - c[1] + c[2];
    T uRl = l[0] + l[1] + l[2];
    T uLr = r[0] - r[1] + r[2];
    T Fp = dg_face(P, uR, uLr);
    T Fm = dg_face(P, uRl, uL);
    T ih = P.inv_hx;
    out[0] = -ih * (-Fp + Fm);
    out[1] = -T(3) * ih * (vol1 - Fp - Fm);
    out[2] = -T(5) * ih * (vol2 - Fp + Fm);
}

// D'(U)^T Psi for one cell k: c = U_k; psi_l, psi_c, psi_r = Psi at k-1, k, k+1
template <typename T>
__device__ __forceinline__ void dg_DT(const Params<T> &P, const T c[3], const T pl[3], const T pc[3],
                                      const T pr[3], T out[3]) {
    const T gx = T(Gauss3::x), w0 = T(Gauss3::w0), w1 = T(Gauss3::w1);
    const T ih = P.inv_hx;
    // S_m = (2m+1)/h Psi_m
    T sc0 = ih * pc[0], sc1 = T(3) * ih * pc[1], sc2 = T(5) * ih * pc[2];
    T sl0 = ih * pl[0], sl1 = T(3) * ih * pl[1], sl2 = T(5) * ih * pl[2];
    T sr0 = ih * pr[0], sr1 = T(3) * ih * pr[1], sr2 = T(5) * ih * pr[2];
    // volume part: -sum_q P_n(xi_q) f'(u_q) w_q sum_m P_m'(xi_q) S_m
    T qm = c[0] - gx * c[1] + T(0.4) * c[2];
    T q0 = c[0] - T(0.5) * c[2];
    T qp = c[0] + gx * c[1] + T(0.4) * c[2];
    T im_ = w0 * dflux(P, qm) * (sc1 - T(3) * gx * sc2);
    T i0_ = w1 * dflux(P, q0) * sc1;
    T ip_ = w0 * dflux(P, qp) * (sc1 + T(3) * gx * sc2);
    T o0 = -(im_ + i0_ + ip_);
    T o1 = -(gx * (ip_ - im_));
    T o2 = -(T(0.4) * (im_ + ip_) - T(0.5) * i0_);
    // interface part
    T Gk = (sc0 + sc1 + sc2) - (sr0 - sr1 + sr2);        // coefficient of Fh_{k+1/2}
    T Gkm = (sl0 + sl1 + sl2) - (sc0 - sc1 + sc2);       // coefficient of Fh_{k-1/2}
    T uR = c[0] + c[1] + c[2];
    T uL = c[0] - c[1] + c[2];
    T dA = T(0.5) * (dflux(P, uR) + P.lf_a);              // dFh_{k+1/2}/duR_k
    T dB = T(0.5) * (dflux(P, uL) - P.lf_a);              // dFh_{k-1/2}/duL_k
    T a = Gk * dA, b = Gkm * dB;
    out[0] = o0 + a + b;
    out[1] = o1 + a - b;
    out[2] = o2 + a + b;
}

// ---------------------------------------------------------------------------
// DG P1 with the nodal basis of Sec. 3.2.2 (nodes x_{j-1/4}, x_{j+1/4}):
// phi_1(xi) = 1/2 - xi, phi_2(xi) = 1/2 + xi, mass matrix (h/12)[[7,-1],[-1,7]],
// so h M^{-1} = [[7,1],[1,7]]/4.  With E_m = int f(u_h) phi_m' dxi
// - Fh_{j+1/2} phi_m(1) + Fh_{j-1/2} phi_m(-1), the residual is D = -M^{-1} E.
// Volume integral by 2-point Gauss (exact for quadratic f); interface flux
// upwind f(u-) or global Lax-Friedrichs.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ bool is_dg(int space) { return space >= DG_P2_LF; }

template <typename T>
__device__ __forceinline__ T dg1_face(const Params<T> &P, T a, T b) {
    if (P.space == DG_P1_UPWIND) return flux(P, a);
    return T(0.5) * (flux(P, a) + flux(P, b)) - T(0.5) * P.lf_a * (b - a);
}

template <typename T>
__device__ __forceinline__ void dg1_D(const Params<T> &P, const T c[2], const T l[2], const T r[2], T out[2]) {
    const T g = T(0.57735026918962576451);                  // 1/sqrt(3)
    const T qm = c[0] * (T(0.5) + g) + c[1] * (T(0.5) - g);   // u_h(-g)
    const T qp = c[0] * (T(0.5) - g) + c[1] * (T(0.5) + g);   // u_h(+g)
    const T V = flux(P, qm) + flux(P, qp);
    const T uR = T(-0.5) * c[0] + T(1.5) * c[1], uL = T(1.5) * c[0] - T(0.5) * c[1];
    const T uRl = T(-0.5) * l[0] + T(1.5) * l[1], uLr = T(1.5) * r[0] - T(0.5) * r[1];
    const T Fp = dg1_face(P, uR, uLr), Fm = dg1_face(P, uRl, uL);
    const T E0 = -V + T(0.5) * Fp + T(1.5) * Fm;
    const T E1 = V - T(1.5) * Fp - T(0.5) * Fm;
    const T s = T(-0.25) * P.inv_hx;
    out[0] = s * (T(7) * E0 + E1);
    out[1] = s * (E0 + T(7) * E1);
}

// D'(U)^T Psi for cell k: c = U_k; pl, pc, pr = Psi at k-1, k, k+1.
// With A = -(h M)^{-1} Psi (per cell) the pairing is sum_j A_j . dE_j; the volume
// term is cell-local, Fh_{k+1/2} carries G_k = -sum_m phi_m(1) A_m(k) +
// sum_m phi_m(-1) A_m(k+1) and is differentiated in its left state uR_k, and
// Fh_{k-1/2} (coefficient G_{k-1}) in its right state uL_k.
template <typename T>
__device__ __forceinline__ void dg1_DT(const Params<T> &P, const T c[2], const T pl[2], const T pc[2],
                                       const T pr[2], T out[2]) {
    const T g = T(0.57735026918962576451);
    const T s = T(-0.25) * P.inv_hx;
    const T a0 = s * (T(7) * pc[0] + pc[1]), a1 = s * (pc[0] + T(7) * pc[1]);
    const T l0 = s * (T(7) * pl[0] + pl[1]), l1 = s * (pl[0] + T(7) * pl[1]);
    const T r0 = s * (T(7) * pr[0] + pr[1]), r1 = s * (pr[0] + T(7) * pr[1]);
    const T qm = c[0] * (T(0.5) + g) + c[1] * (T(0.5) - g);
    const T qp = c[0] * (T(0.5) - g) + c[1] * (T(0.5) + g);
    const T cV = a1 - a0;
    const T dm = dflux(P, qm) * cV, dp = dflux(P, qp) * cV;
    T o0 = (T(0.5) + g) * dm + (T(0.5) - g) * dp;
    T o1 = (T(0.5) - g) * dm + (T(0.5) + g) * dp;
    const T Gk = (T(0.5) * a0 - T(1.5) * a1) + (T(1.5) * r0 - T(0.5) * r1);
    const T Gkm = (T(0.5) * l0 - T(1.5) * l1) + (T(1.5) * a0 - T(0.5) * a1);
    const T uR = T(-0.5) * c[0] + T(1.5) * c[1], uL = T(1.5) * c[0] - T(0.5) * c[1];
    T da, db;
    if (P.space == DG_P1_UPWIND) { da = dflux(P, uR); db = T(0); }
    else { da = T(0.5) * (dflux(P, uR) + P.lf_a); db = T(0.5) * (dflux(P, uL) - P.lf_a); }
    const T A = Gk * da, B = Gkm * db;
    o0 += T(-0.5) * A + T(1.5) * B;      // phi(1) = (-1/2, 3/2), phi(-1) = (3/2, -1/2)
    o1 += T(1.5) * A + T(-0.5) * B;
    out[0] = o0;
    out[1] = o1;
}

// DG dispatch for either basis (nm = 3: P2 Legendre, nm = 2: P1 nodal)
template <typename T>
__device__ __forceinline__ void dgx_D(const Params<T> &P, const T c[3], const T l[3], const T r[3], T out[3]) {
    if (P.space == DG_P2_LF) dg_D(P, c, l, r, out);
    else dg1_D(P, c, l, r, out);
}
template <typename T>
__device__ __forceinline__ void dgx_DT(const Params<T> &P, const T c[3], const T pl[3], const T pc[3], const T pr[3],
                                       T out[3]) {
    if (P.space == DG_P2_LF) dg_DT(P, c, pl, pc, pr, out);
    else dg1_DT(P, c, pl, pc, pr, out);
}

// ---------------------------------------------------------------------------
// residual norms (Eq. 2.12) in double: per-block partial sums, fixed order (block
// sum of the threads' records by warp shuffles, then over the warps)
//   acc[0] = sum R^2, acc[1] = sum (J^T phi)^2 over l >= 1, acc[2] = sum phi R,
//   acc[3] = sum (u^0 - u0)^2, acc[4] = sum (h_t (J^T phi)^0 + lambda)^2,
//   acc[5] = sum lambda (u^0 - u0)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_sum6(double acc[6], double *out) {
    __shared__ double red[32][6];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    if (lane == 0)
        for (int k = 0; k < 6; ++k) red[wid][k] = acc[k];
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < 6; ++k) {
            double v = lane < nw ? red[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) out[k] = v;
        }
    }
}

}  // namespace pdhg

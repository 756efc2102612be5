// kernels_fused2d.cu -- the fused iteration of Algorithm 1 (Sec. 3.3) for 2D
// finite differences in float32: four kernels per iteration.
//
//   primal  (every slice at once, in place) u^n = u^{n-1} - tau_u J(u^{n-1})^T phit^{n-1},
//           and the u^0 / lambda row.
//   rows-R  (row blocks of H rows x a chunk of time slices, marching in t)
//           residual R^{l}(u^n) on the block's rows, real FFT along x of each
//           residual row, and a transposed store of the spectrum (layout [l][kx][y]).
//   cols    (one kx column per block, marching in t forward then backward)
//           complex FFT along y, forward elimination of (T_t + kappa h_t^2)
//           per mode with the spill written in place, back substitution, and
//           inverse FFT along y, written in place: the x-spectrum of z.
//   rows-C  (tiles of H rows x one slice; at nx = 1024 persistent blocks whose tiles'
//           spectra arrive by TMA) inverse real FFT along x, dual step
//           phi^n = phi^{n-1} + tau_phi z and extrapolation phit = phi^n + tau_phi z.
// Also here: the residual norms of a 2D finite-difference state (k_check2d, float32 and
// float64).  Debug builds (-DPDHG_DEBUG) check the global indices of these kernels
// (common.cuh::dbg_idx).
#include <algorithm>
#include <type_traits>

#include "fused2d.h"
#include "fft_smem.cuh"
#include "stockham.cuh"
#include "tma.cuh"

namespace pdhg {

constexpr int FH = 4;          // rows per block in the row kernels
constexpr int FTHREADS = 256;
constexpr int ATHREADS = 256;  // rows-R block size

// ---------------------------------------------------------------------------
// primal (every slice at once): u^n = u^{n-1} - tau_u J(u^{n-1})^T phit^{n-1}.
// J^T phit at (m, y, x) needs u only at that point (f'(u) multiplies the
// transposed stencil of phit^{m-1}), so the update is in place.  A thread owns
// one float4 of x and RY consecutive rows of one slice and slides a three-row
// window of phit^{m-1} down them, so each phit^{m-1} value is loaded once per
// thread column (plus one halo row above and below).
// ---------------------------------------------------------------------------
constexpr int PRY = 4;          // rows per thread in the primal kernel

// The part of (J(u)^T phit)^m at one point that comes from phit^{m-1}: the time
// coefficient cn times phit^{m-1} there, plus the transposed stencil linearised at
// c = u^m (multipliers mx, p0, qx at x-1, x, x+1 and my, qy at y-1, y+1):
//   LF: (f'(u) (m - q) + a (2p - m - q)) / 2h;  upwind: f'(u) (p - q) / h;
//   viscous: -nu (q - 2p + m) / h^2.
__device__ __forceinline__ float primal_g1(const Params<float> &P, bool lf, float c, float cn, float p0, float mx,
                                           float qx, float my, float qy) {
    const float df = dflux(P, c);
    float tx, ty;
    if (lf) {
        tx = 0.5f * (df * (mx - qx) + P.lf_a * (2.f * p0 - mx - qx));
        ty = 0.5f * (df * (my - qy) + P.lf_a * (2.f * p0 - my - qy));
    } else {
        tx = df * (p0 - qx);
        ty = df * (p0 - qy);
    }
    float g = cn * p0 + tx * P.inv_hx + ty * P.inv_hy;
    if (P.nu != 0.f)
        g -= P.nu * ((qx - 2.f * p0 + mx) * P.inv_hx * P.inv_hx + (qy - 2.f * p0 + my) * P.inv_hy * P.inv_hy);
    return g;
}

template <int NX>
__global__ void __launch_bounds__(256) k_primal2d(Params<float> P, float *__restrict__ u,
                                                  const float *__restrict__ phit, float *__restrict__ lam,
                                                  float *__restrict__ lamt, const float *__restrict__ u0) {
    constexpr int V = NX / 4;                        // blockDim = (min(V, 256), max(256 / V, 1))
    const int x4 = threadIdx.x + (V > 256 ? blockIdx.z * 256 : 0);
    const int ya = (blockIdx.x * blockDim.y + threadIdx.y) * PRY;
    const int m = blockIdx.y;
    const int ny = P.ny, nt = P.nt;
    const int64_t S = P.S, nU = (int64_t)(nt + 1) * S, nF = (int64_t)nt * S;
    float *um = u + (int64_t)m * S;
    const int64_t nUm = nU - (int64_t)m * S;                // elements from um to the end of u
    const float cc = m <= nt - 1 ? coef_cur(P, m) : 0.f;
    const float co = (P.time == BDF2 && m + 1 <= nt - 1) ? coef_old(P, m + 1) : 0.f;
    if (m == 0) {
        if (P.init != INIT_LAMBDA) return;              // u^0 pinned to u0
        // u^0 -= tau_u0 (h_t (J^T phit)^0 + lamt); lambda ascent and extrapolation
#pragma unroll
        for (int r = 0; r < PRY; ++r) {
            const int64_t i = (int64_t)(ya + r) * NX + 4 * x4;
            float4 *up = reinterpret_cast<float4 *>(um + dbg_idx(P, i, nUm - 3, 101));
            const float4 c = *up;
            const float4 tc = __ldg(reinterpret_cast<const float4 *>(phit + dbg_idx(P, i, nF - 3, 102)));
            float4 tn = make_float4(0.f, 0.f, 0.f, 0.f);
            if (co != 0.f) tn = __ldg(reinterpret_cast<const float4 *>(phit + dbg_idx(P, S + i, nF - 3, 103)));
            const float cv[4] = {c.x, c.y, c.z, c.w};
            const float gv[4] = {cc * tc.x + co * tn.x, cc * tc.y + co * tn.y, cc * tc.z + co * tn.z,
                                 cc * tc.w + co * tn.w};
            float un[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t k = dbg_idx(P, i + e, S, 104);
                un[e] = cv[e] - P.tau_u0 * (P.ht * gv[e] + lamt[k]);
                const float r0 = un[e] - u0[k];
                const float ln = lam[k] + P.tau_lambda * r0;
                lam[k] = ln;
                lamt[k] = ln + P.tau_lambda * r0;
            }
            *up = make_float4(un[0], un[1], un[2], un[3]);
        }
        return;
    }
    const float cn = coef_new(P, m - 1);
    const float *pp = phit + (int64_t)(m - 1) * S;        // phit^{m-1}: transposed stencil
    const float *pc = phit + (int64_t)m * S;              // phit^m: pointwise (m <= nt-1)
    const int64_t npp = nF - (int64_t)(m - 1) * S, npc = nF - (int64_t)m * S;
    const bool lf = P.space != FD_UPWIND;
    auto prow = [&](int y) -> int64_t {                  // element offset of row y in pp
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        return (int64_t)y * NX;
    };
    float4 pu = __ldg(reinterpret_cast<const float4 *>(pp + dbg_idx(P, prow(ya - 1) + 4 * x4, npp - 3, 105)));
    float4 pm = __ldg(reinterpret_cast<const float4 *>(pp + dbg_idx(P, prow(ya) + 4 * x4, npp - 3, 105)));
#pragma unroll
    for (int r = 0; r < PRY; ++r) {
        const int y = ya + r;
        const int64_t row = (int64_t)y * NX;
        const float4 pd = __ldg(reinterpret_cast<const float4 *>(pp + dbg_idx(P, prow(y + 1) + 4 * x4, npp - 3, 105)));
        const float lft = __ldg(pp + dbg_idx(P, row + (x4 == 0 ? NX - 1 : 4 * x4 - 1), npp, 106));
        const float rgt = __ldg(pp + dbg_idx(P, row + (x4 == V - 1 ? 0 : 4 * x4 + 4), npp, 106));
        const int64_t i = (int64_t)y * NX + 4 * x4;
        float4 *up = reinterpret_cast<float4 *>(um + dbg_idx(P, i, nUm - 3, 107));
        const float4 c = *up;
        float4 tc = make_float4(0.f, 0.f, 0.f, 0.f), tn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (cc != 0.f) tc = __ldg(reinterpret_cast<const float4 *>(pc + dbg_idx(P, i, npc - 3, 108)));
        if (co != 0.f) tn = __ldg(reinterpret_cast<const float4 *>(pc + dbg_idx(P, S + i, npc - 3, 109)));
        const float pr[6] = {lft, pm.x, pm.y, pm.z, pm.w, rgt};
        const float uv[4] = {pu.x, pu.y, pu.z, pu.w}, dv[4] = {pd.x, pd.y, pd.z, pd.w};
        const float cv[4] = {c.x, c.y, c.z, c.w};
        const float gv[4] = {cc * tc.x + co * tn.x, cc * tc.y + co * tn.y, cc * tc.z + co * tn.z,
                             cc * tc.w + co * tn.w};
        float un[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float ge = primal_g1(P, lf, cv[e], cn, pr[e + 1], pr[e], pr[e + 2], uv[e], dv[e]) + gv[e];
            un[e] = cv[e] - P.tau_u * ge;
        }
        *up = make_float4(un[0], un[1], un[2], un[3]);
        pu = pm;
        pm = pd;
    }
}

// ---------------------------------------------------------------------------
// rows-R: residual R^l(u^n) and its real FFT along x, spectrum stored
// transposed ([l][kx][y]).  A block owns FH rows and a chunk of time slices and
// marches in t over a ring of u rows y0-1 .. y0+FH (the y-stencil needs one
// halo row each side); the rows of step m+1 are fetched into registers while
// step m computes.  Shared memory (x fastest):
//   us  [NR][FH+2][NX]  u^m, u^{m-1} (and u^{m-2} for BDF2)
//   scr [FH][PN]        FFT scratch
// The FFT input aliases the u slot that the residual no longer needs, so BE
// takes 67 KB at nx = 1024: three blocks per SM.
// ---------------------------------------------------------------------------
template <int NX, int N>
__device__ __forceinline__ void fetch_rows(float4 (&reg)[N], const Params<float> &P, const float *__restrict__ u,
                                           int64_t slice_off, int ybase, int ny) {
    constexpr int V = NX / 4;
    const int64_t nU = (int64_t)(P.nt + 1) * P.S;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int idx = threadIdx.x + j * ATHREADS;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < (FH + 2) * V) {
            const int r = idx / V, c = idx - r * V;
            int y = ybase + r;
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            v = __ldg(reinterpret_cast<const float4 *>(u + dbg_idx(P, slice_off + (int64_t)y * NX + 4 * c, nU - 3, 201)));
        }
        reg[j] = v;
    }
}

template <int NX, int N>
__device__ __forceinline__ void store_rows(float *dst, const float4 (&reg)[N]) {
    constexpr int V = NX / 4;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int idx = threadIdx.x + j * ATHREADS;
        if (idx < (FH + 2) * V) reinterpret_cast<float4 *>(dst)[idx] = reg[j];
    }
}

template <int LOG2M, bool BDF2_>
__global__ void __launch_bounds__(ATHREADS, (LOG2M >= 10 ? 1 : (BDF2_ ? 2 : 3)))
k_rowsR(Params<float> P, const float *__restrict__ u, float2 *__restrict__ spec,
        const float2 *__restrict__ twN, const float2 *__restrict__ tw8, int Tc) {
    constexpr int M = 1 << LOG2M, NX = 2 * M;
    constexpr int NR = BDF2_ ? 3 : 2;            // u ring slots
    constexpr int RU = FH + 2;                   // u rows: block rows + one halo row each side
    constexpr int PN = R8<LOG2M>::PN;            // FFT row stride (radix-8 layout, stockham.cuh)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *us = reinterpret_cast<float *>(smem_raw);                  // [NR][RU][NX]
    float2 *scr = reinterpret_cast<float2 *>(us + NR * RU * NX);     // [FH][PN]

    const int ny = P.ny, nt = P.nt;
    const int64_t S = P.S;
    const int y0 = blockIdx.x * FH;
    const int l0 = blockIdx.y * Tc;
    const int l1 = min(l0 + Tc, nt);              // residual slices [l0, l1)
    const int mstart = (BDF2_ && l0 > 0) ? l0 - 1 : l0;
    constexpr int UPT = (RU * (NX / 4) + ATHREADS - 1) / ATHREADS;
    float4 ru[UPT];
    fetch_rows<NX>(ru, P, u, (int64_t)mstart * S, y0 - 1, ny);
    for (int m = mstart; m <= l1; ++m) {
        float *uc = us + (m % NR) * RU * NX;             // u^m
        store_rows<NX>(uc, ru);
        if (m + 1 <= l1) fetch_rows<NX>(ru, P, u, (int64_t)(m + 1) * S, y0 - 1, ny);
        __syncthreads();
        const int lr = m - 1;
        if (lr >= l0 && lr < l1) {
            const float *un = uc;
            const float *ucur = us + ((m + NR - 1) % NR) * RU * NX;
            const float *uold = us + ((m + NR - 2) % NR) * RU * NX;
            const float kn = coef_new(P, lr), kc = coef_cur(P, lr), ko = coef_old(P, lr);
            // thread -> CPT float4 columns x RPT consecutive rows (a sliding window over
            // the rows, so each value's flux is evaluated once per thread column)
            constexpr int V = NX / 4;
            constexpr int TX = V < ATHREADS ? V : ATHREADS;       // threads across a row
            constexpr int RPT = FH * TX / ATHREADS;                // rows per thread
            constexpr int CPT = V / TX;                            // columns per thread
            const int xb = threadIdx.x % TX, rb = (threadIdx.x / TX) * RPT;
            const bool lf = P.space != FD_UPWIND;
            float4 R[CPT][RPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int x4 = xb + c * TX;
                float4 up = reinterpret_cast<const float4 *>(un + rb * NX)[x4];
                float fu[4] = {flux(P, up.x), flux(P, up.y), flux(P, up.z), flux(P, up.w)};
                float4 v4 = reinterpret_cast<const float4 *>(un + (rb + 1) * NX)[x4];
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    const int r = rb + q + 1;                      // ring row of the residual row
                    const float *row = un + r * NX;
                    const float4 dn = reinterpret_cast<const float4 *>(un + (r + 1) * NX)[x4];
                    const float4 cu = reinterpret_cast<const float4 *>(ucur + r * NX)[x4];
                    const float lft = row[x4 == 0 ? NX - 1 : 4 * x4 - 1];
                    const float rgt = row[x4 == V - 1 ? 0 : 4 * x4 + 4];
                    const float vr[6] = {lft, v4.x, v4.y, v4.z, v4.w, rgt};
                    const float uv[4] = {up.x, up.y, up.z, up.w}, dv[4] = {dn.x, dn.y, dn.z, dn.w};
                    const float cv[4] = {cu.x, cu.y, cu.z, cu.w};
                    float ov[4] = {0.f, 0.f, 0.f, 0.f};
                    if (BDF2_ && lr >= 1) {
                        const float4 o4 = reinterpret_cast<const float4 *>(uold + r * NX)[x4];
                        ov[0] = o4.x; ov[1] = o4.y; ov[2] = o4.z; ov[3] = o4.w;
                    }
                    // D in flux-difference form with each f(v) evaluated once per value:
                    //   LF: (F_{j+1/2} - F_{j-1/2}) = (f_{j+1} - f_{j-1})/2 - a (v_{j+1} - 2 v_j + v_{j-1})/2
                    //   upwind: f_j - f_{j-1};  viscous: -nu (v_{j+1} - 2 v_j + v_{j-1}) / h^2
                    float fx[6], fd[4];
                    fx[0] = flux(P, lft);
                    fx[5] = flux(P, rgt);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        fx[e + 1] = flux(P, vr[e + 1]);
                        fd[e] = flux(P, dv[e]);
                    }
                    float Rv[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float v = vr[e + 1];
                        const float lx = vr[e] - 2.f * v + vr[e + 2], ly = uv[e] - 2.f * v + dv[e];
                        float dx, dy;
                        if (lf) {
                            dx = 0.5f * (fx[e + 2] - fx[e]) - 0.5f * P.lf_a * lx;
                            dy = 0.5f * (fd[e] - fu[e]) - 0.5f * P.lf_a * ly;
                        } else {
                            dx = fx[e + 1] - fx[e];
                            dy = fx[e + 1] - fu[e];
                        }
                        float rv = dx * P.inv_hx + dy * P.inv_hy + kn * v + kc * cv[e];
                        if (P.nu != 0.f) rv -= P.nu * (lx * P.inv_hx * P.inv_hx + ly * P.inv_hy * P.inv_hy);
                        if (BDF2_ && lr >= 1) rv += ko * ov[e];
                        Rv[e] = rv;
                    }
                    R[c][q] = make_float4(Rv[0], Rv[1], Rv[2], Rv[3]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) fu[e] = fx[e + 1];
                    up = v4;
                    v4 = dn;
                }
            }
            __syncthreads();
            // FFT input in the u slot the residual no longer needs (BE: u^{m-1}, BDF2: u^{m-2})
            float2 *fin2 = reinterpret_cast<float2 *>(const_cast<float *>(BDF2_ ? uold : ucur));
#pragma unroll
            for (int c = 0; c < CPT; ++c)               // z_n = R_{2n} + i R_{2n+1}
#pragma unroll
                for (int q = 0; q < RPT; ++q)
                    *reinterpret_cast<float4 *>(fin2 + (rb + q) * PN + 2 * (xb + c * TX)) = R[c][q];
            __syncthreads();
            const float2 *res = stockham8<LOG2M, false, FH, ATHREADS>(fin2, scr, tw8);
            // split pairs (k, M-k), k = 0..M/2, both outputs from one pair of loads
            const int64_t dst0 = (int64_t)lr * P.nkx * ny + y0, nX = (int64_t)P.nt * P.nkx * ny;
            for (int idx = threadIdx.x; idx < (M / 2 + 1) * FH; idx += blockDim.x) {
                const int k = idx / FH, rr = idx - k * FH;
                const float2 *row = res + rr * PN;
                float2 xk, xm;
                rfft_split_pair(row[k], row[k == 0 ? 0 : M - k], __ldg(twN + k), xk, xm);
                spec[dbg_idx(P, dst0 + (int64_t)k * ny + rr, nX, 202)] = xk;
                if (k != M / 2) spec[dbg_idx(P, dst0 + (int64_t)(M - k) * ny + rr, nX, 202)] = xm;
            }
        }
        __syncthreads();
    }
}

// rows-R for nx = 1024 (M = 512), the u window in registers: thread t owns the float4
// column x = 4t..4t+3 of the window rows y0-1..y0+4 of u^m (global loads; the halo rows
// are also the neighbouring row blocks' rows and come from L2) and of rows y0..y0+3 of
// u^{m-1} (and u^{m-2} for BDF2), carried over from the previous steps.  The
// x-neighbours 4t-1 and 4t+4 come from the adjacent lanes by shuffles; lanes 0 and 31
// load theirs.  Each flux value is evaluated once per step and row.  The next step's u
// rows are loaded after the transform, so they arrive during the split.  The
// residual rows go to fa, the three radix-8 stages run fa -> fb -> fa -> fb, and the
// split reads fb while the next step's residual is written to fa: four barriers per
// step.  R is evaluated with the Lax-Friedrichs and viscous second differences folded
// into per-block coefficients (the same R as k_rowsR up to rounding order).
template <bool BDF2_>
__global__ void __launch_bounds__(ATHREADS, 3)
k_rowsR1024(Params<float> P, const float *__restrict__ u, float2 *__restrict__ spec,
            const float2 *__restrict__ twN, const float2 *__restrict__ tw8, int Tc) {
    constexpr int LOG2M = 9, M = 512, NX = 1024, PN = R8<LOG2M>::PN, RU = FH + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *fa = reinterpret_cast<float2 *>(smem_raw);      // [FH][PN] FFT input z_n = R_2n + i R_2n+1
    float2 *fb = fa + FH * PN;                               // [FH][PN]
    const int ny = P.ny, nt = P.nt;
    const int64_t S = P.S, nU = (int64_t)(nt + 1) * S;
    const int t = threadIdx.x, lane = t & 31;
    const int y0 = blockIdx.x * FH;
    const int l0 = blockIdx.y * Tc;
    const int l1 = min(l0 + Tc, nt);                         // residual slices [l0, l1)
    const int mstart = (BDF2_ && l0 > 0) ? l0 - 1 : l0;
    const bool lf = P.space != FD_UPWIND;
    // window row r = y0 - 1 + r (periodic in y): element offsets within a slice
    const int obase = y0 * NX;
    const int oup = (y0 == 0 ? ny - 1 : y0 - 1) * NX, odn = (y0 + FH == ny ? 0 : y0 + FH) * NX;
    auto roff = [&](int r) { return r == 0 ? oup : (r == RU - 1 ? odn : obase + (r - 1) * NX); };
    // the x-neighbour column that lane 0 (left) or lane 31 (right) loads itself
    const int xe = lane == 0 ? (t == 0 ? NX - 1 : 4 * t - 1) : (t == ATHREADS - 1 ? 0 : 4 * t + 4);
    float4 cur[RU], prv[FH], old[FH];
    float ed[FH];                                            // lanes 0 / 31: that neighbour in rows 1..4
    auto load = [&](int m) {
        const float *um = u + (int64_t)m * S;
        const int64_t nUm = nU - (int64_t)m * S;
#pragma unroll
        for (int r = 0; r < RU; ++r)
            cur[r] = __ldg(reinterpret_cast<const float4 *>(um + dbg_idx(P, (int64_t)roff(r) + 4 * t, nUm - 3, 203)));
        if (lane == 0 || lane == 31) {
#pragma unroll
            for (int r = 0; r < FH; ++r) ed[r] = __ldg(um + dbg_idx(P, (int64_t)roff(r + 1) + xe, nUm, 204));
        }
    };
#pragma unroll
    for (int r = 0; r < FH; ++r) {
        prv[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        old[r] = prv[r];
        ed[r] = 0.f;
    }
    load(mstart);
    for (int m = mstart; m <= l1; ++m) {
        const int lr = m - 1;
        const bool act = lr >= l0 && lr < l1;                // block-uniform
        if (act) {
            const float kc = coef_cur(P, lr), ko = coef_old(P, lr);
            // R = A1 F1 + A2 F2 - ax (v_{x-1} + v_{x+1}) - ay (v_{y-1} + v_{y+1}) + cv v + kc u^{m-1}
            //     (+ ko u^{m-2}), with the flux differences F1 (x), F2 (y) of the scheme and the
            //     Lax-Friedrichs and viscous second differences folded into ax, ay, cv
            const float ax = (lf ? 0.5f * P.lf_a * P.inv_hx : 0.f) + P.nu * P.inv_hx * P.inv_hx;
            const float ay = (lf ? 0.5f * P.lf_a * P.inv_hy : 0.f) + P.nu * P.inv_hy * P.inv_hy;
            const float A1 = lf ? 0.5f * P.inv_hx : P.inv_hx, A2 = lf ? 0.5f * P.inv_hy : P.inv_hy;
            const float cvc = coef_new(P, lr) + 2.f * (ax + ay);
            float fu[4] = {flux(P, cur[0].x), flux(P, cur[0].y), flux(P, cur[0].z), flux(P, cur[0].w)};
            float fm[4] = {flux(P, cur[1].x), flux(P, cur[1].y), flux(P, cur[1].z), flux(P, cur[1].w)};
#pragma unroll
            for (int r = 1; r <= FH; ++r) {
                const float4 v4 = cur[r], up = cur[r - 1], dn = cur[r + 1], cu = prv[r - 1];
                float lft = __shfl_up_sync(0xffffffffu, v4.w, 1);
                float rgt = __shfl_down_sync(0xffffffffu, v4.x, 1);
                if (lane == 0) lft = ed[r - 1];
                if (lane == 31) rgt = ed[r - 1];
                const float vr[6] = {lft, v4.x, v4.y, v4.z, v4.w, rgt};
                const float uv[4] = {up.x, up.y, up.z, up.w}, dv[4] = {dn.x, dn.y, dn.z, dn.w};
                const float cv[4] = {cu.x, cu.y, cu.z, cu.w};
                float ov[4] = {0.f, 0.f, 0.f, 0.f};
                if (BDF2_ && lr >= 1) {
                    const float4 o4 = old[r - 1];
                    ov[0] = o4.x; ov[1] = o4.y; ov[2] = o4.z; ov[3] = o4.w;
                }
                const float fx[6] = {flux(P, lft), fm[0], fm[1], fm[2], fm[3], flux(P, rgt)};
                float fd[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) fd[e] = flux(P, dv[e]);
                float Rv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float v = vr[e + 1];
                    const float F1 = lf ? fx[e + 2] - fx[e] : fx[e + 1] - fx[e];
                    const float F2 = lf ? fd[e] - fu[e] : fx[e + 1] - fu[e];
                    float rv = A1 * F1 + A2 * F2 - ax * (vr[e] + vr[e + 2]) - ay * (uv[e] + dv[e]) + cvc * v +
                               kc * cv[e];
                    if (BDF2_ && lr >= 1) rv += ko * ov[e];
                    Rv[e] = rv;
                }
                *reinterpret_cast<float4 *>(fa + (r - 1) * PN + 2 * t) = make_float4(Rv[0], Rv[1], Rv[2], Rv[3]);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    fu[e] = fm[e];
                    fm[e] = fd[e];
                }
            }
        }
        // slide the window in t: u^{m-1} -> u^{m-2}, u^m -> u^{m-1}; fetch u^{m+1}
#pragma unroll
        for (int r = 0; r < FH; ++r) {
            if (BDF2_) old[r] = prv[r];
            prv[r] = cur[r + 1];
        }
        const float2 *res = fb;
        if (act) {
            __syncthreads();                                  // FFT input complete
            res = stockham8<LOG2M, false, FH, ATHREADS>(fa, fb, tw8);
        }
        if (m + 1 <= l1) load(m + 1);                         // arrives during the split and the other blocks' work
        if (act) {
            // split pairs (k, M-k) of two rows 2p, 2p+1 per item: both outputs of each row from
            // one pair of loads, and the two rows' values at one kx stored as one float4
            const int64_t dst0 = (int64_t)lr * P.nkx * ny + y0, nX = (int64_t)P.nt * P.nkx * ny;
            for (int idx = t; idx < (M / 2 + 1) * 2; idx += ATHREADS) {
                const int k = idx >> 1, p = idx & 1;
                const float2 *ra = res + (2 * p) * PN, *rb = ra + PN;
                const float2 w = __ldg(twN + k);
                const int km = k == 0 ? 0 : M - k;
                float2 ak, am, bk, bm;
                rfft_split_pair(ra[k], ra[km], w, ak, am);
                rfft_split_pair(rb[k], rb[km], w, bk, bm);
                *reinterpret_cast<float4 *>(spec + dbg_idx(P, dst0 + (int64_t)k * ny + 2 * p, nX - 1, 202)) =
                    make_float4(ak.x, ak.y, bk.x, bk.y);
                if (k != M / 2)
                    *reinterpret_cast<float4 *>(spec + dbg_idx(P, dst0 + (int64_t)(M - k) * ny + 2 * p, nX - 1, 202)) =
                        make_float4(am.x, am.y, bm.x, bm.y);
            }
        }
    }
}

static size_t smem_rowsR1024() { return (size_t)2 * FH * R8<9>::PN * 8; }

// ---------------------------------------------------------------------------
// cols: y-FFT, t-solve per mode (closed-form pivots, see kernels_plain.cu),
// inverse y-FFT; spectrum, spill and result share one buffer, in place.
// ---------------------------------------------------------------------------
// The pivots only shape the preconditioner (they change the iterates, never the
// fixed point R(u*) = 0), so the fast exponential and division intrinsics serve:
// their relative errors (~1e-6) are far below what the iteration notices.  Past
// (2l+1) theta = 17, w < 2^-24 and 1 + w, 1 + q w round to 1: the pivot is e^{-theta}
// itself, with no exponential and no division (most steps of most modes).
__device__ __forceinline__ float rho_f(float th, float emt, float q, int l) {
    const float x = (float)(2 * l + 1) * th;
    if (x > 17.f) return emt;
    const float w = __expf(-x);
    return __fdividef(emt * (1.f + w), 1.f + q * w);
}

template <int LOG2NY>
__global__ void __launch_bounds__(FTHREADS) k_cols(Params<float> P, float2 *__restrict__ spec,
                                                   const float2 *__restrict__ twY,
                                                   const float *__restrict__ thetaT) {
    // One kx column per block (all 513 blocks resident at 1024^2).  The y-FFTs of
    // TB consecutive slices are independent, so they run as one batch; only the
    // cheap recurrence over those slices is sequential.
    constexpr int NY = 1 << LOG2NY;
    constexpr int TB = 2;
    constexpr int NPT = NY / FTHREADS > 0 ? NY / FTHREADS : 1;     // modes per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *ba = reinterpret_cast<float2 *>(smem_raw);              // [TB][NY]
    float2 *bb = ba + TB * NY;                                      // [TB][NY]
    float2 *tw = bb + TB * NY;                                      // [NY]
    const int kx = blockIdx.x;
    const int nt = P.nt;
    const int64_t cs = (int64_t)P.nkx * NY;      // slice stride of the spectrum
    float2 *col = spec + (int64_t)kx * NY;
    const int t = threadIdx.x;
    for (int j = t; j < NY; j += FTHREADS) tw[j] = twY[j];
    float th[NPT], emt[NPT], q[NPT];
    float2 acc[NPT], pf[TB][NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int k = t + j * FTHREADS;
        th[j] = thetaT[(int64_t)kx * NY + k];
        emt[j] = expf(-th[j]);
        q[j] = emt[j] * emt[j];
        acc[j] = make_float2(0.f, 0.f);
    }
    const int nb = (nt + TB - 1) / TB;           // slice batches
    // forward sweep: y_l = r_l + rho_{l-1} y_{l-1}
#pragma unroll
    for (int b = 0; b < TB; ++b)
#pragma unroll
        for (int j = 0; j < NPT; ++j)
            pf[b][j] = b < nt ? col[(int64_t)b * cs + t + j * FTHREADS] : make_float2(0.f, 0.f);
    for (int g = 0; g < nb; ++g) {
        const int lb = g * TB;
#pragma unroll
        for (int b = 0; b < TB; ++b)
#pragma unroll
            for (int j = 0; j < NPT; ++j) ba[b * NY + t + j * FTHREADS] = pf[b][j];
        __syncthreads();
        if (g + 1 < nb) {
#pragma unroll
            for (int b = 0; b < TB; ++b) {
                const int l = lb + TB + b;
#pragma unroll
                for (int j = 0; j < NPT; ++j)
                    pf[b][j] = l < nt ? col[(int64_t)l * cs + t + j * FTHREADS] : make_float2(0.f, 0.f);
            }
        }
        const float2 *res = stockham<LOG2NY, false, TB, FTHREADS, 0>(ba, bb, tw);
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            const int l = lb + b;
            if (l >= nt) break;
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                const int k = t + j * FTHREADS;
                float2 v = res[b * NY + k];
                if (l > 0) v = cadd(v, cscale(acc[j], rho_f(th[j], emt[j], q[j], l - 1)));
                acc[j] = v;
                col[(int64_t)l * cs + k] = v;
            }
        }
        __syncthreads();
    }
    // backward sweep: z_{nt-1} = rho y, z_l = rho_l (y_l + z_{l+1}); then inverse y-FFT,
    // batches taken from the top: slices hi-TB+1 .. hi
    int hi = nt - 1;
#pragma unroll
    for (int b = 0; b < TB; ++b)
#pragma unroll
        for (int j = 0; j < NPT; ++j)
            pf[b][j] = hi - b >= 0 ? col[(int64_t)(hi - b) * cs + t + j * FTHREADS] : make_float2(0.f, 0.f);
    for (int g = 0; g < nb; ++g, hi -= TB) {
#pragma unroll
        for (int b = 0; b < TB; ++b) {              // b-th slice from the top of this batch
            const int l = hi - b;
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                float2 v = make_float2(0.f, 0.f);
                if (l >= 0) {
                    float2 y = pf[b][j];
                    if (l < nt - 1) y = cadd(y, acc[j]);
                    acc[j] = cscale(y, rho_f(th[j], emt[j], q[j], l));
                    v = acc[j];
                }
                ba[b * NY + t + j * FTHREADS] = v;
            }
        }
        __syncthreads();
        if (g + 1 < nb) {
#pragma unroll
            for (int b = 0; b < TB; ++b) {
                const int l = hi - TB - b;
#pragma unroll
                for (int j = 0; j < NPT; ++j)
                    pf[b][j] = l >= 0 ? col[(int64_t)l * cs + t + j * FTHREADS] : make_float2(0.f, 0.f);
            }
        }
        const float2 *res = stockham<LOG2NY, true, TB, FTHREADS, 0>(ba, bb, tw);
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            const int l = hi - b;
            if (l < 0) break;
#pragma unroll
            for (int j = 0; j < NPT; ++j) col[(int64_t)l * cs + t + j * FTHREADS] = res[b * NY + t + j * FTHREADS];
        }
        __syncthreads();
    }
}

// ny = 1024 with 256 threads as 4 x 8 x 8 x 4: thread t owns modes t + 256 q
// (q = 0..3), which are exactly the inputs of the first radix-4 stage (span 1) and
// the outputs of the last radix-4 stage (span 256).  Those two stages run in
// registers; the two radix-8 stages between them (spans 4 and 32) go through
// shared memory (radix-8 layout of stockham.cuh: c = 2 after the first two stages,
// c = 0 after the third).  Twiddles (twY): radix-8 span p at (p - 4) + (q-1) p + k,
// radix-4 span 256 at 252 + (q-1) 256 + k.  One slice per step (TB = 1) at 63
// registers: four blocks per SM, so all 513 kx columns are resident at once on the
// 152 SMs (three blocks per SM, with two slices per step, left 57 columns for a
// second wave: 0.898 against 0.857 ms at 1024^2 x 256).
// The recurrence state of the t-solve: float2 and the float32 pivots, or (T64: the
// PDHG_FLAG_T_SOLVE_FP64 variant) double2 and pivots in double, each stored value rounded
// to float once.
template <bool T64> struct TRec;
template <> struct TRec<false> {
    typedef float2 A;
    typedef float R;
    __device__ static R rho(R th, R emt, R q, int l) { return rho_f(th, emt, q, l); }
    __device__ static R ex(R x) { return expf(x); }
    __device__ static A fwd(float2 v, A acc, R r, bool first) { return first ? v : cadd(v, cscale(acc, r)); }
    __device__ static A bwd(float2 y, A acc, R r, bool last) { return cscale(last ? y : cadd(y, acc), r); }
    __device__ static float2 out(A a) { return a; }
    __device__ static A zero() { return make_float2(0.f, 0.f); }
};
template <> struct TRec<true> {
    typedef double2 A;
    typedef double R;
    __device__ static R rho(R th, R emt, R q, int l) {
        const double w = exp(-(double)(2 * l + 1) * th);
        return emt * (1.0 + w) / (1.0 + q * w);
    }
    __device__ static R ex(R x) { return exp(x); }
    __device__ static A fwd(float2 v, A acc, R r, bool first) {
        return first ? make_double2(v.x, v.y) : make_double2((double)v.x + r * acc.x, (double)v.y + r * acc.y);
    }
    __device__ static A bwd(float2 y, A acc, R r, bool last) {
        return last ? make_double2(r * y.x, r * y.y) : make_double2(r * ((double)y.x + acc.x), r * ((double)y.y + acc.y));
    }
    __device__ static float2 out(A a) { return make_float2((float)a.x, (float)a.y); }
    __device__ static A zero() { return make_double2(0.0, 0.0); }
};

template <bool T64>
__global__ void __launch_bounds__(FTHREADS, 4) k_cols1024(Params<float> P, float2 *__restrict__ spec,
                                                       const float2 *__restrict__ twY,
                                                       const float *__restrict__ thetaT) {
    constexpr int LOG2NY = 10, NY = 1024, Q = 256, TB = 1, PN = R8<LOG2NY>::PN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *ba = reinterpret_cast<float2 *>(smem_raw);              // [TB][PN] (padded)
    float2 *bb = ba + TB * PN;                                      // [TB][PN]
    float2 *tw = bb + TB * PN;                                      // [NY]
    const int kx = blockIdx.x;
    const int nt = P.nt;
    const int64_t cs = (int64_t)P.nkx * NY;
    float2 *col = spec + (int64_t)kx * NY;
    const int64_t ncol = (int64_t)nt * P.nkx * NY - (int64_t)kx * NY;     // elements from col to the end
    const int t = threadIdx.x;
    for (int j = t; j < NY; j += FTHREADS) tw[j] = twY[j];
    typedef TRec<T64> TR;
    typename TR::R th[4], emt[4], q4[4];
    typename TR::A acc[4];
    float2 pf[TB][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        th[q] = thetaT[dbg_idx(P, (int64_t)kx * NY + t + q * Q, (int64_t)P.nkx * NY, 302)];
        emt[q] = TR::ex(-th[q]);
        q4[q] = emt[q] * emt[q];
        acc[q] = TR::zero();
    }
    const int nb = (nt + TB - 1) / TB;
    // ---- forward sweep ----
#pragma unroll
    for (int b = 0; b < TB; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) pf[b][q] = b < nt ? col[dbg_idx(P, ((int64_t)b * cs + t + q * Q), ncol, 301)] : make_float2(0.f, 0.f);
    __syncthreads();                                                // twiddles
    for (int g = 0; g < nb; ++g) {
        const int lb = g * TB;
        // stage 1 (span 1) in registers: inputs t + 256 r, outputs 4 t + q
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            float2 x0 = pf[b][0], x1 = pf[b][1], x2 = pf[b][2], x3 = pf[b][3];
            dft4<false>(x0, x1, x2, x3);
            float4 *d = reinterpret_cast<float4 *>(ba + b * PN + padc<2>(4 * t));
            d[0] = make_float4(x0.x, x0.y, x1.x, x1.y);
            d[1] = make_float4(x2.x, x2.y, x3.x, x3.y);
        }
        __syncthreads();
        if (g + 1 < nb) {
#pragma unroll
            for (int b = 0; b < TB; ++b) {
                const int l = lb + TB + b;
#pragma unroll
                for (int q = 0; q < 4; ++q) pf[b][q] = l < nt ? col[dbg_idx(P, ((int64_t)l * cs + t + q * Q), ncol, 301)] : make_float2(0.f, 0.f);
            }
        }
        stage_r8<LOG2NY, false, 4, 2, 2, TB, FTHREADS, 4>(ba, bb, tw);
        __syncthreads();
        stage_r8<LOG2NY, false, 32, 2, 0, TB, FTHREADS, 4>(bb, ba, tw);
        __syncthreads();
        const float2 *res = ba;
        // last stage (radix 4, span 256) in registers: inputs t + 256 r with twiddles W^{r t},
        // outputs t + 256 q
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            const int l = lb + b;
            const float2 *rb = res + b * PN;
            float2 x0 = rb[t];
            float2 x1 = cmul(rb[t + Q], tw[252 + t]);
            float2 x2 = cmul(rb[t + 2 * Q], tw[252 + 256 + t]);
            float2 x3 = cmul(rb[t + 3 * Q], tw[252 + 512 + t]);
            dft4<false>(x0, x1, x2, x3);
            if (l < nt) {
                float2 y[4] = {x0, x1, x2, x3};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[q] = TR::fwd(y[q], acc[q], l > 0 ? TR::rho(th[q], emt[q], q4[q], l - 1) : 0, l == 0);
                    col[dbg_idx(P, ((int64_t)l * cs + t + q * Q), ncol, 301)] = TR::out(acc[q]);
                }
            }
        }
        __syncthreads();                 // res (= ba) takes the next batch's first stage
    }
    // ---- backward sweep (batches from the top) ----
    int hi = nt - 1;
#pragma unroll
    for (int b = 0; b < TB; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            pf[b][q] = hi - b >= 0 ? col[dbg_idx(P, ((int64_t)(hi - b) * cs + t + q * Q), ncol, 301)] : make_float2(0.f, 0.f);
    for (int g = 0; g < nb; ++g, hi -= TB) {
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            const int l = hi - b;
            float2 z[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                z[q] = make_float2(0.f, 0.f);
                if (l >= 0) {
                    acc[q] = TR::bwd(pf[b][q], acc[q], TR::rho(th[q], emt[q], q4[q], l), l == nt - 1);
                    z[q] = TR::out(acc[q]);
                }
            }
            // inverse stage 1 (span 1) in registers
            dft4<true>(z[0], z[1], z[2], z[3]);
            float4 *d = reinterpret_cast<float4 *>(ba + b * PN + padc<2>(4 * t));
            d[0] = make_float4(z[0].x, z[0].y, z[1].x, z[1].y);
            d[1] = make_float4(z[2].x, z[2].y, z[3].x, z[3].y);
        }
        __syncthreads();
        if (g + 1 < nb) {
#pragma unroll
            for (int b = 0; b < TB; ++b) {
                const int l = hi - TB - b;
#pragma unroll
                for (int q = 0; q < 4; ++q) pf[b][q] = l >= 0 ? col[dbg_idx(P, ((int64_t)l * cs + t + q * Q), ncol, 301)] : make_float2(0.f, 0.f);
            }
        }
        stage_r8<LOG2NY, true, 4, 2, 2, TB, FTHREADS, 4>(ba, bb, tw);
        __syncthreads();
        stage_r8<LOG2NY, true, 32, 2, 0, TB, FTHREADS, 4>(bb, ba, tw);
        __syncthreads();
        const float2 *res = ba;
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            const int l = hi - b;
            const float2 *rb = res + b * PN;
            float2 x0 = rb[t];
            float2 x1 = cmulconj(rb[t + Q], tw[252 + t]);
            float2 x2 = cmulconj(rb[t + 2 * Q], tw[252 + 256 + t]);
            float2 x3 = cmulconj(rb[t + 3 * Q], tw[252 + 512 + t]);
            dft4<true>(x0, x1, x2, x3);
            if (l >= 0) {
                col[dbg_idx(P, ((int64_t)l * cs + t), ncol, 301)] = x0;
                col[dbg_idx(P, ((int64_t)l * cs + t + Q), ncol, 301)] = x1;
                col[dbg_idx(P, ((int64_t)l * cs + t + 2 * Q), ncol, 301)] = x2;
                col[dbg_idx(P, ((int64_t)l * cs + t + 3 * Q), ncol, 301)] = x3;
            }
        }
        __syncthreads();                 // res (= ba) takes the next batch's first stage
    }
}

static size_t smem_cols(int log2ny) {
    const size_t n = (size_t)1 << log2ny;
    return log2ny == 10 ? (2 * (size_t)R8<10>::PN + n) * 8 : 5 * n * 8;    // ny = 1024: radix-8 layout
}

// ---------------------------------------------------------------------------
// rows-C: inverse real FFT along x, dual step and extrapolation.  phi is read
// into registers before the FFT so that its latency overlaps the transform.
// ---------------------------------------------------------------------------
template <int LOG2M>
__global__ void __launch_bounds__(FTHREADS) k_rowsC(Params<float> P, const float2 *__restrict__ spec,
                                                    float *__restrict__ phi, float *__restrict__ phit,
                                                    const float2 *__restrict__ twN, const float2 *__restrict__ twM) {
    constexpr int M = 1 << LOG2M, NX = 2 * M;
    constexpr int VPT = FH * NX / 4 / FTHREADS;              // float4 of phi per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int PN = SeqLayout<LOG2M, 2>::PN;           // padded rows (stockham.cuh)
    float2 *fa = reinterpret_cast<float2 *>(smem_raw);      // [FH][PN]
    float2 *fb = fa + FH * PN;                               // staging [FH][M+1], then scratch [FH][PN]
    const int ny = P.ny;
    const int y0 = blockIdx.x * FH;
    const int l = blockIdx.y;
    const int64_t base = (int64_t)l * P.S + (int64_t)y0 * NX;
    float4 ph[VPT];
#pragma unroll
    for (int j = 0; j < VPT; ++j) ph[j] = __ldg(reinterpret_cast<const float4 *>(phi + base) + threadIdx.x + j * FTHREADS);
    // gather [kx][y0..y0+FH) (FH = 4 complex = two float4 per kx)
    const float4 *src = reinterpret_cast<const float4 *>(spec + (int64_t)l * P.nkx * ny + y0);
    for (int idx = threadIdx.x; idx < (M + 1) * 2; idx += blockDim.x) {
        const int k = idx >> 1, h = idx & 1;
        const float4 v = __ldg(src + (int64_t)k * (ny / 2) + h);
        fb[(2 * h) * (M + 1) + k] = make_float2(v.x, v.y);
        fb[(2 * h + 1) * (M + 1) + k] = make_float2(v.z, v.w);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < FH * M; idx += blockDim.x) {
        const int rr = idx / M, k = idx - rr * M;
        fa[rr * PN + padx(k)] = irfft_merge(fb[rr * (M + 1) + k], fb[rr * (M + 1) + M - k], twN[k]);
    }
    __syncthreads();
    const float2 *res = stockham<LOG2M, true, FH, FTHREADS, 2>(fa, fb, twM);
    float4 *p4 = reinterpret_cast<float4 *>(phi + base);
    float4 *t4 = reinterpret_cast<float4 *>(phit + base);
    const float s = P.dual_scale;
    constexpr int V = NX / 4;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
        const int idx = threadIdx.x + j * FTHREADS;
        const int rr = idx / V, x4 = idx - rr * V;
        const float4 z = *reinterpret_cast<const float4 *>(res + rr * PN + padx(2 * x4));
        float4 pn = ph[j];
        pn.x += s * z.x; pn.y += s * z.y; pn.z += s * z.z; pn.w += s * z.w;
        p4[idx] = pn;
        t4[idx] = make_float4(pn.x + s * z.x, pn.y + s * z.y, pn.z + s * z.z, pn.w + s * z.w);
    }
}

// rows-C for nx = 1024 (M = 512 = 2 * 4^4), persistent with a TMA pipeline: a block
// takes the tiles (4 rows of one slice) blockIdx.x, +gridDim.x, ..., and the spectrum
// of the tile two ahead is loaded by TMA (six 3D boxes of 176 kx rows x 2 complex: rows
// y0, y0+1 into one half of the stage buffer and rows y0+2, y0+3 into the other, each
// half [kx][2]) into the stage buffer the current tile has just released, so the
// 32-byte gathers are in flight during the transform.  A thread reads its kx from both
// halves as 16-byte words at consecutive addresses across the warp (no bank conflicts;
// one [kx][4] array read 32 bytes per lane, two wavefronts per quarter warp).
// The inverse split feeds the first (radix-2, span 1) stage directly in registers,
// three radix-4 stages (spans 2, 8, 32) run in shared memory, and the last (span
// 128) runs in registers, whose outputs -- complex positions i + 128 q, i.e.
// x = 2 (i + 128 q) + {0,1} -- go straight into the dual step.  A stage wait that
// gives up after wait_ns sets *err and the block returns (after a bounded wait for
// its copies in flight).
constexpr int RC_BOX = 176;                    // kx rows per TMA box: 3 boxes >= 513 rows, 2816 bytes (128 | size)
constexpr int RC_ROWS = 3 * RC_BOX;            // rows per stage buffer (rows >= nkx are zero-filled)
constexpr uint32_t RC_TX = RC_ROWS * FH * 8;   // bytes per stage, both halves (whole boxes, fill included)
constexpr uint64_t RC_DRAIN_NS = 1000000000ull; // budget of the waits for copies in flight on exit

__global__ void __launch_bounds__(FTHREADS, 3) k_rowsC1024(Params<float> P, const __grid_constant__ CUtensorMap tmap,
                                                           float *__restrict__ phi, float *__restrict__ phit,
                                                           const float2 *__restrict__ twN,
                                                           const float2 *__restrict__ twM, int *__restrict__ err,
                                                           uint64_t wait_ns) {
    constexpr int LOG2M = 9, M = 512, NX = 1024;
    constexpr int PN = SeqLayout<LOG2M, 2>::PN;           // padded rows (stockham.cuh)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // TMA destinations 128-byte aligned (the launch adds 128 bytes of slack)
    unsigned char *sm = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    float2 *stg = reinterpret_cast<float2 *>(sm);           // [2 halves][2 stages][RC_ROWS][2]
    float2 *fa = stg + 2 * RC_ROWS * FH;                     // [FH][PN]
    float2 *fb = fa + FH * PN;                               // [FH][PN]
    uint64_t *bar = reinterpret_cast<uint64_t *>(fb + FH * PN);   // [2]
    const int nyb = P.ny / FH, ntiles = nyb * P.nt, G = gridDim.x;
    const int64_t nF = (int64_t)P.nt * P.S;
    const int t = threadIdx.x;
    auto issue = [&](int tile, int buf) {                    // one thread
        const int l = tile / nyb, yb = tile - l * nyb;
        mbar_arrive_expect_tx(bar + buf, RC_TX);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int hf = 0; hf < 2; ++hf)
                tma_load_3d(stg + ((2 * hf + buf) * RC_ROWS + b * RC_BOX) * 2, &tmap, 2 * FH * yb + 4 * hf,
                            b * RC_BOX, l, bar + buf);
    };
    if (t == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (t == 0) {
        if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
        if ((int)blockIdx.x + G < ntiles) issue(blockIdx.x + G, 1);
    }
    // the positions this thread updates: rows 2h, 2h+1 (h = t / 128), x = 2(i + 128 q) + {0, 1}
    const int h = t >> 7, i = t & 127;
    const float s = P.dual_scale;
    const float2 w0 = twN[t], w1 = twN[t + 256];
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += G, ++it) {
        const int buf = it & 1;
        const int l = tile / nyb, y0 = (tile - l * nyb) * FH;
        const int64_t base = (int64_t)l * P.S + (int64_t)y0 * NX;
        float2 ph[2][4];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                ph[rr][q] = __ldg(reinterpret_cast<const float2 *>(
                    phi + dbg_idx(P, base + (int64_t)(2 * h + rr) * NX + 2 * (i + 128 * q), nF - 1, 401)));
        const bool ok = mbar_wait_bounded(bar + buf, (it >> 1) & 1, wait_ns);
        if (__syncthreads_or(!ok)) {
            if (t == 0) {
                atomicExch(err, 1);
                // this stage's copy and the other stage's, if one was issued, before the block leaves
                mbar_wait_bounded(bar + buf, (it >> 1) & 1, RC_DRAIN_NS);
                if (tile + G < ntiles) mbar_wait_bounded(bar + (buf ^ 1), ((it + 1) >> 1) & 1, RC_DRAIN_NS);
            }
            return;
        }
        // inverse split (Z_k = E_k + i O_k) for k = t and t + 256, then the radix-2 stage
        // (span 1: outputs 2t, 2t+1) in registers; stage halves are [kx][rows 0, 1] and
        // [kx][rows 2, 3]
        {
            const float4 *A4 = reinterpret_cast<const float4 *>(stg + buf * RC_ROWS * 2);
            const float4 *B4 = reinterpret_cast<const float4 *>(stg + (2 + buf) * RC_ROWS * 2);
            const float4 xa[2] = {A4[t], B4[t]};
            const float4 xb[2] = {A4[M - t], B4[M - t]};
            const float4 xc[2] = {A4[t + 256], B4[t + 256]};
            const float4 xd[2] = {A4[256 - t], B4[256 - t]};
#pragma unroll
            for (int rr = 0; rr < FH; ++rr) {
                const int hh = rr >> 1;
                const bool hi = rr & 1;
                const float2 A = hi ? make_float2(xa[hh].z, xa[hh].w) : make_float2(xa[hh].x, xa[hh].y);
                const float2 B = hi ? make_float2(xb[hh].z, xb[hh].w) : make_float2(xb[hh].x, xb[hh].y);
                const float2 C = hi ? make_float2(xc[hh].z, xc[hh].w) : make_float2(xc[hh].x, xc[hh].y);
                const float2 D = hi ? make_float2(xd[hh].z, xd[hh].w) : make_float2(xd[hh].x, xd[hh].y);
                const float2 z0 = irfft_merge(A, B, w0);
                const float2 z1 = irfft_merge(C, D, w1);
                *reinterpret_cast<float4 *>(fa + rr * PN + padx(2 * t)) =
                    make_float4(z0.x + z1.x, z0.y + z1.y, z0.x - z1.x, z0.y - z1.y);
            }
        }
        __syncthreads();
        if (t == 0 && tile + 2 * G < ntiles) {            // the stage buffer is free: next-but-one tile
            fence_proxy_async_smem();
            issue(tile + 2 * G, buf);
        }
        const float2 *res = stockham_r4_range<LOG2M, true, 2, 128, FH, FTHREADS, 2>(fa, fb, twM);
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const float2 *r = res + (2 * h + rr) * PN;
            float2 x0 = r[padx(i)];
            float2 x1 = cmulconj(r[padx(i + 128)], twM[126 + i]);       // staged block of span 128
            float2 x2 = cmulconj(r[padx(i + 256)], twM[126 + 128 + i]);
            float2 x3 = cmulconj(r[padx(i + 384)], twM[126 + 256 + i]);
            dft4<true>(x0, x1, x2, x3);
            const float2 z[4] = {x0, x1, x2, x3};
            const int64_t rb = base + (int64_t)(2 * h + rr) * NX;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 pn = ph[rr][q];
                pn.x += s * z[q].x;
                pn.y += s * z[q].y;
                const int64_t o = dbg_idx(P, rb + 2 * (i + 128 * q), nF - 1, 402);
                *reinterpret_cast<float2 *>(phi + o) = pn;
                *reinterpret_cast<float2 *>(phit + o) = make_float2(pn.x + s * z[q].x, pn.y + s * z[q].y);
            }
        }
    }
}

static size_t smem_rowsC1024() {
    return 128 + (size_t)2 * RC_ROWS * FH * 8 + 2 * (size_t)FH * SeqLayout<9, 2>::PN * 8 + 2 * sizeof(uint64_t);
}

// ---------------------------------------------------------------------------
// residual norms (Eq. 2.12) of a 2D finite-difference state (the fused path, and
// the plain path's 2D handles): the six sums of block_sum6 for slice row
// l = blockIdx.y, one record per block at partials[(l gx + bx) * 6], the layout of
// the generic check, so the same fixed-order reduction follows.  A thread owns four
// consecutive x and PRY rows of a tile (tiles blockIdx.x, +gridDim.x, ...), slides
// three-row windows of u^{l+1} (the equation R^l) and phi^{l-1} (the row l of
// J(u)^T phi) down them, and sums the tile's 16 values in A (float32 for float32
// fields, folded into float64 per tile; float64 for float64 fields).
// ---------------------------------------------------------------------------
template <typename T> struct Q4 { T x, y, z, w; };
__device__ __forceinline__ Q4<float> ld4(const float *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Q4<double> ld4(const double *p) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}

template <typename T, int NX>
__global__ void __launch_bounds__(256) k_check2d(Params<T> P, const T *__restrict__ u, const T *__restrict__ phi,
                                                 const T *__restrict__ lam, const T *__restrict__ u0,
                                                 double *__restrict__ partials) {
    typedef typename std::conditional<sizeof(T) == 4, float, double>::type A;
    constexpr int V = NX / 4, TX = V < 256 ? V : 256, TY = V < 256 ? 256 / V : 1, XS = V / TX;
    const int l = blockIdx.y, nt = P.nt, ny = P.ny;
    const int64_t S = P.S, nU = (int64_t)(nt + 1) * S, nF = (int64_t)nt * S;
    const int xt = threadIdx.x % TX, yt = threadIdx.x / TX;
    const int ntile = (ny / (PRY * TY)) * XS;
    const bool lf = P.space != FD_UPWIND, bdf2 = P.time == BDF2;
    const T zero = T(0), half = T(0.5), two = T(2);
    // R^l = D(u^{l+1}) + kn u^{l+1} + kc u^l + ko u^{l-1}
    const T kn = l < nt ? coef_new(P, l) : zero, kc = l < nt ? coef_cur(P, l) : zero;
    const T ko = (l < nt && bdf2 && l >= 1) ? coef_old(P, l) : zero;
    // (J^T phi)^l = transposed stencil of phi^{l-1} at u^l + cn phi^{l-1} + cc phi^l + co phi^{l+1}
    const T cn = l >= 1 ? coef_new(P, l - 1) : zero, cc = l <= nt - 1 ? coef_cur(P, l) : zero;
    const T co = (bdf2 && l + 1 <= nt - 1) ? coef_old(P, l + 1) : zero;
    auto wrapy = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int x4 = xt + (tile % XS) * TX;
        const int ya = ((tile / XS) * TY + yt) * PRY;
        A part[6] = {0, 0, 0, 0, 0, 0};
        if (l < nt) {
            const int64_t oN = (int64_t)(l + 1) * S, oC = (int64_t)l * S, oO = (int64_t)(l >= 1 ? l - 1 : 0) * S;
            Q4<T> up = ld4(u + dbg_idx(P, oN + (int64_t)wrapy(ya - 1) * NX + 4 * x4, nU - 3, 501));
            Q4<T> v4 = ld4(u + dbg_idx(P, oN + (int64_t)ya * NX + 4 * x4, nU - 3, 501));
#pragma unroll
            for (int r = 0; r < PRY; ++r) {
                const int y = ya + r;
                const int64_t row = oN + (int64_t)y * NX;
                const Q4<T> dn = ld4(u + dbg_idx(P, oN + (int64_t)wrapy(y + 1) * NX + 4 * x4, nU - 3, 501));
                const T lft = __ldg(u + dbg_idx(P, row + (x4 == 0 ? NX - 1 : 4 * x4 - 1), nU, 502));
                const T rgt = __ldg(u + dbg_idx(P, row + (x4 == V - 1 ? 0 : 4 * x4 + 4), nU, 502));
                const int64_t i = (int64_t)y * NX + 4 * x4;
                const Q4<T> cu = ld4(u + dbg_idx(P, oC + i, nU - 3, 503)), p4 = ld4(phi + dbg_idx(P, oC + i, nF - 3, 504));
                Q4<T> o4 = {zero, zero, zero, zero};
                if (ko != zero) o4 = ld4(u + dbg_idx(P, oO + i, nU - 3, 505));
                const T vr[6] = {lft, v4.x, v4.y, v4.z, v4.w, rgt};
                const T uv[4] = {up.x, up.y, up.z, up.w}, dv[4] = {dn.x, dn.y, dn.z, dn.w};
                const T cv[4] = {cu.x, cu.y, cu.z, cu.w}, ov[4] = {o4.x, o4.y, o4.z, o4.w};
                const T pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const T v = vr[e + 1];
                    const T lx = vr[e] - two * v + vr[e + 2], ly = uv[e] - two * v + dv[e];
                    T dx, dy;
                    if (lf) {
                        dx = half * (flux(P, vr[e + 2]) - flux(P, vr[e])) - half * P.lf_a * lx;
                        dy = half * (flux(P, dv[e]) - flux(P, uv[e])) - half * P.lf_a * ly;
                    } else {
                        dx = flux(P, v) - flux(P, vr[e]);
                        dy = flux(P, v) - flux(P, uv[e]);
                    }
                    T rv = dx * P.inv_hx + dy * P.inv_hy + kn * v + kc * cv[e] + ko * ov[e];
                    if (P.nu != zero) rv -= P.nu * (lx * P.inv_hx * P.inv_hx + ly * P.inv_hy * P.inv_hy);
                    part[0] += (A)(rv * rv);
                    part[2] += (A)(pv[e] * rv);
                }
                up = v4;
                v4 = dn;
            }
        }
        if (l >= 1) {
            const int64_t oP = (int64_t)(l - 1) * S, oL = (int64_t)l * S;
            Q4<T> pu = ld4(phi + dbg_idx(P, oP + (int64_t)wrapy(ya - 1) * NX + 4 * x4, nF - 3, 506));
            Q4<T> pm = ld4(phi + dbg_idx(P, oP + (int64_t)ya * NX + 4 * x4, nF - 3, 506));
#pragma unroll
            for (int r = 0; r < PRY; ++r) {
                const int y = ya + r;
                const int64_t row = oP + (int64_t)y * NX;
                const Q4<T> pd = ld4(phi + dbg_idx(P, oP + (int64_t)wrapy(y + 1) * NX + 4 * x4, nF - 3, 506));
                const T lft = __ldg(phi + dbg_idx(P, row + (x4 == 0 ? NX - 1 : 4 * x4 - 1), nF, 507));
                const T rgt = __ldg(phi + dbg_idx(P, row + (x4 == V - 1 ? 0 : 4 * x4 + 4), nF, 507));
                const int64_t i = (int64_t)y * NX + 4 * x4;
                const Q4<T> c = ld4(u + dbg_idx(P, oL + i, nU - 3, 508));
                Q4<T> tc = {zero, zero, zero, zero}, tn = {zero, zero, zero, zero};
                if (cc != zero) tc = ld4(phi + dbg_idx(P, oL + i, nF - 3, 509));
                if (co != zero) tn = ld4(phi + dbg_idx(P, oL + S + i, nF - 3, 510));
                const T pr[6] = {lft, pm.x, pm.y, pm.z, pm.w, rgt};
                const T uv[4] = {pu.x, pu.y, pu.z, pu.w}, dv[4] = {pd.x, pd.y, pd.z, pd.w};
                const T cv[4] = {c.x, c.y, c.z, c.w};
                const T gv[4] = {cc * tc.x + co * tn.x, cc * tc.y + co * tn.y, cc * tc.z + co * tn.z,
                                 cc * tc.w + co * tn.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const T p0 = pr[e + 1], df = dflux(P, cv[e]);
                    const T mx = pr[e], qx = pr[e + 2], my = uv[e], qy = dv[e];
                    T tx, ty;
                    if (lf) {
                        tx = half * (df * (mx - qx) + P.lf_a * (two * p0 - mx - qx));
                        ty = half * (df * (my - qy) + P.lf_a * (two * p0 - my - qy));
                    } else {
                        tx = df * (p0 - qx);
                        ty = df * (p0 - qy);
                    }
                    T g = gv[e] + cn * p0 + tx * P.inv_hx + ty * P.inv_hy;
                    if (P.nu != zero)
                        g -= P.nu * ((qx - two * p0 + mx) * P.inv_hx * P.inv_hx + (qy - two * p0 + my) * P.inv_hy * P.inv_hy);
                    part[1] += (A)(g * g);
                }
                pu = pm;
                pm = pd;
            }
        } else {
            // the initial row: u^0 - u0, and h_t (J^T phi)^0 + lambda (its time part only)
#pragma unroll
            for (int r = 0; r < PRY; ++r) {
                const int64_t i = (int64_t)(ya + r) * NX + 4 * x4;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int64_t k0 = dbg_idx(P, i + e, S, 511);
                    const double r0 = (double)u[k0] - (double)u0[k0];
                    part[3] += (A)(r0 * r0);
                    if (P.init == INIT_LAMBDA) {
                        const T t0 = cc * phi[k0] + (co != zero ? co * phi[dbg_idx(P, S + i + e, nF, 512)] : zero);
                        const double g0 = (double)P.ht * (double)t0 + (double)lam[k0];
                        part[4] += (A)(g0 * g0);
                        part[5] += (A)((double)lam[k0] * r0);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] += (double)part[k];
    }
    block_sum6(acc, partials + ((int64_t)l * gridDim.x + blockIdx.x) * 6);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int ilog2i(int64_t v) { int r = 0; while ((int64_t(1) << r) < v) ++r; return r; }

bool fused2d_supported(int dims, int space, int time, int prec, int64_t nx, int64_t ny, int64_t nt, double nu) {
    (void)nu;
    if (dims != 2 || prec != 1) return false;
    if (space != FD_UPWIND && space != FD_LF) return false;
    if (nt < 1) return false;
    auto p2 = [](int64_t v) { return v > 0 && (v & (v - 1)) == 0; };
    if (time == BDF2 && nx > 1024) return false;     // three u slots no longer fit shared memory
    return p2(nx) && p2(ny) && nx >= 256 && nx <= 2048 && ny >= 256 && ny <= 1024;
}

static size_t al(size_t v) { return (v + 255) & ~size_t(255); }

size_t fused2d_workspace_bytes(int64_t nx, int64_t ny, int64_t nt) {
    const int64_t nkx = nx / 2 + 1;
    return al(4) +                             // error flag of the pipelined rows-C
           al(nt * nkx * ny * 8) +             // spectrum [l][kx][y]
           al(nx / 2 * 8) + al(ny * 8) +       // twiddles W_M, W_ny
           al(nx / 2 * 8) +                    // radix-8 twiddles W_M
           al(nkx * ny * 4);                   // theta [kx][ky]
}

void fused2d_layout(Fused2D *f, void *ws, int64_t nx, int64_t ny, int64_t nt) {
    const int64_t nkx = nx / 2 + 1;
    char *p = (char *)ws;
    f->err = (int *)p; p += al(4);
    f->spec = (float2 *)p; p += al(nt * nkx * ny * 8);
    f->twM = (float2 *)p; p += al(nx / 2 * 8);
    f->twY = (float2 *)p; p += al(ny * 8);
    f->twM8 = (float2 *)p; p += al(nx / 2 * 8);
    f->thetaT = (float *)p;
}

static size_t smem_rowsR(int log2m, bool bdf2) {
    const int M = 1 << log2m, NX = 2 * M, PN = M + M / 8 + 4;     // R8<log2m>::PN
    return (size_t)(bdf2 ? 3 : 2) * (FH + 2) * NX * 4 + (size_t)FH * PN * 8;
}
static size_t smem_rowsC(int log2m) {
    const int M = 1 << log2m, PN = M + M / 4 + 4;                // SeqLayout<log2m, 2>::PN
    return (size_t)FH * PN * 8 * 2;
}

static cudaError_t attr_rows1024() {
    cudaError_t e = cudaFuncSetAttribute(k_rowsR1024<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_rowsR1024());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_rowsR1024<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rowsR1024());
    return e;
}

template <int L> static cudaError_t attr_rows() {
    cudaError_t e = cudaFuncSetAttribute(k_rowsR<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_rowsR(L, false));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_rowsR<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rowsR(L, true));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_rowsC<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rowsC(L));
    return e;
}

// Resident rows-R blocks on the whole device (occupancy x multiprocessors).
template <int L> static cudaError_t rowsR_slots(const Params<float> &P, Fused2D *f) {
    int per_sm = 0;
    const bool b2 = P.time == BDF2;
    cudaError_t e;
    if (L == 9)
        e = b2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowsR1024<true>, ATHREADS, smem_rowsR1024())
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowsR1024<false>, ATHREADS, smem_rowsR1024());
    else
        e = b2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowsR<L, true>, ATHREADS, smem_rowsR(L, true))
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowsR<L, false>, ATHREADS, smem_rowsR(L, false));
    f->rows_slots = std::max(1, per_sm) * f->nsm;
    return e;
}

// Time slices per rows-R block.  A block of tc slices marches tc + 1 steps (tc + 2
// for BDF2); nb = rows x ceil(nt / tc) blocks run in ceil(nb / slots) rounds of the
// resident slots, so the launch takes about rounds x (tc + 1) steps: the chunk
// minimising that avoids a nearly empty last round (at 1024^2 x 256 on 152 SMs with
// three blocks each, 32 slices give 4.5 rounds, 37 give 3.9).
int rowsR_chunk(int nt, int rows, int slots, bool bdf2) {
    if (nt < 8) return 2;
    int best = 8;
    double best_cost = 1e300;
    for (int tc = 8; tc <= std::min(nt, 64); ++tc) {
        const int64_t nb = (int64_t)rows * ((nt + tc - 1) / tc);
        const int64_t rounds = (nb + slots - 1) / slots;
        const double cost = (double)rounds * (tc + 1 + (bdf2 ? 1 : 0));
        if (cost <= best_cost) { best_cost = cost; best = tc; }      // ties: the longer chunk
    }
    return best;
}

cudaError_t fused2d_init(Fused2D *f, const Params<float> &P, void *ws, const float *twx, const float *twy,
                         const float *theta) {
    (void)twy; (void)theta;
    cudaError_t ec = cudaFuncSetAttribute(k_cols1024<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_cols(10));
    if (ec == cudaSuccess)
        ec = cudaFuncSetAttribute(k_cols1024<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols(10));
    if (ec == cudaSuccess)
        ec = cudaFuncSetAttribute(k_rowsC1024, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rowsC1024());
    if (ec != cudaSuccess) return ec;
    fused2d_layout(f, ws, P.nx, P.ny, P.nt);
    f->twN = (const float2 *)twx;
    f->wait_ns = FUSED2D_WAIT_NS_DEFAULT;
    {
        int dev = 0;
        ec = cudaGetDevice(&dev);
        if (ec == cudaSuccess) ec = cudaDeviceGetAttribute(&f->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (ec == cudaSuccess) ec = cudaMemset(f->err, 0, sizeof(int));
        if (ec != cudaSuccess) return ec;
    }
    if (P.nx == 1024) {
        // the spectrum as a 3D float32 tensor [nt][nkx][2 ny] for rows-C's TMA boxes
        // of 2 complex (4 floats, 16 bytes) x RC_BOX kx rows x 1 slice
        typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                      const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                      CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        ec = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (ec != cudaSuccess) return ec;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        const cuuint64_t dims[3] = {(cuuint64_t)(2 * P.ny), (cuuint64_t)P.nkx, (cuuint64_t)P.nt};
        const cuuint64_t strides[2] = {(cuuint64_t)(2 * P.ny * 4), (cuuint64_t)P.nkx * (cuuint64_t)(2 * P.ny * 4)};
        const cuuint32_t box[3] = {4, RC_BOX, 1}, estr[3] = {1, 1, 1};
        CUresult r = ((encode_fn)fn)(&f->tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, f->spec, dims, strides, box,
                                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    switch (ilog2i(P.nx / 2)) {
    case 7: ec = attr_rows<7>(); if (ec == cudaSuccess) ec = rowsR_slots<7>(P, f); break;
    case 8: ec = attr_rows<8>(); if (ec == cudaSuccess) ec = rowsR_slots<8>(P, f); break;
    case 9:
        ec = attr_rows<9>();
        if (ec == cudaSuccess) ec = attr_rows1024();
        if (ec == cudaSuccess) ec = rowsR_slots<9>(P, f);
        break;
    case 10: ec = attr_rows<10>(); if (ec == cudaSuccess) ec = rowsR_slots<10>(P, f); break;
    default: return cudaErrorInvalidValue;
    }
    if (ec != cudaSuccess) return ec;
    f->tc = rowsR_chunk(P.nt, P.ny / FH, f->rows_slots, P.time == BDF2);
    return cudaSuccess;
}

template <int L>
static cudaError_t launch_rowsR(const Fused2D *f, const Params<float> &P, const float *u, cudaStream_t s) {
    dim3 grid((unsigned)(P.ny / FH), (unsigned)((P.nt + f->tc - 1) / f->tc));
    if (L == 9) {
        if (P.time == BDF2)
            k_rowsR1024<true><<<grid, ATHREADS, smem_rowsR1024(), s>>>(P, u, f->spec, f->twN, f->twM8, f->tc);
        else
            k_rowsR1024<false><<<grid, ATHREADS, smem_rowsR1024(), s>>>(P, u, f->spec, f->twN, f->twM8, f->tc);
        return cudaGetLastError();
    }
    if (P.time == BDF2)
        k_rowsR<L, true><<<grid, ATHREADS, smem_rowsR(L, true), s>>>(P, u, f->spec, f->twN, f->twM8, f->tc);
    else
        k_rowsR<L, false><<<grid, ATHREADS, smem_rowsR(L, false), s>>>(P, u, f->spec, f->twN, f->twM8, f->tc);
    return cudaGetLastError();
}

template <int NX>
static cudaError_t launch_primal2d(const Params<float> &P, float *u, const float *phit, float *lam, float *lamt,
                                   const float *u0, cudaStream_t s) {
    constexpr int V = NX / 4;
    const dim3 block(V < 256 ? V : 256, V < 256 ? 256 / V : 1);
    const dim3 grid((unsigned)(P.ny / (PRY * (int)block.y)), (unsigned)(P.nt + 1), V > 256 ? V / 256 : 1);
    k_primal2d<NX><<<grid, block, 0, s>>>(P, u, phit, lam, lamt, u0);
    return cudaGetLastError();
}

template <int L>
static cudaError_t launch_rowsC(const Fused2D *f, const Params<float> &P, float *phi, float *phit, cudaStream_t s) {
    dim3 grid((unsigned)(P.ny / FH), (unsigned)P.nt);
    k_rowsC<L><<<grid, FTHREADS, smem_rowsC(L), s>>>(P, f->spec, phi, phit, f->twN, f->twM);
    return cudaGetLastError();
}

cudaError_t fused2d_primal(const Params<float> &P, float *u, const float *phit, float *lam, float *lamt,
                           const float *u0, cudaStream_t s) {
    switch (P.nx) {
    case 256: return launch_primal2d<256>(P, u, phit, lam, lamt, u0, s);
    case 512: return launch_primal2d<512>(P, u, phit, lam, lamt, u0, s);
    case 1024: return launch_primal2d<1024>(P, u, phit, lam, lamt, u0, s);
    case 2048: return launch_primal2d<2048>(P, u, phit, lam, lamt, u0, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
bool check2d_applies(const Params<T> &P) {
    const bool nx_ok = P.nx == 256 || P.nx == 512 || P.nx == 1024 || P.nx == 2048;
    const int rows_per_tile = PRY * (P.nx / 4 < 256 ? 256 / (P.nx / 4) : 1);
    return P.dims == 2 && (P.space == FD_UPWIND || P.space == FD_LF) && nx_ok && P.ny % rows_per_tile == 0 &&
           !P.ulin && !P.tshift && !P.gamma_half;
}

template <typename T>
cudaError_t launch_check2d(const Params<T> &P, const T *u, const T *phi, const T *lam, const T *u0,
                           double *partials, int gx, cudaStream_t s) {
    const dim3 grid((unsigned)gx, (unsigned)(P.nt + 1));
    switch (P.nx) {
    case 256: k_check2d<T, 256><<<grid, 256, 0, s>>>(P, u, phi, lam, u0, partials); break;
    case 512: k_check2d<T, 512><<<grid, 256, 0, s>>>(P, u, phi, lam, u0, partials); break;
    case 1024: k_check2d<T, 1024><<<grid, 256, 0, s>>>(P, u, phi, lam, u0, partials); break;
    case 2048: k_check2d<T, 2048><<<grid, 256, 0, s>>>(P, u, phi, lam, u0, partials); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template bool check2d_applies<float>(const Params<float> &);
template bool check2d_applies<double>(const Params<double> &);
template cudaError_t launch_check2d<float>(const Params<float> &, const float *, const float *, const float *,
                                           const float *, double *, int, cudaStream_t);
template cudaError_t launch_check2d<double>(const Params<double> &, const double *, const double *, const double *,
                                            const double *, double *, int, cudaStream_t);

cudaError_t fused2d_rowsR(Fused2D *f, const Params<float> &P, const float *u, cudaStream_t s) {
    switch (ilog2i(P.nx / 2)) {
    case 7: return launch_rowsR<7>(f, P, u, s);
    case 8: return launch_rowsR<8>(f, P, u, s);
    case 9: return launch_rowsR<9>(f, P, u, s);
    case 10: return launch_rowsR<10>(f, P, u, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t fused2d_cols(Fused2D *f, const Params<float> &P, cudaStream_t s) {
    const unsigned grid = (unsigned)P.nkx;
    switch (ilog2i(P.ny)) {
    case 8: k_cols<8><<<grid, FTHREADS, smem_cols(8), s>>>(P, f->spec, f->twY, f->thetaT); break;
    case 9: k_cols<9><<<grid, FTHREADS, smem_cols(9), s>>>(P, f->spec, f->twY, f->thetaT); break;
    case 10:
        if (P.t64) k_cols1024<true><<<grid, FTHREADS, smem_cols(10), s>>>(P, f->spec, f->twY, f->thetaT);
        else k_cols1024<false><<<grid, FTHREADS, smem_cols(10), s>>>(P, f->spec, f->twY, f->thetaT);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t fused2d_rowsC(Fused2D *f, const Params<float> &P, float *phi, float *phit, cudaStream_t s) {
    if (P.nx == 1024) {
        const int64_t ntiles = (int64_t)(P.ny / FH) * P.nt;
        const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)f->nsm * 3);
        k_rowsC1024<<<grid, FTHREADS, smem_rowsC1024(), s>>>(P, f->tmC, phi, phit, f->twN, f->twM, f->err,
                                                              f->wait_ns);
        return cudaGetLastError();
    }
    switch (ilog2i(P.nx / 2)) {
    case 7: return launch_rowsC<7>(f, P, phi, phit, s);
    case 8: return launch_rowsC<8>(f, P, phi, phit, s);
    case 9: return launch_rowsC<9>(f, P, phi, phit, s);
    case 10: return launch_rowsC<10>(f, P, phi, phit, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pdhg

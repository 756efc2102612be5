// kernels_fused2d.cu -- the fused iteration of Algorithm 1 (Sec. 3.3) for 2D
// finite differences in float32: three kernels per iteration.
//
//   rows-A  (row blocks of H rows x a chunk of time slices, marching in t)
//           primal step u^n = u^{n-1} - tau_u J(u^{n-1})^T phit^{n-1} on the
//           block's rows plus one halo row on each side, residual R^{l}(u^n)
//           on the block's rows, real FFT along x of each residual row, and a
//           transposed store of the spectrum (layout [l][kx][y]).
//   cols    (one kx column per block, marching in t forward then backward)
//           complex FFT along y, forward elimination of (T_t + kappa h_t^2)
//           per mode with the spill written in place, back substitution, and
//           inverse FFT along y, written in place: the x-spectrum of z.
//   rows-C  (H rows x one slice per block) inverse real FFT along x, dual
//           step phi^n = phi^{n-1} + tau_phi z and extrapolation phit = phi^n + tau_phi z.
//
// u is double-buffered (rows-A reads u^{n-1} from one buffer and writes u^n
// to the other) because a block recomputes its neighbours' halo rows.
#include "fused2d.h"
#include "fft_smem.cuh"
#include "stockham.cuh"

namespace pdhg {

constexpr int FH = 4;          // rows per block in the row kernels
constexpr int FTHREADS = 256;

// ---------------------------------------------------------------------------
// rows-A
// Shared memory per block (x fastest):
//   ph  [2][FH+4][NX]  phit^{m-1}, phit^m rows y0-2 .. y0+FH+1 (a ring over m)
//   us  [NR][FH+2][NX] u rows y0-1 .. y0+FH: raw u^m, then u^n in place (ring)
// The FFT input aliases the u slot that the residual no longer needs and the
// FFT scratch aliases the phit slot of m-1, so BE needs 2 x 112 KB at nx = 1024.
// Each step loads its rows with independent float4 loads (one latency per
// step) before computing.
// ---------------------------------------------------------------------------
template <int NX>
__device__ __forceinline__ void load_rows(float *dst, const float *__restrict__ src_slice, int ybase, int nrows,
                                          int ny, bool zero) {
    constexpr int V = NX / 4;
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int idx = threadIdx.x; idx < nrows * V; idx += blockDim.x) {
        const int r = idx / V, c = idx - r * V;
        int y = ybase + r;
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        d4[idx] = zero ? make_float4(0.f, 0.f, 0.f, 0.f)
                       : __ldg(reinterpret_cast<const float4 *>(src_slice + (int64_t)y * NX) + c);
    }
}

template <int LOG2M, bool BDF2_>
__global__ void __launch_bounds__(FTHREADS) k_rowsA(Params<float> P, const float *__restrict__ u_in,
                                                    float *__restrict__ u_out, const float *__restrict__ phit,
                                                    float *__restrict__ lam, float *__restrict__ lamt,
                                                    const float *__restrict__ u0, float2 *__restrict__ spec,
                                                    const float2 *__restrict__ twN, const float2 *__restrict__ twM,
                                                    int Tc) {
    constexpr int M = 1 << LOG2M, NX = 2 * M;
    constexpr int NR = BDF2_ ? 3 : 2;            // u ring slots
    constexpr int RU = FH + 2;                   // u rows: block rows + one halo row each side
    constexpr int RP = FH + 4;                   // phit rows: two halo rows each side
    constexpr int RPT = FH * NX / FTHREADS;      // residual values per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *ph = reinterpret_cast<float *>(smem_raw);            // [2][RP][NX]
    float *us = ph + 2 * RP * NX;                                // [NR][RU][NX]

    const int ny = P.ny, nt = P.nt;
    const int64_t S = P.S;
    const int y0 = blockIdx.x * FH;
    const int l0 = blockIdx.y * Tc;
    const int l1 = min(l0 + Tc, nt);              // residual slices [l0, l1)
    const int mstart = (BDF2_ && l0 > 0) ? l0 - 1 : l0;

    if (mstart >= 1) load_rows<NX>(ph + ((mstart - 1) & 1) * RP * NX, phit + (int64_t)(mstart - 1) * S, y0 - 2, RP, ny, false);
    for (int m = mstart; m <= l1; ++m) {
        float *pc = ph + (m & 1) * RP * NX;              // phit^m
        float *pp = ph + ((m + 1) & 1) * RP * NX;        // phit^{m-1}
        float *uc = us + (m % NR) * RU * NX;             // u^m -> u^n
        // (0) rows of this step
        load_rows<NX>(pc, phit + (int64_t)m * S, y0 - 2, RP, ny, m >= nt);
        load_rows<NX>(uc, u_in + (int64_t)m * S, y0 - 1, RU, ny, false);
        __syncthreads();
        // (1) primal step on slice m, rows y0-1 .. y0+FH (in place in uc)
        const bool own_write = (m >= l0) && (m < l1 || m == nt);
        const float cn = m >= 1 ? coef_new(P, m - 1) : 0.f;
        const float cc = m <= nt - 1 ? coef_cur(P, m) : 0.f;
        const float co = (BDF2_ && m + 1 <= nt - 1) ? coef_old(P, m + 1) : 0.f;
        for (int idx = threadIdx.x; idx < RU * NX; idx += blockDim.x) {
            const int r = idx / NX, x = idx - r * NX;
            const bool own = (r >= 1 && r <= FH);
            if (m == 0 && !own) continue;                      // slice-0 halo is never read
            const int q = r + 1;                               // phit row of the same y
            const float c = uc[idx];
            // the phit^{m-1} slot is not loaded for m = 0: never read it there
            float g = cc * pc[q * NX + x];
            if (m >= 1) g += cn * pp[q * NX + x];
            if (BDF2_ && co != 0.f) {
                int y = y0 - 1 + r;
                y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
                g += co * __ldg(phit + (int64_t)(m + 1) * S + (int64_t)y * NX + x);
            }
            float un = c;
            if (m >= 1) {
                const int xm = x == 0 ? NX - 1 : x - 1, xp = x == NX - 1 ? 0 : x + 1;
                const float *row = pp + q * NX;
                g += fd_dir_T(P, c, row[xm], row[x], row[xp], P.inv_hx) +
                     fd_dir_T(P, c, pp[(q - 1) * NX + x], row[x], pp[(q + 1) * NX + x], P.inv_hy);
                un = c - P.tau_u * g;
            } else if (P.init == INIT_LAMBDA) {
                const int64_t i = (int64_t)(y0 - 1 + r) * NX + x;    // own rows only: no wrap
                un = c - P.tau_u0 * (P.ht * g + lamt[i]);
                const float r0 = un - u0[i];
                const float ln = lam[i] + P.tau_lambda * r0;
                lam[i] = ln;
                lamt[i] = ln + P.tau_lambda * r0;
            }
            uc[idx] = un;
            if (own && own_write) u_out[(int64_t)m * S + (int64_t)(y0 - 1 + r) * NX + x] = un;
        }
        __syncthreads();
        // (2) residual R^{m-1} on the block's rows, then its x-FFT
        const int lr = m - 1;
        if (lr >= l0 && lr < l1) {
            const float *un = uc;
            const float *ucur = us + ((m + NR - 1) % NR) * RU * NX;
            const float *uold = us + ((m + NR - 2) % NR) * RU * NX;
            const float kn = coef_new(P, lr), kc = coef_cur(P, lr), ko = coef_old(P, lr);
            float R[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const int idx = threadIdx.x + j * FTHREADS;
                const int rr = idx / NX, x = idx - rr * NX;
                const int r = rr + 1;
                const int xm = x == 0 ? NX - 1 : x - 1, xp = x == NX - 1 ? 0 : x + 1;
                const float v = un[r * NX + x];
                float Rv = fd_dir(P, un[r * NX + xm], v, un[r * NX + xp], P.inv_hx) +
                           fd_dir(P, un[(r - 1) * NX + x], v, un[(r + 1) * NX + x], P.inv_hy);
                Rv += kn * v + kc * ucur[r * NX + x];
                if (BDF2_ && lr >= 1) Rv += ko * uold[r * NX + x];
                R[j] = Rv;
            }
            __syncthreads();
            // FFT input in the u slot the residual no longer needs (BE: u^{m-1}, BDF2: u^{m-2}),
            // FFT scratch in the phit slot of m-1
            float *fin = BDF2_ ? const_cast<float *>(uold) : const_cast<float *>(ucur);
#pragma unroll
            for (int j = 0; j < RPT; ++j) fin[threadIdx.x + j * FTHREADS] = R[j];   // z_n = R_{2n} + i R_{2n+1}
            __syncthreads();
            const float2 *res = stockham<LOG2M, false>(reinterpret_cast<float2 *>(fin),
                                                       reinterpret_cast<float2 *>(pp), FH, twM);
            float2 *dst = spec + (int64_t)lr * P.nkx * ny + y0;
            for (int idx = threadIdx.x; idx < (M + 1) * FH; idx += blockDim.x) {
                const int k = idx / FH, rr = idx - k * FH;
                dst[(int64_t)k * ny + rr] = rfft_split(res + rr * M, M, k, twN);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// cols: y-FFT, t-solve per mode (closed-form pivots, see kernels_plain.cu),
// inverse y-FFT; spectrum, spill and result share one buffer, in place.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rho_f(float th, float emt, float q, int l) {
    const float w = expf(-(float)(2 * l + 1) * th);
    return emt * (1.f + w) / (1.f + q * w);
}

template <int LOG2NY>
__global__ void __launch_bounds__(FTHREADS) k_cols(Params<float> P, float2 *__restrict__ spec,
                                                   const float2 *__restrict__ twY,
                                                   const float *__restrict__ thetaT) {
    // CW kx columns per block: the transforms of both run as one batch, so every
    // barrier covers twice the work and twice the loads are in flight.
    constexpr int NY = 1 << LOG2NY;
    constexpr int CW = 2;
    constexpr int NPT = CW * NY / FTHREADS > 0 ? CW * NY / FTHREADS : 1;
    __shared__ __align__(16) float2 ba[CW * NY];
    __shared__ __align__(16) float2 bb[CW * NY];
    __shared__ __align__(16) float2 tw[NY];
    const int kx0 = blockIdx.x * CW;
    const int ncol = min(CW, P.nkx - kx0);
    const int nt = P.nt;
    const int64_t cs = (int64_t)P.nkx * NY;      // slice stride of the spectrum
    float2 *base = spec + (int64_t)kx0 * NY;     // CW columns are contiguous: [kx][y]
    const int t = threadIdx.x;
    for (int j = t; j < NY; j += FTHREADS) tw[j] = twY[j];
    float th[NPT], emt[NPT], q[NPT];
    float2 acc[NPT], pf[NPT];
    bool act[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int e = t + j * FTHREADS;          // element of the batch: column e / NY, mode e % NY
        act[j] = e < ncol * NY;
        th[j] = act[j] ? thetaT[(int64_t)kx0 * NY + e] : 0.f;
        emt[j] = expf(-th[j]);
        q[j] = emt[j] * emt[j];
        acc[j] = make_float2(0.f, 0.f);
        pf[j] = act[j] ? base[e] : make_float2(0.f, 0.f);
    }
    // forward sweep: y_l = r_l + rho_{l-1} y_{l-1}
    for (int l = 0; l < nt; ++l) {
#pragma unroll
        for (int j = 0; j < NPT; ++j) ba[t + j * FTHREADS] = pf[j];
        __syncthreads();
        if (l + 1 < nt) {
#pragma unroll
            for (int j = 0; j < NPT; ++j)
                if (act[j]) pf[j] = base[(int64_t)(l + 1) * cs + t + j * FTHREADS];
        }
        const float2 *res = stockham<LOG2NY, false>(ba, bb, CW, tw);
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const int e = t + j * FTHREADS;
            float2 v = res[e];
            if (l > 0) v = cadd(v, cscale(acc[j], rho_f(th[j], emt[j], q[j], l - 1)));
            acc[j] = v;
            if (act[j]) base[(int64_t)l * cs + e] = v;
        }
        __syncthreads();
    }
    // backward sweep: z_{nt-1} = rho y, z_l = rho_l (y_l + z_{l+1}); then inverse y-FFT
#pragma unroll
    for (int j = 0; j < NPT; ++j) pf[j] = act[j] ? base[(int64_t)(nt - 1) * cs + t + j * FTHREADS] : pf[j];
    for (int l = nt - 1; l >= 0; --l) {
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            float2 y = pf[j];
            if (l < nt - 1) y = cadd(y, acc[j]);
            acc[j] = cscale(y, rho_f(th[j], emt[j], q[j], l));
            ba[t + j * FTHREADS] = acc[j];
        }
        __syncthreads();
        if (l > 0) {
#pragma unroll
            for (int j = 0; j < NPT; ++j)
                if (act[j]) pf[j] = base[(int64_t)(l - 1) * cs + t + j * FTHREADS];
        }
        const float2 *res = stockham<LOG2NY, true>(ba, bb, CW, tw);
#pragma unroll
        for (int j = 0; j < NPT; ++j)
            if (act[j]) base[(int64_t)l * cs + t + j * FTHREADS] = res[t + j * FTHREADS];
        __syncthreads();
    }
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
    float2 *fa = reinterpret_cast<float2 *>(smem_raw);      // [FH][M]
    float2 *fb = fa + FH * (M + 1);                          // staging [FH][M+1], then scratch
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
        fa[rr * M + k] = irfft_merge(fb[rr * (M + 1) + k], fb[rr * (M + 1) + M - k], twN[k]);
    }
    __syncthreads();
    const float2 *res = stockham<LOG2M, true>(fa, fb, FH, twM);
    const float4 *z4 = reinterpret_cast<const float4 *>(res);
    float4 *p4 = reinterpret_cast<float4 *>(phi + base);
    float4 *t4 = reinterpret_cast<float4 *>(phit + base);
    const float s = P.dual_scale;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
        const int idx = threadIdx.x + j * FTHREADS;
        const float4 z = z4[idx];
        float4 pn = ph[j];
        pn.x += s * z.x; pn.y += s * z.y; pn.z += s * z.z; pn.w += s * z.w;
        p4[idx] = pn;
        t4[idx] = make_float4(pn.x + s * z.x, pn.y + s * z.y, pn.z + s * z.z, pn.w + s * z.w);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int ilog2i(int64_t v) { int r = 0; while ((int64_t(1) << r) < v) ++r; return r; }

bool fused2d_supported(int dims, int space, int time, int prec, int64_t nx, int64_t ny, int64_t nt, double nu) {
    (void)nu;
    if (dims != 2 || prec != 1) return false;
    if (space != FD_UPWIND && space != FD_LF) return false;
    if (nt < 2) return false;
    auto p2 = [](int64_t v) { return v > 0 && (v & (v - 1)) == 0; };
    if (time == BDF2 && nx > 1024) return false;     // three u slots no longer fit shared memory
    return p2(nx) && p2(ny) && nx >= 256 && nx <= 2048 && ny >= 256 && ny <= 1024;
}

static size_t al(size_t v) { return (v + 255) & ~size_t(255); }

size_t fused2d_workspace_bytes(int64_t nx, int64_t ny, int64_t nt) {
    const int64_t S = nx * ny, nkx = nx / 2 + 1;
    return al((nt + 1) * S * 4) +              // second u buffer
           al(nt * nkx * ny * 8) +             // spectrum [l][kx][y]
           al(nx / 2 * 8) + al(ny * 8) +       // twiddles W_M, W_ny
           al(nkx * ny * 4);                   // theta [kx][ky]
}

void fused2d_layout(Fused2D *f, void *ws, int64_t nx, int64_t ny, int64_t nt) {
    const int64_t S = nx * ny, nkx = nx / 2 + 1;
    char *p = (char *)ws;
    f->u2 = (float *)p; p += al((nt + 1) * S * 4);
    f->spec = (float2 *)p; p += al(nt * nkx * ny * 8);
    f->twM = (float2 *)p; p += al(nx / 2 * 8);
    f->twY = (float2 *)p; p += al(ny * 8);
    f->thetaT = (float *)p;
}

static size_t smem_rowsA(int log2m, bool bdf2) {
    const int M = 1 << log2m, NX = 2 * M;
    return (size_t)2 * (FH + 4) * NX * 4 + (size_t)(bdf2 ? 3 : 2) * (FH + 2) * NX * 4;
}
static size_t smem_rowsC(int log2m) {
    const int M = 1 << log2m;
    return (size_t)FH * (M + 1) * 8 * 2;
}

template <int L> static cudaError_t attr_rows() {
    cudaError_t e = cudaFuncSetAttribute(k_rowsA<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_rowsA(L, false));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_rowsA<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rowsA(L, true));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_rowsC<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rowsC(L));
    return e;
}

cudaError_t fused2d_init(Fused2D *f, const Params<float> &P, void *ws, const float *twx, const float *twy,
                         const float *theta) {
    (void)twy; (void)theta;
    fused2d_layout(f, ws, P.nx, P.ny, P.nt);
    f->twN = (const float2 *)twx;
    f->cur = 0;
    f->tc = P.nt >= 64 ? 32 : (P.nt >= 8 ? 8 : 2);
    switch (ilog2i(P.nx / 2)) {
    case 7: return attr_rows<7>();
    case 8: return attr_rows<8>();
    case 9: return attr_rows<9>();
    case 10: return attr_rows<10>();
    default: return cudaErrorInvalidValue;
    }
}

template <int L>
static cudaError_t launch_rowsA(const Fused2D *f, const Params<float> &P, const float *uin, float *uout,
                                const float *phit, float *lam, float *lamt, const float *u0, cudaStream_t s) {
    dim3 grid((unsigned)(P.ny / FH), (unsigned)((P.nt + f->tc - 1) / f->tc));
    if (P.time == BDF2)
        k_rowsA<L, true><<<grid, FTHREADS, smem_rowsA(L, true), s>>>(P, uin, uout, phit, lam, lamt, u0, f->spec,
                                                                     f->twN, f->twM, f->tc);
    else
        k_rowsA<L, false><<<grid, FTHREADS, smem_rowsA(L, false), s>>>(P, uin, uout, phit, lam, lamt, u0, f->spec,
                                                                       f->twN, f->twM, f->tc);
    return cudaGetLastError();
}

template <int L>
static cudaError_t launch_rowsC(const Fused2D *f, const Params<float> &P, float *phi, float *phit, cudaStream_t s) {
    dim3 grid((unsigned)(P.ny / FH), (unsigned)P.nt);
    k_rowsC<L><<<grid, FTHREADS, smem_rowsC(L), s>>>(P, f->spec, phi, phit, f->twN, f->twM);
    return cudaGetLastError();
}

cudaError_t fused2d_rowsA(Fused2D *f, const Params<float> &P, const float *uin, float *uout, const float *phit,
                          float *lam, float *lamt, const float *u0, cudaStream_t s) {
    switch (ilog2i(P.nx / 2)) {
    case 7: return launch_rowsA<7>(f, P, uin, uout, phit, lam, lamt, u0, s);
    case 8: return launch_rowsA<8>(f, P, uin, uout, phit, lam, lamt, u0, s);
    case 9: return launch_rowsA<9>(f, P, uin, uout, phit, lam, lamt, u0, s);
    case 10: return launch_rowsA<10>(f, P, uin, uout, phit, lam, lamt, u0, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t fused2d_cols(Fused2D *f, const Params<float> &P, cudaStream_t s) {
    const unsigned grid = (unsigned)((P.nkx + 1) / 2);
    switch (ilog2i(P.ny)) {
    case 8: k_cols<8><<<grid, FTHREADS, 0, s>>>(P, f->spec, f->twY, f->thetaT); break;
    case 9: k_cols<9><<<grid, FTHREADS, 0, s>>>(P, f->spec, f->twY, f->thetaT); break;
    case 10: k_cols<10><<<grid, FTHREADS, 0, s>>>(P, f->spec, f->twY, f->thetaT); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t fused2d_rowsC(Fused2D *f, const Params<float> &P, float *phi, float *phit, cudaStream_t s) {
    switch (ilog2i(P.nx / 2)) {
    case 7: return launch_rowsC<7>(f, P, phi, phit, s);
    case 8: return launch_rowsC<8>(f, P, phi, phit, s);
    case 9: return launch_rowsC<9>(f, P, phi, phit, s);
    case 10: return launch_rowsC<10>(f, P, phi, phit, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pdhg

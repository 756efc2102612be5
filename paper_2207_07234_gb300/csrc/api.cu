// api.cu -- the C ABI of include/pdhg.h: validation, workspace layout, host
// preparation of the preconditioner tables, and the iteration driver of
// Algorithm 1 (Sec. 3.3).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pdhg.h"
#include "fused2d.h"
#include "plain.h"
#include "variants.h"

using namespace pdhg;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static pdhg_status fail(pdhg_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}
static pdhg_status cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return PDHG_ERR_CUDA;
}
#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

extern "C" const char *pdhg_last_error(void) { return g_last_error.c_str(); }

// lets other translation units of the library report through pdhg_last_error()
void pdhg::set_last_error(const std::string &msg) { g_last_error = msg; }

// ---------------------------------------------------------------------------
// layout
// ---------------------------------------------------------------------------
namespace {

constexpr int kMaxCanaries = 32;
constexpr unsigned char kCanaryByte = 0xA5;
struct Layout {
    size_t u, phi, phit, lam, lamt, u0, gamma, spec, twx, twy, theta, V, tfac, rtab, partials, scal, dbg, fused;
    size_t blu_tw, blu_c, blu_b;
    size_t twx32, twy32, theta32;    // float32 preconditioner tables (Geom::pre32)
    size_t total;
    // debug builds: the bytes after each sub-buffer up to the next 256-byte boundary plus
    // 256 more, filled with kCanaryByte at create and verified at every residual read
    int ncan;
    size_t can_off[kMaxCanaries];
    uint32_t can_len[kMaxCanaries];
};

inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
inline int ilog2(int64_t v) { int r = 0; while ((int64_t(1) << r) < v) ++r; return r; }
inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Geom {
    int dims, space, time, init, prec, path;
    int64_t nx, ny, nt, S, nkx, lines, modes;
    size_t esz;      // element size
    bool has_gamma;
    bool fused;
    int blu_log2L;   // > 0: Bluestein x-transform (1D FD, nx not a power of two)
    bool pre32;      // float64 state with the preconditioner applied in float32 (plain FD path)
    bool exact_t;    // time part of K_d: the scheme's own h_t^2 D_t D_t^T (PDHG_FLAG_EXACT_TIME_PRECOND)
    bool t64;        // float32 fields, t-solve recurrence in float64 (PDHG_FLAG_T_SOLVE_FP64)
    bool rtab;       // t-solve pivots from a [nt][modes] table (1D finite differences, few modes)
};

// Checks of the grid, the scheme and the coefficients (everything but u0 and the
// step sizes); fills G.  Shared with pdhg_residual_noalloc through check_shape().
pdhg_status validate_shape(const pdhg_problem *p, const pdhg_grid *g, const pdhg_scheme *s, Geom *G,
                           bool pre32) {
    if (!p || !g || !s) return fail(PDHG_ERR_INVALID_ARG, "null problem/grid/scheme");
    if (g->dims != 1 && g->dims != 2) return fail(PDHG_ERR_INVALID_ARG, "dims must be 1 or 2");
    if (s->time != PDHG_TIME_BE && s->time != PDHG_TIME_BDF2) return fail(PDHG_ERR_INVALID_ARG, "bad time scheme");
    if (s->space < PDHG_SPACE_FD_UPWIND || s->space > PDHG_SPACE_DG_P1_LF)
        return fail(PDHG_ERR_INVALID_ARG, "bad space scheme");
    if (s->precision != PDHG_FP64 && s->precision != PDHG_FP32) return fail(PDHG_ERR_INVALID_ARG, "bad precision");
    if (s->init != PDHG_INIT_LAMBDA && s->init != PDHG_INIT_PINNED) return fail(PDHG_ERR_INVALID_ARG, "bad init");
    if (s->path < PDHG_PATH_AUTO || s->path > PDHG_PATH_FUSED) return fail(PDHG_ERR_INVALID_ARG, "bad path");
    if (g->nt < 1 || g->nt > 65534) return fail(PDHG_ERR_INVALID_ARG, "nt must be in [1, 65534]");
    if (g->nx < 1 || (g->dims == 2 && g->ny < 1)) return fail(PDHG_ERR_INVALID_ARG, "nx, ny must be positive");
    if (!(g->T > 0) || !(g->lx > 0) || (g->dims == 2 && !(g->ly > 0)))
        return fail(PDHG_ERR_INVALID_ARG, "T, lx, ly must be positive");
    if (!std::isfinite(p->alpha) || !std::isfinite(p->beta) || !(p->nu >= 0) || !std::isfinite(p->nu) ||
        !std::isfinite(p->c) || !std::isfinite(p->gamma_hat) || !(p->lf_a >= 0) || !std::isfinite(p->lf_a))
        return fail(PDHG_ERR_INVALID_ARG, "non-finite or negative coefficient");
    const bool dg = s->space >= PDHG_SPACE_DG_P2_LF;
    if (dg) {
        if (g->dims != 1) return fail(PDHG_ERR_UNSUPPORTED, "DG is 1D only");
        if (p->gamma_half) return fail(PDHG_ERR_UNSUPPORTED, "DG has no variable-coefficient Laplacian");
        if (p->nu != 0) return fail(PDHG_ERR_UNSUPPORTED, "DG has no viscous term");
        if (p->gamma_hat != 0) return fail(PDHG_ERR_UNSUPPORTED, "the DG preconditioner uses c only");
    }
    if (g->dims == 2 && p->gamma_half) return fail(PDHG_ERR_UNSUPPORTED, "gamma_half is 1D only");
    G->blu_log2L = 0;
    if (!is_pow2(g->nx)) {
        if (g->dims != 1 || dg || g->nx < 4 || g->nx > 4096)
            return fail(PDHG_ERR_UNSUPPORTED, "nx must be a power of two in [4, 8192] (1D finite differences: any "
                                              "nx in [4, 4096])");
        G->blu_log2L = ilog2(2 * g->nx - 1);
    } else if (g->nx < 4 || g->nx > 8192) {
        return fail(PDHG_ERR_UNSUPPORTED, "nx must be a power of two in [4, 8192]");
    }
    if (g->dims == 2 && (!is_pow2(g->ny) || g->ny < 4 || g->ny > 2048))
        return fail(PDHG_ERR_UNSUPPORTED, "ny must be a power of two in [4, 2048]");
    G->dims = g->dims; G->space = s->space; G->time = s->time; G->init = s->init;
    G->prec = s->precision; G->path = s->path;
    G->nx = g->nx; G->ny = g->dims == 2 ? g->ny : 1; G->nt = g->nt;
    const int nm = s->space == PDHG_SPACE_DG_P2_LF ? 3 : (dg ? 2 : 1);
    G->S = dg ? nm * g->nx : g->nx * G->ny;
    G->nkx = g->nx / 2 + 1;
    G->lines = dg ? nm : G->ny;
    G->modes = dg ? nm * G->nkx : G->lines * G->nkx;
    G->esz = s->precision == PDHG_FP64 ? 8 : 4;
    G->has_gamma = p->gamma_half != nullptr;
    G->fused = false;
    if (s->flags & ~(int32_t)(PDHG_FLAG_EXACT_TIME_PRECOND | PDHG_FLAG_U0_ON_DEVICE | PDHG_FLAG_T_SOLVE_FP64))
        return fail(PDHG_ERR_INVALID_ARG, "unknown scheme flag");
    G->exact_t = (s->flags & PDHG_FLAG_EXACT_TIME_PRECOND) != 0;
    G->t64 = (s->flags & PDHG_FLAG_T_SOLVE_FP64) != 0 && s->precision == PDHG_FP32;
    if (G->t64 && (dg || G->exact_t))
        return fail(PDHG_ERR_UNSUPPORTED, "the float64 t-recurrence serves the finite-difference schemes with T_t");
    if (G->t64 && s->path == PDHG_PATH_FUSED && G->ny != 1024)
        return fail(PDHG_ERR_UNSUPPORTED, "the fused path's float64 t-recurrence needs ny = 1024");
    if (G->exact_t) {
        if (s->path == PDHG_PATH_FUSED)
            return fail(PDHG_ERR_UNSUPPORTED, "the exact time preconditioner runs on the plain path");
        if ((double)G->modes * (double)G->nt > (double)(int64_t(1) << 24))
            return fail(PDHG_ERR_UNSUPPORTED, "the exact time preconditioner's factor table is limited to "
                                              "2^24 (mode, slice) pairs");
    }
    if (!G->exact_t && (s->path == PDHG_PATH_FUSED || s->path == PDHG_PATH_AUTO)) {
        bool ok = fused2d_supported(g->dims, s->space, s->time, s->precision, g->nx, G->ny, g->nt, p->nu) &&
                  !(G->t64 && G->ny != 1024);
        if (s->path == PDHG_PATH_FUSED && !ok)
            return fail(PDHG_ERR_UNSUPPORTED, "the fused path needs 2D FD, FP32, nx in [256, 2048], ny in [256, 1024] (powers of two)");
        G->fused = ok;
    }
    G->pre32 = pre32 && s->precision == PDHG_FP64 && !G->fused && !dg && G->blu_log2L == 0 && !G->exact_t;
    // 1D: a few thousand modes, each swept by one thread, so the sweeps run at the latency
    // of their per-step pivot evaluation; a table of the same values (computed once at
    // create, at most 2^23 entries) turns each pivot into one load
    G->rtab = g->dims == 1 && !dg && !G->fused && !G->exact_t && !G->t64 && !G->pre32 &&
              (double)G->modes * (double)G->nt <= (double)(int64_t(1) << 23);
    return PDHG_OK;
}

pdhg_status validate(const pdhg_problem *p, const pdhg_grid *g, const pdhg_scheme *s, Geom *G,
                     bool pre32 = false) {
    pdhg_status st = validate_shape(p, g, s, G, pre32);
    if (st != PDHG_OK) return st;
    if (!p->u0) return fail(PDHG_ERR_INVALID_ARG, "u0 is NULL");
    if (!(p->tau_u > 0) || !(p->tau_phi > 0)) return fail(PDHG_ERR_INVALID_ARG, "tau_u, tau_phi must be > 0");
    if (s->init == PDHG_INIT_LAMBDA && (!(p->tau_u0 > 0) || !(p->tau_lambda > 0)))
        return fail(PDHG_ERR_INVALID_ARG, "tau_u0, tau_lambda must be > 0");
    return PDHG_OK;
}

Layout layout_of(const Geom &G) {
    Layout L;
    L.ncan = 0;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
#ifdef PDHG_DEBUG
        if (L.ncan < kMaxCanaries) {
            L.can_off[L.ncan] = at + bytes;
            L.can_len[L.ncan] = (uint32_t)(o + 256 - (at + bytes));
            ++L.ncan;
        }
        o += 256;
#endif
        return at;
    };
    const size_t e = G.esz;
    L.u = take((G.nt + 1) * G.S * e);
    L.phi = take(G.nt * G.S * e);
    L.phit = take(G.nt * G.S * e);
    L.lam = take(G.S * e);
    L.lamt = take(G.S * e);
    L.u0 = take(G.S * e);
    L.gamma = take(G.has_gamma ? G.S * e : 0);
    L.spec = take(G.fused ? 0 : (size_t)G.nt * G.lines * G.nkx * 2 * e);
    L.twx = take(G.nkx * 2 * e);
    L.twy = take(G.dims == 2 ? G.ny * 2 * e : 0);
    L.theta = take(G.modes * e);
    L.V = take(G.space >= PDHG_SPACE_DG_P2_LF ? G.nkx * 9 * 2 * e : 0);
    L.tfac = take(G.exact_t ? 3 * G.nt * G.modes * e : 0);
    L.rtab = take(G.rtab ? G.nt * G.modes * e : 0);
    int64_t units = G.space >= PDHG_SPACE_DG_P2_LF ? G.nx : G.S;
    int64_t nblk = check_blocks_per_row(units, G.nt) * (G.nt + 1);    // k_check grid
    L.partials = take(nblk * 6 * sizeof(double));
    L.scal = take(16 * sizeof(double));
    L.dbg = take(sizeof(int));                  // debug builds: first out-of-range site
    L.fused = take(G.fused ? fused2d_workspace_bytes(G.nx, G.ny, G.nt) : 0);
    const size_t lb = G.blu_log2L ? ((size_t)1 << G.blu_log2L) : 0;
    L.blu_tw = take(lb * 2 * e);
    L.blu_c = take(G.blu_log2L ? G.nx * 2 * e : 0);
    L.blu_b = take(lb * 2 * e);
    L.twx32 = take(G.pre32 ? G.nkx * 2 * sizeof(float) : 0);
    L.twy32 = take(G.pre32 && G.dims == 2 ? G.ny * 2 * sizeof(float) : 0);
    L.theta32 = take(G.pre32 ? G.modes * sizeof(float) : 0);
    L.total = o;
    return L;
}

// ---------------------------------------------------------------------------
// host tables
// ---------------------------------------------------------------------------
typedef std::complex<double> cd;

// theta with cosh(theta) = 1 + s/2, i.e. theta = 2 asinh(sqrt(s)/2), s = kappa h_t^2 >= 0
double theta_of(double s) { return s <= 0 ? 0.0 : 2.0 * std::asinh(0.5 * std::sqrt(s)); }

// The exact time operator of the ablation: K = A_t A_t^T, A_t the scheme's time
// differences times h_t acting on u^1..u^nt (u^0 held fixed; row m = equation R^m,
// entries coef(m, m+1), coef(m, m), coef(m, m-1) in units of 1/h_t), so K is T_t for
// backward Euler and pentadiagonal for BDF2.  For each mode the LDL^T factors of K + s
// (L unit lower triangular with sub-diagonals e_l = L_{l,l-1}, f_l = L_{l,l-2}) go to
// tab[3][nt][modes] as 1/d_l, e_l, f_l.
template <typename T>
void exact_t_factors(int time, int64_t nt, const std::vector<double> &s, std::vector<T> &tab) {
    const int64_t modes = (int64_t)s.size();
    auto Aj = [&](int64_t m, int j) -> double {           // A_t[m][m - j], column m - j = u^{m+1-j}
        if (m < 0 || m >= nt || m - j < 0 || j > 2) return 0.0;
        const bool be = time == PDHG_TIME_BE || m == 0;
        if (j == 0) return be ? 1.0 : 1.5;
        if (j == 1) return be ? -1.0 : -2.0;
        return be ? 0.0 : 0.5;
    };
    std::vector<double> a(nt), b(nt), c(nt);                // K[l][l], K[l][l+1], K[l][l+2]
    for (int64_t l = 0; l < nt; ++l) {
        a[l] = b[l] = c[l] = 0.0;
        for (int j = 0; j < 3; ++j) {
            a[l] += Aj(l, j) * Aj(l, j);
            b[l] += Aj(l, j) * Aj(l + 1, j + 1);
            c[l] += Aj(l, j) * Aj(l + 2, j + 2);
        }
    }
    tab.assign(3 * nt * modes, (T)0);
    for (int64_t k = 0; k < modes; ++k) {
        double d1 = 1.0, d2 = 1.0, e1 = 0.0;               // d_{l-1}, d_{l-2}, e_{l-1}
        for (int64_t l = 0; l < nt; ++l) {
            const double f = l >= 2 ? c[l - 2] / d2 : 0.0;
            const double e = l >= 1 ? (b[l - 1] - f * e1 * d2) / d1 : 0.0;
            const double d = a[l] + s[k] - e * e * d1 - f * f * d2;
            tab[l * modes + k] = (T)(1.0 / d);
            tab[(nt + l) * modes + k] = (T)e;
            tab[(2 * nt + l) * modes + k] = (T)f;
            d2 = d1;
            d1 = d;
            e1 = e;
        }
    }
}

// L(theta_k) = (2 - 2 cos(2 pi k/n))/h^2 written as 4 sin^2(pi k/n)/h^2
double symbol_L(int64_t k, int64_t n, double h) {
    double s = std::sin(M_PI * (double)k / (double)n);
    return 4.0 * s * s / (h * h);
}

// Cyclic Jacobi for an n x n (n <= 3) Hermitian matrix: A = V diag(w) V^H.
void jacobi_herm(int n, cd A[3][3], double w[3], cd V[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0, dia = 0;
        for (int i = 0; i < n; ++i) {
            dia += std::abs(A[i][i].real());
            for (int j = i + 1; j < n; ++j) off += std::abs(A[i][j]);
        }
        if (off <= 1e-300 || off <= 1e-17 * dia) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double r = std::abs(A[p][q]);
                if (r == 0.0) continue;
                cd ph = A[p][q] / r;                      // A_pq = r e^{i phi}
                double app = A[p][p].real(), aqq = A[q][q].real();
                double tau = (aqq - app) / (2.0 * r);
                double t = (tau >= 0 ? 1.0 : -1.0) / (std::abs(tau) + std::sqrt(1.0 + tau * tau));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                // unitary G acting on columns p, q: col_p' = c col_p - s conj(ph) col_q, col_q' = s ph col_p + c col_q
                cd gpp = c, gqp = -s * std::conj(ph), gpq = s * ph, gqq = c;
                for (int k = 0; k < n; ++k) {               // A <- A G
                    cd akp = A[k][p], akq = A[k][q];
                    A[k][p] = akp * gpp + akq * gqp;
                    A[k][q] = akp * gpq + akq * gqq;
                }
                for (int k = 0; k < n; ++k) {               // A <- G^H A
                    cd apk = A[p][k], aqk = A[q][k];
                    A[p][k] = std::conj(gpp) * apk + std::conj(gqp) * aqk;
                    A[q][k] = std::conj(gpq) * apk + std::conj(gqq) * aqk;
                }
                for (int k = 0; k < n; ++k) {               // V <- V G
                    cd vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = vkp * gpp + vkq * gqp;
                    V[k][q] = vkp * gpq + vkq * gqq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i][i].real();
}

// S(theta) of the DG P1 nodal operator (Sec. 3.2.2) of c u_x with the upwind flux
// (Lax-Friedrichs with a = |c|), from the weak form: with phi(1) = R = (-1/2, 3/2),
// phi(-1) = L = (3/2, -1/2), phi' = (-1, 1) and int phi = (1, 1),
//   E(j) = B0 U_j + Bm U_{j-1} + Bp U_{j+1},
//   B0[m][n] = phi_m' c - R_m cp R_n + L_m cm L_n,  Bm[m][n] = L_m cp R_n,  Bp[m][n] = -R_m cm L_n,
// cp = max(c, 0), cm = min(c, 0); D = -M^{-1} E with h M^{-1} = [[7,1],[1,7]]/4.
// (For c > 0 the U_j block is the negative of the paper's A1 of Eq. 3.5.)
void dg1_symbol(double c, double h, double theta, cd S[3][3]) {
    const double R[2] = {-0.5, 1.5}, L[2] = {1.5, -0.5}, dphi[2] = {-1.0, 1.0};
    const double cp = 0.5 * (c + std::fabs(c)), cm = 0.5 * (c - std::fabs(c));
    const double Mi[2][2] = {{7.0 / 4.0, 1.0 / 4.0}, {1.0 / 4.0, 7.0 / 4.0}};
    cd em = std::exp(cd(0, -theta)), ep = std::exp(cd(0, theta));
    cd E[2][2];
    for (int m = 0; m < 2; ++m)
        for (int n = 0; n < 2; ++n) {
            double b0 = dphi[m] * c - R[m] * cp * R[n] + L[m] * cm * L[n];
            double bm = L[m] * cp * R[n];
            double bp = -R[m] * cm * L[n];
            E[m][n] = cd(b0) + cd(bm) * em + cd(bp) * ep;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i][j] = 0.0;
    for (int m = 0; m < 2; ++m)
        for (int n = 0; n < 2; ++n) S[m][n] = -(Mi[m][0] * E[0][n] + Mi[m][1] * E[1][n]) / h;
}

// S(theta) of the DG P2 operator of c u_x with the upwind flux (Lax-Friedrichs
// with a = |c|): D_m = -(2m+1)/h [vol_m - Fh_{j+1/2} + (-1)^m Fh_{j-1/2}],
// vol_1 = 2 c U_0, vol_2 = 2 c U_1, Fh_{j+1/2} = cp uR_j + cm uL_{j+1}.
void dg_symbol(double c, double h, double theta, cd S[3][3]) {
    double cp = 0.5 * (c + std::fabs(c)), cm = 0.5 * (c - std::fabs(c));
    cd em = std::exp(cd(0, -theta)), ep = std::exp(cd(0, theta));
    for (int m = 0; m < 3; ++m) {
        double sm = (m % 2) ? -1.0 : 1.0;
        for (int n = 0; n < 3; ++n) {
            double sn = (n % 2) ? -1.0 : 1.0;
            double vol = (m == 1 && n == 0) ? 2 * c : (m == 2 && n == 1) ? 2 * c : 0.0;
            double s0 = vol - cp + sm * cm * sn;       // from U_j
            double sl = sm * cp;                        // from U_{j-1}
            double sr = -cm * sn;                       // from U_{j+1}
            double f = -(2 * m + 1) / h;
            S[m][n] = f * (cd(s0) + cd(sl) * em + cd(sr) * ep);
        }
    }
}

}  // namespace

// The grid, scheme and coefficient checks of pdhg_create for a caller that brings
// its own state (no u0, no step sizes); the path is not part of it.
pdhg_status pdhg::check_shape(const pdhg_problem *p, const pdhg_grid *g, const pdhg_scheme *s) {
    if (!s) return fail(PDHG_ERR_INVALID_ARG, "null problem/grid/scheme");
    pdhg_scheme plain = *s;
    plain.path = PDHG_PATH_PLAIN;
    Geom G;
    return validate_shape(p, g, &plain, &G, false);
}

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct EvRec { int stage; cudaEvent_t a, b; };

struct pdhg_handle {
    Geom G;
    Layout L;
    char *ws;
    cudaStream_t stream;
    Params<float> pf;
    Params<double> pd;
    double ht, wx;
    int64_t iters;
    double res_init;
    double last_res[4];      // Res at the last check of pdhg_iterate
    int64_t launches;
    bool profiling;
    std::vector<EvRec> recs;
    std::vector<cudaEvent_t> pool;
    double stage_ms[PDHG_NUM_STAGES];
    int64_t stage_n[PDHG_NUM_STAGES];
    Fused2D fused;
    size_t u_off;            // offset of the current u buffer
    int res_norm;            // 0: space-time norms of Eq. 2.12; 1: per time slice (Sec. 3.5)
    // CUDA graph of `gchunk` iterations plus the residual check (plain path)
    bool graphs;
    cudaGraphExec_t gexec;
    cudaStream_t gstream;
    int32_t gchunk;
    int64_t glaunches;       // kernel launches per replay
    bool u0_dev;             // the problem's u0 was given in device memory (PDHG_FLAG_U0_ON_DEVICE)
    // Res at every check of pdhg_iterate: rows [iterations done, Res entries 0..3], the
    // newest kHistoryRows kept (a ring: hist_next is the next row to write)
    std::vector<double> hist;
    int64_t hist_next;
    int64_t hist_count;
};

constexpr int64_t kHistoryRows = 65536;

static void history_push(pdhg_handle *h, const double r[4]) {
    if (h->hist.empty()) h->hist.assign((size_t)kHistoryRows * 5, 0.0);
    double *row = h->hist.data() + (size_t)(h->hist_next % kHistoryRows) * 5;
    row[0] = (double)h->iters;
    for (int k = 0; k < 4; ++k) row[1 + k] = r[k];
    ++h->hist_next;
    h->hist_count = std::min<int64_t>(h->hist_count + 1, kHistoryRows);
}

static void graph_drop(pdhg_handle *h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->gchunk = 0;
}

template <typename T> static Params<T> &params_of(pdhg_handle *h);
template <> Params<float> &params_of<float>(pdhg_handle *h) { return h->pf; }
template <> Params<double> &params_of<double>(pdhg_handle *h) { return h->pd; }

template <typename T> static T *F(pdhg_handle *h, size_t off) { return reinterpret_cast<T *>(h->ws + off); }

static cudaEvent_t ev_get(pdhg_handle *h) {
    if (!h->pool.empty()) { cudaEvent_t e = h->pool.back(); h->pool.pop_back(); return e; }
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// run one stage launch, bracketed by events when profiling
template <typename Fn>
static cudaError_t stage(pdhg_handle *h, int st, int nlaunch, Fn fn) {
    // NVTX names of the stages (host ranges around each stage's launches while profiling)
    static const char *const names[PDHG_NUM_STAGES] = {"pdhg primal", "pdhg residual + x-FFT", "pdhg y-FFT",
                                                       "pdhg t-solve", "pdhg dual", "pdhg residual norms",
                                                       "pdhg fused rows", "pdhg fused cols"};
    EvRec r{st, nullptr, nullptr};
    if (h->profiling) {
        nvtxRangePushA(names[st]);
        r.a = ev_get(h); r.b = ev_get(h);
        if (r.a) cudaEventRecord(r.a, h->stream);
    }
    cudaError_t e = fn();
    h->launches += nlaunch;
    if (h->profiling) {
        if (r.b) {
            cudaEventRecord(r.b, h->stream);
            h->recs.push_back(r);
        }
        nvtxRangePop();
    }
    return e;
}

template <typename T>
static void fill_params(Params<T> &P, const Geom &G, const pdhg_problem *p, const pdhg_grid *g, double lf_a) {
    memset(&P, 0, sizeof(P));
    P.dims = G.dims; P.space = G.space; P.time = G.time; P.init = G.init;
    P.nx = (int32_t)G.nx; P.ny = (int32_t)G.ny; P.nt = (int32_t)G.nt;
    P.log2m = ilog2(G.nx / 2); P.log2ny = G.dims == 2 ? ilog2(G.ny) : 0;
    P.S = G.S; P.nkx = (int32_t)G.nkx; P.lines = (int32_t)G.lines;
    double ht = g->T / (double)g->nt, hx = g->lx / (double)g->nx;
    double hy = G.dims == 2 ? g->ly / (double)g->ny : 1.0;
    P.alpha = (T)p->alpha; P.beta = (T)p->beta; P.nu = (T)p->nu; P.lf_a = (T)lf_a;
    P.ht = (T)ht; P.inv_ht = (T)(1.0 / ht); P.inv_hx = (T)(1.0 / hx); P.inv_hy = (T)(1.0 / hy);
    P.tau_u = (T)p->tau_u; P.tau_u0 = (T)p->tau_u0; P.tau_phi = (T)p->tau_phi; P.tau_lambda = (T)p->tau_lambda;
    P.dual_scale = (T)(p->tau_phi * ht * ht / ((double)(G.nx / 2) * (double)G.ny));
    P.gamma_half = nullptr;
    P.blu_log2L = G.blu_log2L;
    P.blu_scale = (T)(p->tau_phi * ht * ht);
}

// In-place iterative radix-2 FFT (forward, unnormalised) of n = 2^k values, host, double.
static void host_fft(std::vector<std::complex<double>> &a) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> w(std::cos(ang * (double)k), std::sin(ang * (double)k));
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

// Bluestein tables for a length-N DFT through length-L FFTs: stage-grouped W_L, the
// chirp c_n = exp(i pi n^2 / N) (n^2 reduced mod 2N before scaling), FFT_L(b).
template <typename T>
static void bluestein_tables(int64_t N, int log2L, std::vector<T> &tw, std::vector<T> &c, std::vector<T> &bh) {
    const int64_t L = int64_t(1) << log2L;
    tw.assign(2 * L, (T)0);                   // stage s: entries (2^s - 1) + pos, pos < 2^s
    for (int s = 0; s < log2L; ++s) {
        const int64_t hs = int64_t(1) << s;
        for (int64_t pos = 0; pos < hs; ++pos) {
            const double a = -2.0 * M_PI * (double)(pos * (L / (2 * hs))) / (double)L;
            tw[2 * (hs - 1 + pos)] = (T)std::cos(a);
            tw[2 * (hs - 1 + pos) + 1] = (T)std::sin(a);
        }
    }
    std::vector<std::complex<double>> cd(N), b(L, 0.0);
    for (int64_t n = 0; n < N; ++n) {
        const int64_t q = (n * n) % (2 * N);
        cd[n] = std::polar(1.0, M_PI * (double)q / (double)N);
    }
    for (int64_t m = 0; m < N; ++m) {
        b[m] = cd[m];
        if (m > 0) b[L - m] = cd[m];
    }
    host_fft(b);
    c.resize(2 * N);
    for (int64_t n = 0; n < N; ++n) { c[2 * n] = (T)cd[n].real(); c[2 * n + 1] = (T)cd[n].imag(); }
    bh.resize(2 * L);
    for (int64_t m = 0; m < L; ++m) { bh[2 * m] = (T)b[m].real(); bh[2 * m + 1] = (T)b[m].imag(); }
}

extern "C" pdhg_status pdhg_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                           const pdhg_scheme *scheme, size_t *bytes) {
    Geom G;
    pdhg_status st = validate(prob, grid, scheme, &G);
    if (st != PDHG_OK) return st;
    if (!bytes) return fail(PDHG_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = layout_of(G).total;
    return PDHG_OK;
}

// Twiddles of a length-N Stockham transform grouped by stage: the radix-4 stage of
// span p (p = P0, 4 P0, ... with P0 = 1 for even log2 N, 2 for odd) owns entries
// (p - P0) + q p + k = W_N^{(q+1) k N/(4p)}, q = 0..2, k < p.  N complex entries
// (interleaved re, im), unused ones zero.
static std::vector<float> staged_twiddles(int64_t N) {
    std::vector<float> t(2 * N, 0.f);
    int lg = 0;
    while ((int64_t(1) << lg) < N) ++lg;
    const int64_t p0 = (lg & 1) ? 2 : 1;
    for (int64_t p = p0; 4 * p <= N; p *= 4)
        for (int64_t q = 0; q < 3; ++q)
            for (int64_t k = 0; k < p; ++k) {
                const int64_t e = (p - p0) + q * p + k;
                const double a = 2.0 * M_PI * (double)((q + 1) * k * (N / (4 * p))) / (double)N;
                t[2 * e] = (float)std::cos(a);
                t[2 * e + 1] = (float)(-std::sin(a));
            }
    return t;
}

// Twiddles of the radix-8 Stockham transform of length N: the radix-8 stage of span
// p (p = P0, 8 P0, ... with P0 = 2^(log2 N mod 3)) owns entries
// (p - P0) + (q-1) p + k = W_N^{q k N/(8p)}, q = 1..7, k < p.
static std::vector<float> staged_twiddles8(int64_t N) {
    std::vector<float> t(2 * N, 0.f);
    int lg = 0;
    while ((int64_t(1) << lg) < N) ++lg;
    const int64_t p0 = int64_t(1) << (lg % 3);
    for (int64_t p = p0; 8 * p <= N; p *= 8)
        for (int64_t q = 1; q < 8; ++q)
            for (int64_t k = 0; k < p; ++k) {
                const int64_t e = (p - p0) + (q - 1) * p + k;
                const double a = 2.0 * M_PI * (double)(q * k * (N / (8 * p))) / (double)N;
                t[2 * e] = (float)std::cos(a);
                t[2 * e + 1] = (float)(-std::sin(a));
            }
    return t;
}

// Twiddles of the 4 x 8 x 8 x 4 transform of length 1024 along y (fused 2D path):
// the radix-8 stage of span p (4, 32) owns entries (p - 4) + (q-1) p + k =
// W^{q k 1024/(8p)}, q = 1..7, k < p; the final radix-4 stage (span 256) owns
// 252 + (q-1) 256 + k = W^{q k}, q = 1..3, with W = exp(-2 pi i / 1024).
static std::vector<float> cols1024_twiddles() {
    const int64_t N = 1024;
    std::vector<float> t(2 * N, 0.f);
    auto put = [&](int64_t e, int64_t expo) {
        const double a = 2.0 * M_PI * (double)expo / (double)N;
        t[2 * e] = (float)std::cos(a);
        t[2 * e + 1] = (float)(-std::sin(a));
    };
    for (int64_t p : {int64_t(4), int64_t(32)})
        for (int64_t q = 1; q < 8; ++q)
            for (int64_t k = 0; k < p; ++k) put((p - 4) + (q - 1) * p + k, q * k * (N / (8 * p)));
    for (int64_t q = 1; q < 4; ++q)
        for (int64_t k = 0; k < 256; ++k) put(252 + (q - 1) * 256 + k, q * k);
    return t;
}

// Run fn(r0, r1) over [0, nrows) in contiguous chunks on up to 16 host threads when
// the work (total elements) is large; inline otherwise.  Results do not depend on
// the split: every element is computed the same way.
template <typename Fn>
static void parallel_rows(int64_t nrows, int64_t total, Fn fn) {
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::min<unsigned>(nt == 0 ? 1 : nt, 16);
    if (total < (int64_t(1) << 16) || nt <= 1 || nrows < 2) { fn(0, nrows); return; }
    nt = (unsigned)std::min<int64_t>(nt, nrows);
    std::vector<std::thread> pool;
    const int64_t chunk = (nrows + nt - 1) / nt;
    for (unsigned t = 0; t < nt; ++t) {
        const int64_t r0 = t * chunk, r1 = std::min<int64_t>(nrows, r0 + chunk);
        if (r0 < r1) pool.emplace_back(fn, r0, r1);
    }
    for (auto &th : pool) th.join();
}

// u0 in device memory (PDHG_FLAG_U0_ON_DEVICE): the largest |f'(u0)| = |2 alpha u0 + beta|
// and the number of non-finite values, without copying u0 out.  out[0] holds the bits
// of the maximum (non-negative doubles order like their bit patterns), out[1] the count.
__global__ void k_u0_scan(const double *__restrict__ u0, int64_t n, double alpha, double beta,
                          unsigned long long *out) {
    double m = 0.0;
    unsigned long long bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = u0[i];
        if (!isfinite(v)) ++bad;
        else m = fmax(m, fabs(2.0 * alpha * v + beta));
    }
    for (int o = 16; o; o >>= 1) {
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(m));
        if (bad) atomicAdd(out + 1, bad);
    }
}

template <typename T>
__global__ void k_u0_convert(const double *__restrict__ src, T *__restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

template <typename T>
static pdhg_status upload_tables(pdhg_handle *h, const pdhg_problem *p, const pdhg_grid *g, double lf_a) {
    const Geom &G = h->G;
    cudaStream_t s = h->stream;
    std::vector<T> buf;
    // u0 extended in t; phi = phit = 0; lambda = lambdat = 0 (Sec. 3.3)
    buf.resize(G.S);
    if (h->u0_dev) {
        k_u0_convert<T><<<(unsigned)std::min<int64_t>((G.S + 255) / 256, 1024), 256, 0, s>>>(p->u0, F<T>(h, h->L.u0),
                                                                                            G.S);
        CK(cudaGetLastError());
    } else {
        for (int64_t i = 0; i < G.S; ++i) buf[i] = (T)p->u0[i];
        CK(cudaMemcpyAsync(F<T>(h, h->L.u0), buf.data(), G.S * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    CK(launch_fill_slices<T>(F<T>(h, h->L.u), F<T>(h, h->L.u0), G.S, G.nt + 1, s));
    CK(cudaMemsetAsync(F<T>(h, h->L.phi), 0, G.nt * G.S * sizeof(T), s));
    CK(cudaMemsetAsync(F<T>(h, h->L.phit), 0, G.nt * G.S * sizeof(T), s));
    CK(cudaMemsetAsync(F<T>(h, h->L.lam), 0, G.S * sizeof(T), s));
    CK(cudaMemsetAsync(F<T>(h, h->L.lamt), 0, G.S * sizeof(T), s));
    CK(cudaStreamSynchronize(s));
    if (G.has_gamma) {
        for (int64_t i = 0; i < G.S; ++i) buf[i] = (T)p->gamma_half[i];
        CK(cudaMemcpy(F<T>(h, h->L.gamma), buf.data(), G.S * sizeof(T), cudaMemcpyHostToDevice));
    }
    // twiddles W_N^k = exp(-2 pi i k/N)
    std::vector<T> tw(2 * G.nkx);
    for (int64_t k = 0; k < G.nkx; ++k) {
        double a = 2.0 * M_PI * (double)k / (double)G.nx;
        tw[2 * k] = (T)std::cos(a); tw[2 * k + 1] = (T)(-std::sin(a));
    }
    CK(cudaMemcpy(F<T>(h, h->L.twx), tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice));
    if (G.dims == 2) {
        std::vector<T> twy(2 * G.ny);
        for (int64_t k = 0; k < G.ny; ++k) {
            double a = 2.0 * M_PI * (double)k / (double)G.ny;
            twy[2 * k] = (T)std::cos(a); twy[2 * k + 1] = (T)(-std::sin(a));
        }
        CK(cudaMemcpy(F<T>(h, h->L.twy), twy.data(), twy.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    // preconditioner: theta per Fourier mode (and the DG eigenvectors)
    double ht = g->T / (double)g->nt, hx = g->lx / (double)g->nx;
    double hy = G.dims == 2 ? g->ly / (double)g->ny : 1.0;
    std::vector<T> th(G.modes);
    std::vector<double> sv(G.exact_t ? G.modes : 0);      // s = kappa h_t^2 per mode (exact time operator)
    if (G.space >= PDHG_SPACE_DG_P2_LF) {
        const int nm = (int)G.lines;
        std::vector<T> V(G.nkx * 18, (T)0);
        for (int64_t k = 0; k < G.nkx; ++k) {
            cd S[3][3], A[3][3], Vm[3][3];
            double w[3];
            const double theta = 2.0 * M_PI * (double)k / (double)G.nx;
            if (G.space == PDHG_SPACE_DG_P2_LF) dg_symbol(p->c, hx, theta, S);
            else dg1_symbol(p->c, hx, theta, S);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    cd acc = 0;
                    for (int m = 0; m < nm; ++m) acc += std::conj(S[m][i]) * S[m][j];
                    A[i][j] = (i < nm && j < nm) ? acc : cd(0.0);
                }
            jacobi_herm(nm, A, w, Vm);
            for (int i = 0; i < nm; ++i) {
                th[k * nm + i] = (T)theta_of(std::max(w[i], 0.0) * ht * ht);
                if (G.exact_t) sv[k * nm + i] = std::max(w[i], 0.0) * ht * ht;
            }
            for (int m = 0; m < 3; ++m)
                for (int i = 0; i < 3; ++i) {
                    V[(k * 9 + m * 3 + i) * 2] = (T)Vm[m][i].real();
                    V[(k * 9 + m * 3 + i) * 2 + 1] = (T)Vm[m][i].imag();
                }
        }
        CK(cudaMemcpy(F<T>(h, h->L.V), V.data(), V.size() * sizeof(T), cudaMemcpyHostToDevice));
    } else {
        // L = L_x(kx) + L_y(ky) is separable: tabulate both, then one sqrt and asinh per
        // mode, rows of ky spread over host threads (2D grids have up to 1M modes)
        std::vector<double> Lx(G.nkx), Ly(G.lines, 0.0);
        for (int64_t kx = 0; kx < G.nkx; ++kx) Lx[kx] = symbol_L(kx, G.nx, hx);
        if (G.dims == 2)
            for (int64_t ky = 0; ky < G.lines; ++ky) Ly[ky] = symbol_L(ky, G.ny, hy);
        const double c2 = p->c * p->c, g2 = p->gamma_hat * p->gamma_hat;
        auto rows = [&](int64_t y0, int64_t y1) {
            for (int64_t ky = y0; ky < y1; ++ky)
                for (int64_t kx = 0; kx < G.nkx; ++kx) {
                    const double L = Lx[kx] + Ly[ky];
                    th[ky * G.nkx + kx] = (T)theta_of((c2 * L + g2 * L * L) * ht * ht);
                    if (G.exact_t) sv[ky * G.nkx + kx] = (c2 * L + g2 * L * L) * ht * ht;
                }
        };
        parallel_rows(G.lines, G.lines * G.nkx, rows);
    }
    CK(cudaMemcpy(F<T>(h, h->L.theta), th.data(), th.size() * sizeof(T), cudaMemcpyHostToDevice));
    if (G.exact_t) {
        std::vector<T> tab;
        exact_t_factors<T>(G.time, G.nt, sv, tab);
        CK(cudaMemcpy(F<T>(h, h->L.tfac), tab.data(), tab.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    if (G.pre32) {
        // float32 copies of the preconditioner's tables (rounded from the float64 values)
        std::vector<float> t32(tw.begin(), tw.end()), th32(th.begin(), th.end());
        CK(cudaMemcpy(h->ws + h->L.twx32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->ws + h->L.theta32, th32.data(), th32.size() * sizeof(float), cudaMemcpyHostToDevice));
        if (G.dims == 2) {
            std::vector<float> y32(2 * G.ny);
            for (int64_t k = 0; k < G.ny; ++k) {
                double a = 2.0 * M_PI * (double)k / (double)G.ny;
                y32[2 * k] = (float)std::cos(a); y32[2 * k + 1] = (float)(-std::sin(a));
            }
            CK(cudaMemcpy(h->ws + h->L.twy32, y32.data(), y32.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
    }
    if (G.blu_log2L) {
        std::vector<T> btw, bc, bb;
        bluestein_tables<T>(G.nx, G.blu_log2L, btw, bc, bb);
        CK(cudaMemcpy(h->ws + h->L.blu_tw, btw.data(), btw.size() * sizeof(T), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->ws + h->L.blu_c, bc.data(), bc.size() * sizeof(T), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->ws + h->L.blu_b, bb.data(), bb.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    if (G.fused) {
        // fused 2D path: staged twiddle tables for the Stockham transforms of length
        // M = nx/2 (along x) and ny (along y; ny = 1024 has its own plan), and theta
        // in [kx][ky] order
        Fused2D &f = h->fused;
        fused2d_layout(&f, h->ws + h->L.fused, G.nx, G.ny, G.nt);
        std::vector<float> tm = staged_twiddles(G.nx / 2), ty = G.ny == 1024 ? cols1024_twiddles() : staged_twiddles(G.ny),
                           tt(G.nkx * G.ny);
        parallel_rows(G.nkx, G.nkx * G.ny, [&](int64_t x0, int64_t x1) {
            for (int64_t kx = x0; kx < x1; ++kx)
                for (int64_t ky = 0; ky < G.ny; ++ky) tt[kx * G.ny + ky] = (float)th[ky * G.nkx + kx];
        });
        CK(cudaMemcpy(f.twM, tm.data(), tm.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(f.twY, ty.data(), ty.size() * 4, cudaMemcpyHostToDevice));
        const std::vector<float> t8 = staged_twiddles8(G.nx / 2);
        CK(cudaMemcpy(f.twM8, t8.data(), t8.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(f.thetaT, tt.data(), tt.size() * 4, cudaMemcpyHostToDevice));
    }
    Params<T> &P = params_of<T>(h);
    fill_params(P, G, p, g, lf_a);
    if (G.pre32) fill_params(h->pf, G, p, g, lf_a);          // the float32 twin for the spectrum stages
    CK(cudaMemset(h->ws + h->L.dbg, 0, sizeof(int)));
    P.dbg = (int *)(h->ws + h->L.dbg);
    if (G.pre32) h->pf.dbg = P.dbg;
    if (G.has_gamma) P.gamma_half = F<T>(h, h->L.gamma);
    if (G.exact_t) P.tfac = F<T>(h, h->L.tfac);
    P.t64 = G.t64 ? 1 : 0;
    if (G.rtab) {
        P.rtab = F<T>(h, h->L.rtab);
        CK(launch_rho_table<T>(F<T>(h, h->L.theta), G.modes, (int)G.nt, F<T>(h, h->L.rtab), h->stream));
    }
    if (G.blu_log2L) {
        P.blu_tw = h->ws + h->L.blu_tw;
        P.blu_c = h->ws + h->L.blu_c;
        P.blu_b = h->ws + h->L.blu_b;
    }
    CK(init_plain_attributes<T>());
    if (G.pre32) CK(init_plain_attributes<float>());
    return PDHG_OK;
}

template <typename T>
static cudaError_t enqueue_check(pdhg_handle *h) {
    const Params<T> &P = params_of<T>(h);
    return stage(h, PDHG_STAGE_CHECK, 2, [&] {
        if (check2d_applies<T>(P)) {
            const int64_t nb = check_blocks<T>(P);
            cudaError_t e = launch_check2d<T>(P, F<T>(h, h->u_off), F<T>(h, h->L.phi), F<T>(h, h->L.lam),
                                              F<T>(h, h->L.u0), F<double>(h, h->L.partials),
                                              (int)(nb / (P.nt + 1)), h->stream);
            if (e != cudaSuccess) return e;
            return launch_reduce6(F<double>(h, h->L.partials), nb, F<double>(h, h->L.scal), h->stream);
        }
        return launch_check<T>(P, F<T>(h, h->u_off), F<T>(h, h->L.phi), F<T>(h, h->L.lam), F<T>(h, h->L.u0),
                               F<double>(h, h->L.partials), F<double>(h, h->L.scal), h->stream);
    });
}

#ifdef PDHG_DEBUG
// Debug builds: one block per canary region of the handle's workspace; a changed byte
// records site 900 + region in the debug flag (the first site recorded is kept).
struct CanaryList {
    int n;
    unsigned long long off[kMaxCanaries];
    unsigned len[kMaxCanaries];
};

__global__ void k_canary_check(const unsigned char *__restrict__ ws, CanaryList c, int *dbg) {
    const int r = blockIdx.x;
    if (r >= c.n) return;
    const unsigned char *q = ws + c.off[r];
    bool bad = false;
    for (unsigned i = threadIdx.x; i < c.len[r]; i += blockDim.x) bad |= q[i] != kCanaryByte;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(dbg, 0, 900 + r);
}

static CanaryList canaries_of(const pdhg_handle *h) {
    CanaryList c;
    c.n = h->L.ncan;
    for (int i = 0; i < c.n; ++i) { c.off[i] = h->L.can_off[i]; c.len[i] = h->L.can_len[i]; }
    return c;
}

static cudaError_t canary_fill(pdhg_handle *h) {
    for (int i = 0; i < h->L.ncan; ++i) {
        cudaError_t e = cudaMemsetAsync(h->ws + h->L.can_off[i], kCanaryByte, h->L.can_len[i], h->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t canary_check(pdhg_handle *h, cudaStream_t s) {
    if (h->L.ncan == 0) return cudaSuccess;
    k_canary_check<<<h->L.ncan, 256, 0, s>>>((const unsigned char *)h->ws, canaries_of(h), (int *)(h->ws + h->L.dbg));
    return cudaGetLastError();
}
#endif

// message of a recorded debug site: a canary region (900 + region) or an index check
static std::string debug_site_message(int bad) {
    if (bad >= 900 && bad < 900 + kMaxCanaries)
        return "debug canary check: the bytes after workspace buffer " + std::to_string(bad - 900) +
               " (in layout order) were overwritten";
    return "debug bounds check: out-of-range index at site " + std::to_string(bad);
}

static pdhg_status read_res(pdhg_handle *h, double out[4]) {
    double acc[6];
    int err = 0;
#ifdef PDHG_DEBUG
    CK(canary_check(h, h->stream));
#endif
    CK(cudaMemcpyAsync(acc, h->ws + h->L.scal, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
    int bad = 0;
    if (h->G.fused) CK(cudaMemcpyAsync(&err, h->fused.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&bad, h->ws + h->L.dbg, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (err) return fail(PDHG_ERR_TIMEOUT, "a pipelined spectrum load of the fused rows-C kernel did not arrive");
    if (bad) return fail(PDHG_ERR_BOUNDS, debug_site_message(bad));
    double ht = h->ht, wx = h->wx;
    // space-time L2 (weight h_t w_x per equation value), or, for the one-step
    // problems of Algorithm 3, L2 over the domain at one time (weight w_x)
    const double we = h->res_norm == 1 ? wx : ht * wx;
    double a2 = we * acc[0], b2 = we * acc[1], gap = we * acc[2], c2 = wx * acc[3];
    if (h->G.init == PDHG_INIT_LAMBDA) {
        a2 += c2;
        b2 += wx * acc[4];
        gap += wx * acc[5];
    }
    out[0] = std::sqrt(a2); out[1] = std::sqrt(b2); out[2] = std::sqrt(c2); out[3] = gap;
    return PDHG_OK;
}

template <typename T>
static pdhg_status compute_res(pdhg_handle *h, double out[4]) {
    cudaError_t e = enqueue_check<T>(h);
    if (e != cudaSuccess) return cuda_fail(e, "residual check");
    return read_res(h, out);
}

// Lax-Friedrichs constant: explicit, or max |f'(u0)| when 0 (1 if that is 0 too)
// The Lax-Friedrichs constant: prob->lf_a, or max |f'(u0)| when that is 0 (maxdf: that
// maximum when already known, e.g. from the device scan of a u0 in device memory).
static double lf_constant(const pdhg_problem *prob, const Geom &G, double maxdf = -1.0) {
    double lf_a = prob->lf_a;
    if ((G.space == PDHG_SPACE_FD_LF || G.space == PDHG_SPACE_DG_P2_LF || G.space == PDHG_SPACE_DG_P1_LF) &&
        lf_a == 0.0) {
        if (maxdf >= 0.0) lf_a = maxdf;
        else
            for (int64_t i = 0; i < G.S; ++i)
                lf_a = std::max(lf_a, std::fabs(2 * prob->alpha * prob->u0[i] + prob->beta));
        if (lf_a == 0.0) lf_a = 1.0;
    }
    return lf_a;
}

// max |f'(u0)| and the non-finite count of a device u0, through `scratch` (16 bytes of
// device memory); synchronises the stream.
static pdhg_status scan_device_u0(const pdhg_problem *p, int64_t n, void *scratch, cudaStream_t s, double *maxdf,
                                  unsigned long long *bad) {
    unsigned long long *d = (unsigned long long *)scratch, hv[2];
    CK(cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), s));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
    k_u0_scan<<<blocks, 256, 0, s>>>(p->u0, n, p->alpha, p->beta, d);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(hv, d, sizeof(hv), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    long long bits = (long long)hv[0];
    memcpy(maxdf, &bits, sizeof(double));
    *bad = hv[1];
    return PDHG_OK;
}

template <typename T>
static pdhg_status initial_res_sum(pdhg_handle *h, double *a0) {
    const Params<T> &P = params_of<T>(h);
    cudaError_t e = launch_check<T>(P, F<T>(h, h->u_off), F<T>(h, h->L.phi), F<T>(h, h->L.lam), F<T>(h, h->L.u0),
                                    F<double>(h, h->L.partials), F<double>(h, h->L.scal), h->stream, 1);
    if (e != cudaSuccess) return cuda_fail(e, "initial residual");
    double acc[6];
    CK(cudaMemcpyAsync(acc, h->ws + h->L.scal, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *a0 = acc[0];
    return PDHG_OK;
}

static pdhg_status create_impl(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                               void *workspace, size_t bytes, void *stream, pdhg_handle **out, bool pre32) {
    Geom G;
    pdhg_status st = validate(prob, grid, scheme, &G, pre32);
    if (st != PDHG_OK) return st;
    if (!out) return fail(PDHG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    Layout L = layout_of(G);
    if (!workspace) return fail(PDHG_ERR_INVALID_ARG, "workspace is NULL");
    if (((uintptr_t)workspace & 255) != 0) return fail(PDHG_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (bytes < L.total) return fail(PDHG_ERR_WORKSPACE_TOO_SMALL, "workspace too small: need " + std::to_string(L.total));
    const bool u0_dev = (scheme->flags & PDHG_FLAG_U0_ON_DEVICE) != 0;
    double maxdf = -1.0;
    if (u0_dev) {
        unsigned long long bad = 0;
        st = scan_device_u0(prob, G.S, (char *)workspace + L.scal, (cudaStream_t)stream, &maxdf, &bad);
        if (st != PDHG_OK) return st;
        if (bad) return fail(PDHG_ERR_INVALID_ARG, "u0 has a non-finite value");
    } else {
        for (int64_t i = 0; i < G.S; ++i)
            if (!std::isfinite(prob->u0[i])) return fail(PDHG_ERR_INVALID_ARG, "u0 has a non-finite value");
    }
    const double lf_a = lf_constant(prob, G, maxdf);
    if (G.has_gamma)
        for (int64_t i = 0; i < G.nx; ++i)
            if (!std::isfinite(prob->gamma_half[i])) return fail(PDHG_ERR_INVALID_ARG, "gamma_half non-finite");
    pdhg_handle *h = new pdhg_handle();
    h->G = G; h->L = L; h->ws = (char *)workspace; h->stream = (cudaStream_t)stream;
    h->u0_dev = u0_dev;
    h->ht = grid->T / (double)grid->nt;
    double hx = grid->lx / (double)grid->nx;
    h->wx = G.dims == 2 ? hx * (grid->ly / (double)grid->ny) : hx;
    h->iters = 0; h->launches = 0; h->profiling = false;
    h->res_norm = 0;
    for (int k = 0; k < 4; ++k) h->last_res[k] = NAN;
    // CUDA graphs of m iterations and the check: the plain path, and fused problems small
    // enough (<= 2^23 cell-iterations) for launch gaps to matter
    h->graphs = !G.fused || (double)G.nt * (double)G.S <= (double)(int64_t(1) << 23);
    h->gexec = nullptr; h->gstream = nullptr; h->gchunk = 0; h->glaunches = 0;
    h->u_off = L.u;
#ifdef PDHG_DEBUG
    if (cudaError_t e = canary_fill(h); e != cudaSuccess) { delete h; return cuda_fail(e, "canary fill"); }
#endif
    memset(h->stage_ms, 0, sizeof(h->stage_ms));
    memset(h->stage_n, 0, sizeof(h->stage_n));
    st = (G.prec == PDHG_FP64) ? upload_tables<double>(h, prob, grid, lf_a) : upload_tables<float>(h, prob, grid, lf_a);
    if (st == PDHG_OK && G.fused) {
        cudaError_t e = fused2d_init(&h->fused, h->pf, h->ws + L.fused, F<float>(h, L.twx), F<float>(h, L.twy),
                                     F<float>(h, L.theta));
        if (e != cudaSuccess) st = cuda_fail(e, "fused2d_init");
    }
    // ||A(u_init)||: at [u0, 0, 0] every slice's residual is D(u0) (the time differences
    // vanish) and the initial row and the phi, lambda terms are zero, so slice 0's sum
    // times nt gives it without a pass over all slices
    double a0 = 0.0;
    if (st == PDHG_OK) st = (G.prec == PDHG_FP64) ? initial_res_sum<double>(h, &a0) : initial_res_sum<float>(h, &a0);
    if (st != PDHG_OK) { delete h; return st; }
    h->res_init = std::sqrt(h->ht * h->wx * (double)G.nt * a0);
    h->launches = 0;
    *out = h;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_create(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                                   void *workspace, size_t bytes, void *stream, pdhg_handle **out) {
    return create_impl(prob, grid, scheme, workspace, bytes, stream, out, false);
}

extern "C" pdhg_status pdhg_destroy(pdhg_handle *h) {
    if (!h) return PDHG_OK;
    graph_drop(h);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    for (auto &r : h->recs) { h->pool.push_back(r.a); h->pool.push_back(r.b); }
    for (auto e : h->pool) if (e) cudaEventDestroy(e);
    delete h;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_set_stream(pdhg_handle *h, void *stream) {
    if (!h) return fail(PDHG_ERR_INVALID_ARG, "null handle");
    CK(cudaStreamSynchronize(h->stream));        // the old stream's work on the state is done
    h->stream = (cudaStream_t)stream;
    return PDHG_OK;
}

template <typename T>
static cudaError_t enqueue_iteration(pdhg_handle *h) {
    const Params<T> &P = params_of<T>(h);
    cudaStream_t s = h->stream;
    T *u = F<T>(h, h->u_off), *phi = F<T>(h, h->L.phi), *phit = F<T>(h, h->L.phit);
    T *lam = F<T>(h, h->L.lam), *lamt = F<T>(h, h->L.lamt), *u0 = F<T>(h, h->L.u0);
    void *spec = h->ws + h->L.spec;
    const void *twx = h->ws + h->L.twx, *twy = h->ws + h->L.twy, *V = h->ws + h->L.V;
    const T *theta = F<T>(h, h->L.theta);
    cudaError_t e;
    if (h->G.fused) {
        if constexpr (sizeof(T) == 4) {
            Fused2D *f = &h->fused;
            float *uf = F<float>(h, h->u_off);
            e = stage(h, PDHG_STAGE_PRIMAL, 1, [&] {
                return fused2d_primal(h->pf, uf, phit, lam, lamt, u0, s);
            });
            if (e != cudaSuccess) return e;
            e = stage(h, PDHG_STAGE_FUSED_ROWS, 1, [&] { return fused2d_rowsR(f, h->pf, uf, s); });
            if (e != cudaSuccess) return e;
            e = stage(h, PDHG_STAGE_FUSED_COLS, 1, [&] { return fused2d_cols(f, h->pf, s); });
            if (e != cudaSuccess) return e;
            return stage(h, PDHG_STAGE_DUAL, 1, [&] { return fused2d_rowsC(f, h->pf, phi, phit, s); });
        }
        return cudaErrorInvalidValue;
    }
    e = stage(h, PDHG_STAGE_PRIMAL, 1, [&] { return launch_primal<T>(P, u, phit, lam, lamt, u0, s); });
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(T) == 8) {
        if (h->G.pre32) {
            // float64 state, K_d^{-1} applied in float32 on a float32 spectrum (in the
            // float64 spectrum's buffer) with the float32 twin of the parameters
            const Params<float> &Q = h->pf;
            const void *tx = h->ws + h->L.twx32, *ty = h->ws + h->L.twy32;
            const float *th32 = F<float>(h, h->L.theta32);
            e = stage(h, PDHG_STAGE_RESIDUAL_FFT, 1, [&] { return launch_residual_rfft_p32(P, u, spec, tx, s); });
            if (e != cudaSuccess) return e;
            if (h->G.dims == 2) {
                e = stage(h, PDHG_STAGE_FFT_Y, 1, [&] { return launch_fft_y<float>(Q, spec, ty, 0, s); });
                if (e != cudaSuccess) return e;
            }
            e = stage(h, PDHG_STAGE_TSOLVE, 1, [&] { return launch_tsolve<float>(Q, spec, th32, nullptr, s); });
            if (e != cudaSuccess) return e;
            if (h->G.dims == 2) {
                e = stage(h, PDHG_STAGE_FFT_Y, 1, [&] { return launch_fft_y<float>(Q, spec, ty, 1, s); });
                if (e != cudaSuccess) return e;
            }
            return stage(h, PDHG_STAGE_DUAL, 1, [&] { return launch_dual_irfft_p32(P, spec, phi, phit, tx, s); });
        }
    }
    e = stage(h, PDHG_STAGE_RESIDUAL_FFT, 1, [&] { return launch_residual_rfft<T>(P, u, spec, twx, s); });
    if (e != cudaSuccess) return e;
    if (h->G.dims == 2) {
        e = stage(h, PDHG_STAGE_FFT_Y, 1, [&] { return launch_fft_y<T>(P, spec, twy, 0, s); });
        if (e != cudaSuccess) return e;
    }
    e = stage(h, PDHG_STAGE_TSOLVE, 1, [&] { return launch_tsolve<T>(P, spec, theta, V, s); });
    if (e != cudaSuccess) return e;
    if (h->G.dims == 2) {
        e = stage(h, PDHG_STAGE_FFT_Y, 1, [&] { return launch_fft_y<T>(P, spec, twy, 1, s); });
        if (e != cudaSuccess) return e;
    }
    return stage(h, PDHG_STAGE_DUAL, 1, [&] { return launch_dual_irfft<T>(P, spec, phi, phit, twx, s); });
}

// Capture m iterations and the residual check as one graph (on a private stream;
// replayed on the handle's stream).  Returns an error if capture is not possible;
// the caller then launches kernel by kernel.
template <typename T>
static cudaError_t graph_build(pdhg_handle *h, int32_t m) {
    graph_drop(h);
    cudaError_t e = cudaSuccess;
    if (!h->gstream) e = cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaStream_t user = h->stream;
    const int64_t l0 = h->launches;
    h->stream = h->gstream;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int32_t i = 0; i < m && e == cudaSuccess; ++i) e = enqueue_iteration<T>(h);
        if (e == cudaSuccess) e = enqueue_check<T>(h);
        cudaError_t e2 = cudaStreamEndCapture(h->gstream, &g);
        if (e == cudaSuccess) e = e2;
    }
    h->stream = user;
    h->glaunches = h->launches - l0;
    h->launches = l0;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e == cudaSuccess) h->gchunk = m;
    else graph_drop(h);
    return e;
}

template <typename T>
static pdhg_status iterate_T(pdhg_handle *h, int64_t max_iters, double tol, int32_t check_every, int32_t relative,
                             int64_t *done) {
    int64_t n = 0;
    double scale = relative ? h->res_init : 1.0;
    for (; n < max_iters;) {
        double r[4];
        pdhg_status st;
        const bool chunk = h->graphs && !h->profiling && check_every > 0 && max_iters - n >= check_every;
        if (chunk && h->gchunk != check_every && graph_build<T>(h, check_every) != cudaSuccess) {
            cudaGetLastError();                          // capture refused: launch kernel by kernel
            h->graphs = false;
        }
        if (chunk && h->gchunk == check_every) {
            cudaError_t e = cudaGraphLaunch(h->gexec, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
            n += check_every;
            h->iters += check_every;
            h->launches += h->glaunches;
            st = read_res(h, r);
        } else {
            cudaError_t e = enqueue_iteration<T>(h);
            if (e != cudaSuccess) return cuda_fail(e, "iteration launch");
            ++n;
            ++h->iters;
            if (!(check_every > 0 && (n % check_every == 0 || n == max_iters))) continue;
            st = compute_res<T>(h, r);
        }
        {
            if (st != PDHG_OK) { if (done) *done = n; return st; }
            history_push(h, r);
            if (!std::isfinite(r[0]) || !std::isfinite(r[1])) {
                if (done) *done = n;
                return fail(PDHG_ERR_NONFINITE, "residual is not finite after " + std::to_string(h->iters) + " iterations");
            }
            if (r[0] > 1e10 * std::max(h->res_init, 1e-300)) {
                if (done) *done = n;
                return fail(PDHG_ERR_DIVERGED, "primal residual grew by more than 1e10");
            }
            for (int k = 0; k < 4; ++k) h->last_res[k] = r[k];
            if (r[0] <= tol * scale && r[1] <= tol * scale) break;
        }
    }
    if (done) *done = n;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_iterate(pdhg_handle *h, int64_t max_iters, double tol, int32_t check_every,
                                    int32_t relative, int64_t *iters_done) {
    if (!h) return fail(PDHG_ERR_INVALID_ARG, "null handle");
    if (max_iters < 0) return fail(PDHG_ERR_INVALID_ARG, "max_iters < 0");
    if (iters_done) *iters_done = 0;
    return h->G.prec == PDHG_FP64 ? iterate_T<double>(h, max_iters, tol, check_every, relative, iters_done)
                                  : iterate_T<float>(h, max_iters, tol, check_every, relative, iters_done);
}

extern "C" pdhg_status pdhg_residual_history(pdhg_handle *h, double *out, int64_t max_rows, int64_t *rows,
                                             int32_t clear) {
    if (!h || !rows) return fail(PDHG_ERR_INVALID_ARG, "null handle or rows");
    if (max_rows < 0 || (max_rows > 0 && !out)) return fail(PDHG_ERR_INVALID_ARG, "out is NULL or max_rows < 0");
    const int64_t n = std::min(h->hist_count, max_rows);
    // the oldest kept row is hist_next - hist_count; copy the oldest n of the kept rows
    const int64_t first = h->hist_next - h->hist_count;
    for (int64_t i = 0; i < n; ++i) {
        const double *row = h->hist.data() + (size_t)((first + i) % kHistoryRows) * 5;
        std::copy(row, row + 5, out + i * 5);
    }
    *rows = max_rows > 0 ? n : h->hist_count;
    if (clear) h->hist_count = 0;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_residual(pdhg_handle *h, double out[4]) {
    if (!h || !out) return fail(PDHG_ERR_INVALID_ARG, "null handle or out");
    return h->G.prec == PDHG_FP64 ? compute_res<double>(h, out) : compute_res<float>(h, out);
}

static pdhg_status field_of(pdhg_handle *h, int32_t field, size_t *off, size_t *count, bool for_set) {
    const Geom &G = h->G;
    switch (field) {
    case PDHG_FIELD_U: *off = h->u_off; *count = (G.nt + 1) * G.S; break;
    case PDHG_FIELD_U_TERMINAL:
        if (for_set) return fail(PDHG_ERR_INVALID_ARG, "U_TERMINAL is read-only");
        *off = h->u_off + G.nt * G.S * G.esz; *count = G.S; break;
    case PDHG_FIELD_PHI: *off = h->L.phi; *count = G.nt * G.S; break;
    case PDHG_FIELD_PHIT: *off = h->L.phit; *count = G.nt * G.S; break;
    case PDHG_FIELD_LAMBDA: *off = h->L.lam; *count = G.S; break;
    case PDHG_FIELD_LAMBDAT: *off = h->L.lamt; *count = G.S; break;
    default: return fail(PDHG_ERR_INVALID_ARG, "unknown field");
    }
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_field(pdhg_handle *h, int32_t field, void *dst, int32_t on_device) {
    if (!h || !dst) return fail(PDHG_ERR_INVALID_ARG, "null handle or dst");
    size_t off, count;
    pdhg_status st = field_of(h, field, &off, &count, false);
    if (st != PDHG_OK) return st;
    CK(cudaMemcpyAsync(dst, h->ws + off, count * h->G.esz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_solution(pdhg_handle *h, void *dst, int32_t dst_on_device, int32_t which) {
    if (which != PDHG_FIELD_U && which != PDHG_FIELD_U_TERMINAL && which != PDHG_FIELD_PHI &&
        which != PDHG_FIELD_LAMBDA)
        return fail(PDHG_ERR_INVALID_ARG, "which must be PDHG_FIELD_U, _U_TERMINAL, _PHI or _LAMBDA");
    return pdhg_get_field(h, which, dst, dst_on_device);
}

extern "C" pdhg_status pdhg_set_field(pdhg_handle *h, int32_t field, const void *src, int32_t on_device) {
    if (!h || !src) return fail(PDHG_ERR_INVALID_ARG, "null handle or src");
    size_t off, count;
    pdhg_status st = field_of(h, field, &off, &count, true);
    if (st != PDHG_OK) return st;
    CK(cudaMemcpyAsync(h->ws + off, src, count * h->G.esz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_info(pdhg_handle *h, int64_t *ndof, int64_t *nt, int64_t *iterations, int32_t *precision,
                                 int32_t *path) {
    if (!h) return fail(PDHG_ERR_INVALID_ARG, "null handle");
    if (ndof) *ndof = h->G.S;
    if (nt) *nt = h->G.nt;
    if (iterations) *iterations = h->iters;
    if (precision) *precision = h->G.prec;
    if (path) *path = h->G.fused ? PDHG_PATH_FUSED : PDHG_PATH_PLAIN;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_launch_count(pdhg_handle *h, int64_t *launches, int32_t reset) {
    if (!h || !launches) return fail(PDHG_ERR_INVALID_ARG, "null handle or launches");
    *launches = h->launches;
    if (reset) h->launches = 0;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_set_profiling(pdhg_handle *h, int32_t enable) {
    if (!h) return fail(PDHG_ERR_INVALID_ARG, "null handle");
    h->profiling = enable != 0;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_stage_times(pdhg_handle *h, double ms[PDHG_NUM_STAGES], int64_t launches[PDHG_NUM_STAGES]) {
    if (!h || !ms || !launches) return fail(PDHG_ERR_INVALID_ARG, "null argument");
    CK(cudaStreamSynchronize(h->stream));
    for (auto &r : h->recs) {
        float t = 0.f;
        if (r.a && r.b && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            h->stage_ms[r.stage] += t;
            h->stage_n[r.stage] += 1;
        }
        if (r.a) h->pool.push_back(r.a);
        if (r.b) h->pool.push_back(r.b);
    }
    h->recs.clear();
    for (int i = 0; i < PDHG_NUM_STAGES; ++i) {
        ms[i] = h->stage_ms[i]; launches[i] = h->stage_n[i];
        h->stage_ms[i] = 0; h->stage_n[i] = 0;
    }
    return PDHG_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 2 (Sec. 3.4): refinement of the time mesh.  Level k has nt >> (levels-1-k)
// slices; consecutive levels live in two alternating regions of the workspace (region
// A holds the final level), so a level is created before the previous one is freed.
// ---------------------------------------------------------------------------
static pdhg_grid level_grid(const pdhg_grid *g, int32_t levels, int32_t k) {
    pdhg_grid c = *g;
    c.nt = g->nt >> (levels - 1 - k);
    return c;
}

static pdhg_status refine_regions(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                                  int32_t levels, size_t *a, size_t *b) {
    if (!grid) return fail(PDHG_ERR_INVALID_ARG, "null grid");
    if (levels < 1 || levels > 16) return fail(PDHG_ERR_INVALID_ARG, "levels must be in [1, 16]");
    if (grid->nt < 1 || (grid->nt % (int64_t(1) << (levels - 1))) != 0)
        return fail(PDHG_ERR_INVALID_ARG, "nt must be divisible by 2^(levels-1)");
    *a = *b = 0;
    for (int32_t k = 0; k < levels; ++k) {
        pdhg_grid gk = level_grid(grid, levels, k);
        size_t n = 0;
        pdhg_status st = pdhg_workspace_size(prob, &gk, scheme, &n);
        if (st != PDHG_OK) return st;
        size_t &r = ((levels - 1 - k) % 2 == 0) ? *a : *b;
        r = std::max(r, n);
    }
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_refine_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                                  const pdhg_scheme *scheme, int32_t levels, size_t *bytes) {
    if (!bytes) return fail(PDHG_ERR_INVALID_ARG, "bytes is NULL");
    size_t a, b;
    pdhg_status st = refine_regions(prob, grid, scheme, levels, &a, &b);
    if (st != PDHG_OK) return st;
    *bytes = align256(a) + b;
    return PDHG_OK;
}

template <typename T>
static cudaError_t transfer_level(pdhg_handle *c, pdhg_handle *f) {
    const int64_t S = c->G.S;
    cudaError_t e = launch_interp_t<T>(F<T>(c, c->u_off), F<T>(c, c->L.phi), F<T>(f, f->u_off), F<T>(f, f->L.phi),
                                       F<T>(f, f->L.phit), S, c->G.nt, f->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f->ws + f->L.lam, c->ws + c->L.lam, S * sizeof(T), cudaMemcpyDeviceToDevice, f->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f->ws + f->L.lamt, c->ws + c->L.lam, S * sizeof(T), cudaMemcpyDeviceToDevice, f->stream);
    f->launches += 1;
    return e;
}

extern "C" pdhg_status pdhg_solve_refine(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                                         int32_t levels, const int64_t *iters, double tol, int32_t check_every,
                                         int32_t relative, void *workspace, size_t bytes, void *stream,
                                         pdhg_handle **out, int64_t *iters_done) {
    if (!out || !iters) return fail(PDHG_ERR_INVALID_ARG, "out or iters is NULL");
    *out = nullptr;
    size_t a, b;
    pdhg_status st = refine_regions(prob, grid, scheme, levels, &a, &b);
    if (st != PDHG_OK) return st;
    if (!workspace) return fail(PDHG_ERR_INVALID_ARG, "workspace is NULL");
    if (bytes < align256(a) + b)
        return fail(PDHG_ERR_WORKSPACE_TOO_SMALL, "workspace too small: need " + std::to_string(align256(a) + b));
    for (int32_t k = 0; k < levels; ++k)
        if (iters[k] < 0) return fail(PDHG_ERR_INVALID_ARG, "iters[k] < 0");
    char *ra = (char *)workspace, *rb = ra + align256(a);
    pdhg_handle *prev = nullptr;
    for (int32_t k = 0; k < levels; ++k) {
        pdhg_grid gk = level_grid(grid, levels, k);
        const bool in_a = (levels - 1 - k) % 2 == 0;
        pdhg_handle *hk = nullptr;
        st = pdhg_create(prob, &gk, scheme, in_a ? ra : rb, in_a ? a : b, stream, &hk);
        if (st != PDHG_OK) { pdhg_destroy(prev); return st; }
        if (prev) {
            cudaError_t e = hk->G.prec == PDHG_FP64 ? transfer_level<double>(prev, hk) : transfer_level<float>(prev, hk);
            pdhg_destroy(prev);
            prev = nullptr;
            if (e != cudaSuccess) { pdhg_destroy(hk); return cuda_fail(e, "time-mesh transfer"); }
        }
        int64_t done = 0;
        st = pdhg_iterate(hk, iters[k], tol, check_every, relative, &done);
        if (iters_done) iters_done[k] = done;
        if (st != PDHG_OK) { pdhg_destroy(hk); return st; }
        prev = hk;
    }
    *out = prev;
    return PDHG_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 3 (Sec. 3.5): one time step at a time.  One handle of nt = 1 on
// [0, h_t] is reused for every step: its u0 becomes the previous end value, its
// state restarts at [u0, u0], 0, 0, and its residual is the per-slice one.
// ---------------------------------------------------------------------------
static pdhg_status one_step_inputs(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                                   pdhg_problem *p1, pdhg_grid *g1) {
    if (!prob || !grid || !scheme) return fail(PDHG_ERR_INVALID_ARG, "null problem/grid/scheme");
    if (scheme->flags & PDHG_FLAG_U0_ON_DEVICE)
        return fail(PDHG_ERR_UNSUPPORTED, "the one-step variant takes u0 in host memory");
    pdhg_scheme sv = *scheme;
    if (sv.flags & PDHG_FLAG_MIXED_STEPS) {
        sv.flags &= ~(int32_t)PDHG_FLAG_MIXED_STEPS;
        sv.precision = PDHG_FP64;
    }
    Geom G;
    pdhg_status st = validate(prob, grid, &sv, &G);
    if (st != PDHG_OK) return st;
    *g1 = *grid;
    g1->nt = 1;
    g1->T = grid->T / (double)grid->nt;
    *p1 = *prob;
    for (int64_t i = 0; i < G.S; ++i)
        if (!std::isfinite(prob->u0[i])) return fail(PDHG_ERR_INVALID_ARG, "u0 has a non-finite value");
    p1->lf_a = lf_constant(prob, G);          // the full problem's constant, for every step
    return PDHG_OK;
}

// The one-step problems are backward-Euler problems: with BDF2 the step l >= 1 is the BE
// step of length 2 h_t / 3 from (4 u^l - u^{l-1}) / 3, on a second handle.
static pdhg_scheme one_step_scheme(const pdhg_scheme *scheme) {
    pdhg_scheme s1 = *scheme;
    s1.time = PDHG_TIME_BE;
    s1.flags &= ~(int32_t)PDHG_FLAG_MIXED_STEPS;
    return s1;
}

static pdhg_status mixed_schemes(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                                 pdhg_scheme *s32, pdhg_scheme *s64, size_t *b32, size_t *b64);

// workspace of one step length: one handle, or (mixed steps) a float32 handle and a
// float64 one; two step lengths for BDF2
static pdhg_status one_step_region(const pdhg_problem *p1, const pdhg_grid *g1, const pdhg_scheme *scheme,
                                   size_t *region, size_t *b32, size_t *b64) {
    const pdhg_scheme s1 = one_step_scheme(scheme);
    if (scheme->flags & PDHG_FLAG_MIXED_STEPS) {
        pdhg_scheme s32, s64;
        pdhg_status st = mixed_schemes(p1, g1, &s1, &s32, &s64, b32, b64);
        if (st != PDHG_OK) return st;
        *region = align256(*b32) + align256(*b64);
        return PDHG_OK;
    }
    *b64 = 0;
    pdhg_status st = pdhg_workspace_size(p1, g1, &s1, b32);
    *region = align256(*b32);
    return st;
}

extern "C" pdhg_status pdhg_one_step_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                                    const pdhg_scheme *scheme, size_t *bytes) {
    if (!bytes) return fail(PDHG_ERR_INVALID_ARG, "bytes is NULL");
    pdhg_problem p1;
    pdhg_grid g1;
    pdhg_status st = one_step_inputs(prob, grid, scheme, &p1, &g1);
    if (st != PDHG_OK) return st;
    size_t region, b32, b64;
    st = one_step_region(&p1, &g1, scheme, &region, &b32, &b64);
    if (st != PDHG_OK) return st;
    *bytes = (scheme->time == PDHG_TIME_BDF2 ? 2 : 1) * region;
    return PDHG_OK;
}

// w = (4 u^l - u^{l-1}) / 3, the start of a BDF2 step written as a BE step
template <typename T>
__global__ void k_bdf2_start(const T *__restrict__ ul, const T *__restrict__ ulm, T *__restrict__ w, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = (T(4) * ul[i] - ulm[i]) / T(3);
}

static cudaError_t restart_step(pdhg_handle *h, const char *u_start) {
    const size_t sb = h->G.S * h->G.esz;
    cudaError_t e = cudaMemcpyAsync(h->ws + h->L.u0, u_start, sb, cudaMemcpyDeviceToDevice, h->stream);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s)
        e = cudaMemcpyAsync(h->ws + h->u_off + s * sb, u_start, sb, cudaMemcpyDeviceToDevice, h->stream);
    const size_t zero[4] = {h->L.phi, h->L.phit, h->L.lam, h->L.lamt};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMemsetAsync(h->ws + zero[i], 0, sb, h->stream);
    return e;
}

// the float32 handle of a mixed step restarted from a float64 start value
static cudaError_t restart_step_narrow(pdhg_handle *h, const double *u_start) {
    const int64_t S = h->G.S;
    const size_t sb = S * sizeof(float);
    k_u0_convert<float><<<(unsigned)std::min<int64_t>((S + 255) / 256, 1024), 256, 0, h->stream>>>(
        u_start, F<float>(h, h->L.u0), S);
    cudaError_t e = cudaGetLastError();
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(h->ws + h->u_off + k * sb, h->ws + h->L.u0, sb, cudaMemcpyDeviceToDevice, h->stream);
    const size_t zero[4] = {h->L.phi, h->L.phit, h->L.lam, h->L.lamt};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMemsetAsync(h->ws + zero[i], 0, sb, h->stream);
    return e;
}

// one mixed step: float32 iterations until Res <= tol or the float32 floor (the worse
// entry of Res not 5% lower than three checks before), then the state widened to the
// float64 handle (u^0 and its initial data the exact float64 start value) and float64
// iterations to tol, checked after 1, 2, 3, 4, 6, 9, ... of them (as pdhg_solve_mixed)
static pdhg_status mixed_step(pdhg_handle *hf, pdhg_handle *hd, const double *u_start, double tol, int64_t cap,
                              int32_t check_every, int64_t *n32_out, int64_t *n64_out) {
    *n32_out = *n64_out = 0;
    cudaError_t e = restart_step_narrow(hf, u_start);
    if (e != cudaSuccess) return cuda_fail(e, "mixed step restart");
    std::vector<double> hist;
    int64_t n32 = 0;
    bool done32 = false;
    while (n32 < cap && !done32) {
        int64_t done = 0;
        pdhg_status st = pdhg_iterate(hf, std::min<int64_t>(check_every, cap - n32), tol, check_every, 0, &done);
        n32 += done;
        *n32_out = n32;
        if (st != PDHG_OK) return st;
        if (hf->last_res[0] <= tol && hf->last_res[1] <= tol) done32 = true;
        hist.push_back(std::max(hf->last_res[0], hf->last_res[1]));
        if (hist.size() >= 4 && hist.back() > 0.95 * hist[hist.size() - 4]) break;
    }
    const int64_t S = hf->G.S;
    struct { size_t src, dst; int64_t n; } parts[5] = {
        {hf->u_off, hd->u_off, 2 * S}, {hf->L.phi, hd->L.phi, S}, {hf->L.phit, hd->L.phit, S},
        {hf->L.lam, hd->L.lam, S}, {hf->L.lamt, hd->L.lamt, S}};
    for (int i = 0; i < 5 && e == cudaSuccess; ++i)
        e = launch_widen((const float *)(hf->ws + parts[i].src), (double *)(hd->ws + parts[i].dst), parts[i].n,
                         hd->stream);
    const size_t sb = S * sizeof(double);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd->ws + hd->L.u0, u_start, sb, cudaMemcpyDeviceToDevice, hd->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd->ws + hd->u_off, u_start, sb, cudaMemcpyDeviceToDevice, hd->stream);
    hd->launches += 5;
    if (e != cudaSuccess) return cuda_fail(e, "float32 -> float64 hand-over");
    int64_t n64 = 0;
    // a step's float64 phase takes about as many iterations as a float64 step (its start
    // is the float32 floor, not the solution): checks after 1, 2, 3, 4, 6, 9, ... of them,
    // then every check_every, whose full chunks replay one CUDA graph
    const int64_t ccap = std::max<int32_t>(1, check_every);
    while (n64 < cap) {
        const int64_t chunk = std::min<int64_t>(std::min<int64_t>(std::max<int64_t>(1, n64 / 2), ccap), cap - n64);
        int64_t done = 0;
        hd->graphs = chunk == ccap;
        pdhg_status st = pdhg_iterate(hd, chunk, tol, (int32_t)chunk, 0, &done);
        n64 += done;
        *n64_out = n64;
        if (st != PDHG_OK) return st;
        if (hd->last_res[0] <= tol && hd->last_res[1] <= tol) break;
    }
    return PDHG_OK;
}

// Algorithm 3 with mixed steps: per step length a float32 and a float64 handle (the
// float64 one applies K_d^{-1} in float32, as the float64 phase of pdhg_solve_mixed)
static pdhg_status one_step_mixed(const pdhg_problem *p1, const pdhg_grid *g1, const pdhg_scheme *s1, bool bdf2,
                                  int64_t nt, double tol, int64_t cap, int32_t check_every, char *ws, size_t region,
                                  size_t b32, size_t b64, cudaStream_t stream, double *uo, int64_t *iters_per_step,
                                  int64_t *iters_total) {
    pdhg_scheme s32, s64;
    size_t c32, c64;
    pdhg_status st = mixed_schemes(p1, g1, s1, &s32, &s64, &c32, &c64);
    if (st != PDHG_OK) return st;
    pdhg_handle *hf[2] = {nullptr, nullptr}, *hd[2] = {nullptr, nullptr};
    auto cleanup = [&] {
        for (int k = 0; k < 2; ++k) { pdhg_destroy(hf[k]); pdhg_destroy(hd[k]); }
    };
    for (int k = 0; k < (bdf2 ? 2 : 1); ++k) {
        pdhg_grid gk = *g1;
        if (k == 1) gk.T = 2.0 * g1->T / 3.0;
        char *r = ws + k * region;
        st = pdhg_create(p1, &gk, &s32, r, b32, stream, &hf[k]);
        if (st == PDHG_OK) st = create_impl(p1, &gk, &s64, r + align256(b32), b64, stream, &hd[k], true);
        if (st != PDHG_OK) { cleanup(); return st; }
        hf[k]->res_norm = 1;
        hd[k]->res_norm = 1;
        hd[k]->graphs = false;               // set per chunk in mixed_step: graphs for full chunks only
    }
    const int64_t S = hf[0]->G.S;
    cudaError_t e = cudaMemcpyAsync(uo, hd[0]->ws + hd[0]->L.u0, S * sizeof(double), cudaMemcpyDeviceToDevice, stream);
    int64_t total = 0;
    for (int64_t l = 0; l < nt && st == PDHG_OK; ++l) {
        const int k = (bdf2 && l >= 1) ? 1 : 0;
        const double *start = uo + l * S;
        if (k == 1 && e == cudaSuccess) {
            const unsigned gb = (unsigned)std::min<int64_t>((S + 255) / 256, 1024);
            k_bdf2_start<double><<<gb, 256, 0, stream>>>(uo + l * S, uo + (l - 1) * S, uo + (l + 1) * S, S);
            e = cudaGetLastError();
            start = uo + (l + 1) * S;
        }
        if (e != cudaSuccess) { st = cuda_fail(e, "one-step restart"); break; }
        int64_t n32 = 0, n64 = 0;
        st = mixed_step(hf[k], hd[k], start, tol, cap, check_every, &n32, &n64);
        total += n32 + n64;
        if (iters_per_step) iters_per_step[l] = n32 + n64;
        if (st != PDHG_OK) break;
        e = cudaMemcpyAsync(uo + (l + 1) * S, hd[k]->ws + hd[k]->u_off + S * sizeof(double), S * sizeof(double),
                            cudaMemcpyDeviceToDevice, stream);
    }
    if (st == PDHG_OK && e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (st == PDHG_OK && e != cudaSuccess) st = cuda_fail(e, "one-step copy");
    if (iters_total) *iters_total = total;
    cleanup();
    return st;
}

extern "C" pdhg_status pdhg_solve_one_step(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                                           double tol, int64_t max_iters_per_step, int32_t check_every,
                                           void *workspace, size_t bytes, void *stream, void *u_out,
                                           int64_t *iters_per_step, int64_t *iters_total) {
    pdhg_problem p1;
    pdhg_grid g1;
    pdhg_status st = one_step_inputs(prob, grid, scheme, &p1, &g1);
    if (st != PDHG_OK) return st;
    if (!u_out) return fail(PDHG_ERR_INVALID_ARG, "u_out is NULL");
    if (max_iters_per_step < 1 || check_every < 1)
        return fail(PDHG_ERR_INVALID_ARG, "max_iters_per_step and check_every must be >= 1");
    if (iters_total) *iters_total = 0;
    const pdhg_scheme s1 = one_step_scheme(scheme);
    const bool bdf2 = scheme->time == PDHG_TIME_BDF2;
    size_t region = 0, b1 = 0, b64 = 0;
    st = one_step_region(&p1, &g1, scheme, &region, &b1, &b64);
    if (st != PDHG_OK) return st;
    if (bytes < (bdf2 ? 2 : 1) * region) return fail(PDHG_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
    if (scheme->flags & PDHG_FLAG_MIXED_STEPS)
        return one_step_mixed(&p1, &g1, &s1, bdf2, grid->nt, tol, max_iters_per_step, check_every, (char *)workspace,
                              region, b1, b64, (cudaStream_t)stream, (double *)u_out, iters_per_step, iters_total);
    pdhg_handle *h1 = nullptr, *h2 = nullptr;
    st = pdhg_create(&p1, &g1, &s1, workspace, b1, stream, &h1);
    if (st != PDHG_OK) return st;
    h1->res_norm = 1;
    if (bdf2) {
        pdhg_grid g2 = g1;
        g2.T = 2.0 * g1.T / 3.0;
        st = pdhg_create(&p1, &g2, &s1, (char *)workspace + region, b1, stream, &h2);
        if (st != PDHG_OK) { pdhg_destroy(h1); return st; }
        h2->res_norm = 1;
    }
    pdhg_handle *h = h1;
    const size_t sb = h1->G.S * h1->G.esz;
    char *uo = (char *)u_out;
    cudaError_t e = cudaMemcpyAsync(uo, h1->ws + h1->L.u0, sb, cudaMemcpyDeviceToDevice, h1->stream);
    int64_t total = 0;
    for (int64_t l = 0; l < grid->nt && st == PDHG_OK; ++l) {
        if (bdf2 && l >= 1) {
            // the BDF2 step as a BE step of length 2 h_t / 3 from w, written where u^{l+1} goes
            h = h2;
            const int64_t n = h->G.S;
            const unsigned gb = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
            if (e == cudaSuccess) {
                if (h->G.prec == PDHG_FP64)
                    k_bdf2_start<double><<<gb, 256, 0, h->stream>>>((const double *)(uo + l * sb),
                                                                  (const double *)(uo + (l - 1) * sb),
                                                                  (double *)(uo + (l + 1) * sb), n);
                else
                    k_bdf2_start<float><<<gb, 256, 0, h->stream>>>((const float *)(uo + l * sb),
                                                                 (const float *)(uo + (l - 1) * sb),
                                                                 (float *)(uo + (l + 1) * sb), n);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = restart_step(h, uo + (l + 1) * sb);
        } else if (e == cudaSuccess && l > 0) {
            e = restart_step(h, uo + l * sb);
        }
        if (e != cudaSuccess) { st = cuda_fail(e, "one-step restart"); break; }
        int64_t done = 0;
        st = pdhg_iterate(h, max_iters_per_step, tol, check_every, 0, &done);
        total += done;
        if (iters_per_step) iters_per_step[l] = done;
        if (st != PDHG_OK) break;
        e = cudaMemcpyAsync(uo + (l + 1) * sb, h->ws + h->u_off + sb, sb, cudaMemcpyDeviceToDevice, h->stream);
    }
    if (st == PDHG_OK && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (st == PDHG_OK && e != cudaSuccess) st = cuda_fail(e, "one-step copy");
    if (iters_total) *iters_total = total;
    pdhg_destroy(h1);
    pdhg_destroy(h2);
    return st;
}

// ---------------------------------------------------------------------------
// Gradient of a terminal objective through the solve.  Forward: Algorithm 1 to
// tol.  Adjoint: Algorithm 1 on the problem linearised at the solution u*, with
// the objective |u*^nt + v^nt - target|^2 added (a convex saddle problem whose
// multipliers phi, lambda are the discrete adjoint).  Workspace: the handle's
// (plain path) followed by u* ((nt+1) S values) and target - u*^nt (S values).
// ---------------------------------------------------------------------------
static pdhg_status gradient_inputs(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                                   pdhg_scheme *s1, size_t *handle_bytes, size_t *total) {
    if (!prob || !grid || !scheme) return fail(PDHG_ERR_INVALID_ARG, "null problem/grid/scheme");
    if (scheme->space != PDHG_SPACE_FD_UPWIND && scheme->space != PDHG_SPACE_FD_LF)
        return fail(PDHG_ERR_UNSUPPORTED, "gradients are implemented for the finite-difference schemes");
    if (scheme->init != PDHG_INIT_LAMBDA) return fail(PDHG_ERR_UNSUPPORTED, "gradients need PDHG_INIT_LAMBDA");
    if (scheme->path == PDHG_PATH_FUSED) return fail(PDHG_ERR_UNSUPPORTED, "gradients run on the plain path");
    *s1 = *scheme;
    s1->path = PDHG_PATH_PLAIN;
    Geom G;
    pdhg_status st = validate(prob, grid, s1, &G);
    if (st != PDHG_OK) return st;
    st = pdhg_workspace_size(prob, grid, s1, handle_bytes);
    if (st != PDHG_OK) return st;
    *total = align256(*handle_bytes) + align256((G.nt + 1) * G.S * G.esz) + align256(G.S * G.esz);
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_gradient_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                                    const pdhg_scheme *scheme, size_t *bytes) {
    if (!bytes) return fail(PDHG_ERR_INVALID_ARG, "bytes is NULL");
    pdhg_scheme s1;
    size_t hb;
    return gradient_inputs(prob, grid, scheme, &s1, &hb, bytes);
}

template <typename T>
static pdhg_status gradient_T(pdhg_handle *h, const double *target, char *ustar, char *tshift, double tol,
                              int64_t max_iters, double adj_tol, int64_t adj_max_iters, int32_t check_every,
                              double *loss, double *du0, double *dnu, int64_t *iters) {
    const Geom &G = h->G;
    const int64_t S = G.S;
    // forward solve
    int64_t done = 0;
    pdhg_status st = pdhg_iterate(h, max_iters, tol, check_every, 0, &done);
    if (iters) iters[0] = done;
    if (st != PDHG_OK) return st;
    // u*, the objective and target - u*^nt
    const size_t ub = (G.nt + 1) * S * sizeof(T);
    CK(cudaMemcpyAsync(ustar, h->ws + h->u_off, ub, cudaMemcpyDeviceToDevice, h->stream));
    std::vector<T> last(S), ts(S);
    CK(cudaMemcpyAsync(last.data(), h->ws + h->u_off + G.nt * S * sizeof(T), S * sizeof(T), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double l2 = 0;
    for (int64_t i = 0; i < S; ++i) {
        if (!std::isfinite(target[i])) return fail(PDHG_ERR_INVALID_ARG, "target has a non-finite value");
        const double d = (double)last[i] - target[i];
        l2 += d * d;
        ts[i] = (T)(target[i] - (double)last[i]);
    }
    if (loss) *loss = h->wx * l2;
    CK(cudaMemcpyAsync(tshift, ts.data(), S * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    // adjoint mode: state v = 0, phi = lambda = 0, initial data 0
    Params<T> &P = params_of<T>(h);
    P.ulin = reinterpret_cast<const T *>(ustar);
    P.tshift = reinterpret_cast<const T *>(tshift);
    graph_drop(h);                                   // the captured launches hold the old parameters
    CK(cudaMemsetAsync(h->ws + h->u_off, 0, ub, h->stream));
    const size_t zero[5] = {h->L.phi, h->L.phit, h->L.lam, h->L.lamt, h->L.u0};
    const size_t zb[5] = {G.nt * S * sizeof(T), G.nt * S * sizeof(T), S * sizeof(T), S * sizeof(T), S * sizeof(T)};
    for (int i = 0; i < 5; ++i) CK(cudaMemsetAsync(h->ws + zero[i], 0, zb[i], h->stream));
    double r[4];
    st = compute_res<T>(h, r);
    if (st != PDHG_OK) return st;
    h->res_init = r[0] > 0 ? r[0] : r[1];
    st = pdhg_iterate(h, adj_max_iters, adj_tol, check_every, 0, &done);
    if (iters) iters[1] = done;
    if (st != PDHG_OK) return st;
    // dLoss/du0 = -w_x lambda;  dLoss/dnu = -h_t w_x sum_l <phi^l, Lap_h u*^{l+1}>
    std::vector<T> lam(S);
    CK(cudaMemcpyAsync(lam.data(), h->ws + h->L.lam, S * sizeof(T), cudaMemcpyDeviceToHost, h->stream));
    double *scal = F<double>(h, h->L.scal) + 8;
    cudaError_t e = launch_phi_lap<T>(P, reinterpret_cast<const T *>(ustar), F<T>(h, h->L.phi),
                                      F<double>(h, h->L.partials), scal, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "phi-Laplacian reduction");
    h->launches += 2;
    double pl = 0;
    CK(cudaMemcpyAsync(&pl, scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (du0)
        for (int64_t i = 0; i < S; ++i) du0[i] = -h->wx * (double)lam[i];
    if (dnu) *dnu = -h->ht * h->wx * pl;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_solve_gradient(const pdhg_problem *prob, const pdhg_grid *grid,
                                           const pdhg_scheme *scheme, const double *target, double tol,
                                           int64_t max_iters, double adj_tol, int64_t adj_max_iters,
                                           int32_t check_every, void *workspace, size_t bytes, void *stream,
                                           double *loss, double *du0, double *dnu, int64_t *iters) {
    pdhg_scheme s1;
    size_t hb, total;
    pdhg_status st = gradient_inputs(prob, grid, scheme, &s1, &hb, &total);
    if (st != PDHG_OK) return st;
    if (!target) return fail(PDHG_ERR_INVALID_ARG, "target is NULL");
    if (!workspace) return fail(PDHG_ERR_INVALID_ARG, "workspace is NULL");
    if (bytes < total) return fail(PDHG_ERR_WORKSPACE_TOO_SMALL, "workspace too small: need " + std::to_string(total));
    if (check_every < 1 || max_iters < 0 || adj_max_iters < 0)
        return fail(PDHG_ERR_INVALID_ARG, "check_every must be >= 1 and iteration bounds >= 0");
    char *ws = (char *)workspace;
    pdhg_handle *h = nullptr;
    st = pdhg_create(prob, grid, &s1, ws, hb, stream, &h);
    if (st != PDHG_OK) return st;
    const size_t ub = align256((grid->nt + 1) * h->G.S * h->G.esz);
    char *ustar = ws + align256(hb), *tshift = ustar + ub;
    st = h->G.prec == PDHG_FP64
             ? gradient_T<double>(h, target, ustar, tshift, tol, max_iters, adj_tol, adj_max_iters, check_every, loss,
                                  du0, dnu, iters)
             : gradient_T<float>(h, target, ustar, tshift, tol, max_iters, adj_tol, adj_max_iters, check_every, loss,
                                 du0, dnu, iters);
    pdhg_destroy(h);
    return st;
}

// ---------------------------------------------------------------------------
// Batches: many independent 1D instances advanced by shared launches (one
// launch per stage for all active instances).  Each instance is an ordinary
// handle (plain path) in its own part of the workspace; the batch adds the
// instance descriptors, the block tables and the reduction buffers.
// ---------------------------------------------------------------------------
enum { TAB_PRIMAL = 0, TAB_ROWS = 1, TAB_TSOLVE = 2, TAB_CHECK = 3, TAB_N = 4 };

struct pdhg_batch {
    int32_t count;
    int32_t prec;
    cudaStream_t stream;
    std::vector<pdhg_handle *> h;
    char *insts;
    BatchEntry *tab[TAB_N];
    int64_t nblk[TAB_N];
    int32_t *list;
    int32_t nlist;
    double *partials, *out;
    std::vector<char> active;
    std::vector<int32_t> order;          // instance ids, most cells first
    size_t smem;
    int64_t launches;
    // persistent launch (one cooperative launch per iteration, work queue)
    bool persistent;
    BatchEntry *queue;                   // device: the work items, stage | items << 2 in pad
    int64_t nqueue;
    int32_t *need;                       // device: items per (instance, stage)
    unsigned int *cnt;                   // device: dequeue counter, then finished items per (instance, stage)
    int *err;                            // device: a bounded wait gave up
    uint64_t wait_ns;
    int32_t blocks_per_sm;               // resident blocks per multiprocessor (0: as many as fit)
    int32_t tiles[8];                    // row items per queue entry, by size class
    int32_t qorder;                      // 0: stage-major queue, 1: instance-major
    int nsm;
    // CUDA graph of check_every iterations and the residual check kernels, replayed while
    // the active set and the launch choice stay the same (dropped by batch_tables)
    bool graphs = true;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    int32_t gchunk = 0;
    int64_t glaunches = 0;
};

static void batch_graph_drop(pdhg_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->gchunk = 0;
}

namespace {

// size class of an instance for the tiles: log2 of its row transform length (the
// Bluestein length, or nx/2 for the packed real FFT) - 8, clamped to [0, 7]
int batch_class(const Geom &G) {
    const int lg = G.blu_log2L ? G.blu_log2L : ilog2(std::max<int64_t>(G.nx / 2, 1));
    return std::min(7, std::max(0, lg - 8));
}

struct BatchLayout {
    size_t insts, tab[TAB_N], list, partials, out, inst0, total;
    size_t queue, need, cnt, err;
    int64_t cap[TAB_N];
    std::vector<size_t> inst_off, inst_bytes;
    std::vector<int64_t> part_off;
    std::vector<Geom> G;
};

// blocks of each table for one instance (grids of the single-instance launchers)
void batch_blocks(const Geom &G, int64_t out[TAB_N], int64_t *gx) {
    const bool dg = G.space >= PDHG_SPACE_DG_P2_LF;
    const int64_t units = dg ? G.nx : G.S;
    const int64_t nlines = dg ? 1 : G.lines;
    const int64_t cols = dg ? G.nkx : G.lines * G.nkx;
    *gx = check_blocks_per_row(units, G.nt);
    out[TAB_PRIMAL] = ((units + 255) / 256) * (G.nt + 1);
    out[TAB_ROWS] = nlines * G.nt;
    out[TAB_TSOLVE] = (cols + 127) / 128;
    out[TAB_CHECK] = *gx * (G.nt + 1);
}

pdhg_status batch_layout(int32_t count, const pdhg_problem *probs, const pdhg_grid *grids, const pdhg_scheme *schemes,
                         BatchLayout *B) {
    if (count < 1 || count > (1 << 20)) return fail(PDHG_ERR_INVALID_ARG, "count must be in [1, 2^20]");
    if (!probs || !grids || !schemes) return fail(PDHG_ERR_INVALID_ARG, "null problem/grid/scheme array");
    B->G.resize(count);
    B->inst_bytes.resize(count);
    B->part_off.resize(count);
    int64_t tabs[TAB_N] = {0, 0, 0, 0}, parts = 0;
    for (int32_t i = 0; i < count; ++i) {
        pdhg_scheme s = schemes[i];
        if (s.path == PDHG_PATH_FUSED) return fail(PDHG_ERR_UNSUPPORTED, "batched instances run on the plain path");
        s.path = PDHG_PATH_PLAIN;
        if (s.precision != schemes[0].precision) return fail(PDHG_ERR_INVALID_ARG, "all instances need one precision");
        pdhg_status st = validate(&probs[i], &grids[i], &s, &B->G[i]);
        if (st != PDHG_OK) return fail(st, "instance " + std::to_string(i) + ": " + g_last_error);
        if (B->G[i].dims != 1) return fail(PDHG_ERR_UNSUPPORTED, "batched instances are 1D");
        B->inst_bytes[i] = layout_of(B->G[i]).total;
        int64_t nb[TAB_N], gx;
        batch_blocks(B->G[i], nb, &gx);
        for (int k = 0; k < TAB_N; ++k) tabs[k] += nb[k];
        B->part_off[i] = parts;
        parts += gx * (B->G[i].nt + 1);
    }
    const size_t isz = schemes[0].precision == PDHG_FP64 ? sizeof(BatchInst<double>) : sizeof(BatchInst<float>);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    B->insts = take(count * isz);
    for (int k = 0; k < TAB_N; ++k) { B->cap[k] = tabs[k]; B->tab[k] = take(tabs[k] * sizeof(BatchEntry)); }
    B->list = take(count * sizeof(int32_t));
    B->partials = take(parts * 6 * sizeof(double));
    B->out = take(count * 6 * sizeof(double));
    // persistent queue: at most one entry per primal block, two per row block (residual
    // and dual), one per 256 t-solve columns (<= the 128-column table's entries)
    B->queue = take((tabs[TAB_PRIMAL] + 2 * tabs[TAB_ROWS] + tabs[TAB_TSOLVE]) * sizeof(BatchEntry));
    B->need = take((size_t)count * 4 * sizeof(int32_t));
    B->cnt = take((1 + (size_t)count * 4) * sizeof(unsigned int));
    B->err = take(sizeof(int));
    B->inst_off.resize(count);
    for (int32_t i = 0; i < count; ++i) B->inst_off[i] = take(B->inst_bytes[i]);
    B->total = o;
    return PDHG_OK;
}

}  // namespace

extern "C" pdhg_status pdhg_batch_workspace_size(int32_t count, const pdhg_problem *probs, const pdhg_grid *grids,
                                                 const pdhg_scheme *schemes, size_t *bytes) {
    if (!bytes) return fail(PDHG_ERR_INVALID_ARG, "bytes is NULL");
    BatchLayout B;
    pdhg_status st = batch_layout(count, probs, grids, schemes, &B);
    if (st != PDHG_OK) return st;
    *bytes = B.total;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_batch_destroy(pdhg_batch *b) {
    if (!b) return PDHG_OK;
    batch_graph_drop(b);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    for (auto *h : b->h) pdhg_destroy(h);
    delete b;
    return PDHG_OK;
}

template <typename T>
static pdhg_status batch_upload_insts(pdhg_batch *b, const BatchLayout &B) {
    std::vector<BatchInst<T>> I(b->count);
    for (int32_t i = 0; i < b->count; ++i) {
        pdhg_handle *h = b->h[i];
        BatchInst<T> &d = I[i];
        d.P = params_of<T>(h);
        d.u = F<T>(h, h->u_off);
        d.phi = F<T>(h, h->L.phi);
        d.phit = F<T>(h, h->L.phit);
        d.lam = F<T>(h, h->L.lam);
        d.lamt = F<T>(h, h->L.lamt);
        d.u0 = F<T>(h, h->L.u0);
        d.spec = h->ws + h->L.spec;
        d.twx = h->ws + h->L.twx;
        d.V = h->ws + h->L.V;
        d.theta = F<T>(h, h->L.theta);
        d.part_off = B.part_off[i];
        int64_t nb[TAB_N], gx;
        batch_blocks(h->G, nb, &gx);
        d.gx = (int32_t)gx;
        const size_t rows = h->G.blu_log2L ? ((size_t)1 << h->G.blu_log2L)
                                           : (size_t)(h->G.space >= PDHG_SPACE_DG_P2_LF ? h->G.lines : 1) * (h->G.nx / 2);
        b->smem = std::max(b->smem, rows * 2 * sizeof(T));
    }
    CK(cudaMemcpyAsync(b->insts, I.data(), I.size() * sizeof(BatchInst<T>), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return PDHG_OK;
}

// tables of the active instances, most cells first
static pdhg_status batch_tables(pdhg_batch *b) {
    batch_graph_drop(b);                         // its launches have the old grids baked in
    std::vector<BatchEntry> t[TAB_N];
    std::vector<int32_t> list;
    for (int32_t i : b->order) {
        if (!b->active[i]) continue;
        const Geom &G = b->h[i]->G;
        int64_t nb[TAB_N], gx;
        batch_blocks(G, nb, &gx);
        const int64_t gxp = nb[TAB_PRIMAL] / (G.nt + 1), nlines = nb[TAB_ROWS] / G.nt;
        // primal entries cover BATCH_PRIMAL_SPAN slices each (pad = the count): a block of 256
        // dofs of one slice is too little work for its launch and setup
        for (int64_t l = 0; l <= G.nt; l += BATCH_PRIMAL_SPAN)
            for (int64_t x = 0; x < gxp; ++x)
                t[TAB_PRIMAL].push_back({i, (int32_t)x, (int32_t)l,
                                         (int32_t)std::min<int64_t>(BATCH_PRIMAL_SPAN, G.nt + 1 - l)});
        // Bluestein rows: the block of an even slice transforms that slice and the next
        // together, so odd slices get no block
        const int64_t lstep = G.blu_log2L ? 2 : 1;
        for (int64_t l = 0; l < G.nt; l += lstep)
            for (int64_t x = 0; x < nlines; ++x) t[TAB_ROWS].push_back({i, (int32_t)x, (int32_t)l, 0});
        for (int64_t x = 0; x < nb[TAB_TSOLVE]; ++x) t[TAB_TSOLVE].push_back({i, (int32_t)x, 0, 0});
        for (int64_t l = 0; l <= G.nt; ++l)
            for (int64_t x = 0; x < gx; ++x) t[TAB_CHECK].push_back({i, (int32_t)x, (int32_t)l, 0});
        list.push_back(i);
    }
    // persistent queue: stage after stage (order 0: instances most cells first within a
    // stage) or instance after instance (order 1: each instance's four stages in turn, so
    // that the stages of different instances overlap); an entry covers `tiles[class]` row
    // items (primal slices, row blocks) or one block of 256 t-solve columns
    std::vector<BatchEntry> q;
    std::vector<int32_t> need((size_t)b->count * 4, 0);
    std::vector<std::pair<int, int32_t>> seq;            // (stage, instance) in queue order
    for (int stage = 0; stage < 4; ++stage)
        for (int32_t i : b->order) seq.push_back({stage, i});
    if (b->qorder == 1)
        std::stable_sort(seq.begin(), seq.end(), [&](const std::pair<int, int32_t> &x, const std::pair<int, int32_t> &y) {
            const auto px = std::find(b->order.begin(), b->order.end(), x.second) - b->order.begin();
            const auto py = std::find(b->order.begin(), b->order.end(), y.second) - b->order.begin();
            return px < py;
        });
    for (const auto &si : seq) {
        {
            const int stage = si.first;
            const int32_t i = si.second;
            if (!b->active[i]) continue;
            const Geom &G = b->h[i]->G;
            int64_t nb[TAB_N], gx;
            batch_blocks(G, nb, &gx);
            const int64_t g = std::max(1, b->tiles[batch_class(G)]);
            if (stage == 0) {
                const int64_t gxp = nb[TAB_PRIMAL] / (G.nt + 1);
                for (int64_t l = 0; l <= G.nt; l += g)
                    for (int64_t x = 0; x < gxp; ++x)
                        q.push_back({i, (int32_t)x, (int32_t)l, (int32_t)(std::min(g, G.nt + 1 - l) << 2)});
            } else if (stage == 2) {
                const bool dg = G.space >= PDHG_SPACE_DG_P2_LF;
                const int64_t cols = dg ? G.nkx : G.lines * G.nkx;
                for (int64_t x = 0; x < (cols + 255) / 256; ++x) q.push_back({i, (int32_t)x, 0, (int32_t)(2 | (1 << 2))});
            } else {
                const int64_t lstep = G.blu_log2L ? 2 : 1, nlines = nb[TAB_ROWS] / G.nt;
                const int64_t rows = (G.nt + lstep - 1) / lstep;          // row items per line
                for (int64_t r = 0; r < rows; r += g)
                    for (int64_t x = 0; x < nlines; ++x)
                        q.push_back({i, (int32_t)x, (int32_t)(r * lstep), (int32_t)(stage | (std::min(g, rows - r) << 2))});
            }
        }
    }
    for (const BatchEntry &e : q) ++need[(size_t)e.inst * 4 + (e.pad & 3)];
    b->nqueue = (int64_t)q.size();
    if (!q.empty())
        CK(cudaMemcpyAsync(b->queue, q.data(), q.size() * sizeof(BatchEntry), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->need, need.data(), need.size() * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream));
    for (int k = 0; k < TAB_N; ++k) {
        b->nblk[k] = (int64_t)t[k].size();
        if (!t[k].empty())
            CK(cudaMemcpyAsync(b->tab[k], t[k].data(), t[k].size() * sizeof(BatchEntry), cudaMemcpyHostToDevice,
                               b->stream));
    }
    b->nlist = (int32_t)list.size();
    if (!list.empty())
        CK(cudaMemcpyAsync(b->list, list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));        // the host vectors go out of scope
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_batch_create(int32_t count, const pdhg_problem *probs, const pdhg_grid *grids,
                                         const pdhg_scheme *schemes, void *workspace, size_t bytes, void *stream,
                                         pdhg_batch **out) {
    if (!out) return fail(PDHG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    BatchLayout B;
    pdhg_status st = batch_layout(count, probs, grids, schemes, &B);
    if (st != PDHG_OK) return st;
    if (!workspace) return fail(PDHG_ERR_INVALID_ARG, "workspace is NULL");
    if (((uintptr_t)workspace & 255) != 0) return fail(PDHG_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (bytes < B.total) return fail(PDHG_ERR_WORKSPACE_TOO_SMALL, "workspace too small: need " + std::to_string(B.total));
    char *ws = (char *)workspace;
    pdhg_batch *b = new pdhg_batch();
    b->count = count;
    b->prec = schemes[0].precision;
    b->stream = (cudaStream_t)stream;
    b->insts = ws + B.insts;
    for (int k = 0; k < TAB_N; ++k) { b->tab[k] = (BatchEntry *)(ws + B.tab[k]); b->nblk[k] = 0; }
    b->list = (int32_t *)(ws + B.list);
    b->partials = (double *)(ws + B.partials);
    b->out = (double *)(ws + B.out);
    b->smem = 0;
    b->launches = 0;
    b->active.assign(count, 1);
    b->persistent = false;
    b->qorder = 0;
    b->queue = (BatchEntry *)(ws + B.queue);
    b->nqueue = 0;
    b->need = (int32_t *)(ws + B.need);
    b->cnt = (unsigned int *)(ws + B.cnt);
    b->err = (int *)(ws + B.err);
    b->wait_ns = 1000000000ull;
    b->blocks_per_sm = 0;
    for (int k = 0; k < 8; ++k) b->tiles[k] = 1;
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "batch create"); }
    }
    for (int32_t i = 0; i < count; ++i) {
        pdhg_scheme s = schemes[i];
        s.path = PDHG_PATH_PLAIN;
        pdhg_handle *h = nullptr;
        st = pdhg_create(&probs[i], &grids[i], &s, ws + B.inst_off[i], B.inst_bytes[i], stream, &h);
        if (st != PDHG_OK) { pdhg_batch_destroy(b); return fail(st, "instance " + std::to_string(i) + ": " + g_last_error); }
        b->h.push_back(h);
    }
    b->order.resize(count);
    for (int32_t i = 0; i < count; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int32_t x, int32_t y) {
        return B.G[x].S * (B.G[x].nt + 1) > B.G[y].S * (B.G[y].nt + 1);
    });
    st = b->prec == PDHG_FP64 ? batch_upload_insts<double>(b, B) : batch_upload_insts<float>(b, B);
    if (st == PDHG_OK) st = batch_tables(b);
    if (st != PDHG_OK) { pdhg_batch_destroy(b); return st; }
    *out = b;
    return PDHG_OK;
}

template <typename T>
static cudaError_t batch_iteration(pdhg_batch *b) {
    const BatchInst<T> *I = (const BatchInst<T> *)b->insts;
    if (b->persistent) {
        int per_sm = 0;
        cudaError_t e = batch_persistent_occupancy<T>(b->smem, &per_sm);
        if (e != cudaSuccess) return e;
        if (b->blocks_per_sm > 0) per_sm = std::min(per_sm, (int)b->blocks_per_sm);
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        e = cudaMemsetAsync(b->cnt, 0, (1 + (size_t)b->count * 4) * sizeof(unsigned int), b->stream);
        if (e == cudaSuccess)
            e = launch_batch_persistent<T>(I, b->queue, b->nqueue, b->need, b->cnt, b->err, b->wait_ns,
                                           per_sm * b->nsm, b->smem, b->stream);
        b->launches += 1;
        return e;
    }
    cudaError_t e = launch_batch<T>(BATCH_PRIMAL, I, b->tab[TAB_PRIMAL], b->nblk[TAB_PRIMAL], 0, nullptr, nullptr,
                                    nullptr, b->stream);
    if (e == cudaSuccess)
        e = launch_batch<T>(BATCH_RESIDUAL, I, b->tab[TAB_ROWS], b->nblk[TAB_ROWS], b->smem, nullptr, nullptr, nullptr,
                            b->stream);
    if (e == cudaSuccess)
        e = launch_batch<T>(BATCH_TSOLVE, I, b->tab[TAB_TSOLVE], b->nblk[TAB_TSOLVE], 0, nullptr, nullptr, nullptr,
                            b->stream);
    if (e == cudaSuccess)
        e = launch_batch<T>(BATCH_DUAL, I, b->tab[TAB_ROWS], b->nblk[TAB_ROWS], b->smem, nullptr, nullptr, nullptr,
                            b->stream);
    b->launches += 4;
    return e;
}

template <typename T>
static cudaError_t batch_check_launch(pdhg_batch *b) {
    const BatchInst<T> *I = (const BatchInst<T> *)b->insts;
    cudaError_t e = launch_batch<T>(BATCH_CHECK, I, b->tab[TAB_CHECK], b->nblk[TAB_CHECK], 0, nullptr, b->partials,
                                    nullptr, b->stream);
    if (e == cudaSuccess)
        e = launch_batch<T>(BATCH_REDUCE, I, nullptr, b->nlist, 0, b->list, b->partials, b->out, b->stream);
    b->launches += 2;
    return e;
}

// the six sums of every instance and the wait flag, after the check kernels
static pdhg_status batch_read(pdhg_batch *b, std::vector<double> &acc) {
    acc.resize((size_t)b->count * 6);
    int err = 0;
    CK(cudaMemcpyAsync(acc.data(), b->out, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (err) {
        CK(cudaMemset(b->err, 0, sizeof(int)));
        return fail(PDHG_ERR_TIMEOUT, "a bounded wait of the persistent batch iteration gave up (the batch state is invalid)");
    }
#ifdef PDHG_DEBUG
    // debug builds: the first out-of-range site recorded by any instance's kernels
    for (int32_t i = 0; i < b->count; ++i) CK(canary_check(b->h[i], b->stream));
    CK(cudaStreamSynchronize(b->stream));
    for (int32_t i = 0; i < b->count; ++i) {
        int bad = 0;
        CK(cudaMemcpy(&bad, b->h[i]->ws + b->h[i]->L.dbg, sizeof(int), cudaMemcpyDeviceToHost));
        if (bad) return fail(PDHG_ERR_BOUNDS, "instance " + std::to_string(i) + ": " + debug_site_message(bad));
    }
#endif
    return PDHG_OK;
}

template <typename T>
static pdhg_status batch_check(pdhg_batch *b, std::vector<double> &acc) {
    cudaError_t e = batch_check_launch<T>(b);
    if (e != cudaSuccess) return cuda_fail(e, "batched residual check");
    return batch_read(b, acc);
}

// capture m iterations and the check kernels on a side stream (the same launches as
// batch_iteration / batch_check_launch, so replays compute what they would)
template <typename T>
static cudaError_t batch_graph_build(pdhg_batch *b, int32_t m) {
    batch_graph_drop(b);
    cudaError_t e = cudaSuccess;
    if (!b->gstream) e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaStream_t user = b->stream;
    const int64_t l0 = b->launches;
    b->stream = b->gstream;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int32_t i = 0; i < m && e == cudaSuccess; ++i) e = batch_iteration<T>(b);
        if (e == cudaSuccess) e = batch_check_launch<T>(b);
        cudaError_t e2 = cudaStreamEndCapture(b->gstream, &g);
        if (e == cudaSuccess) e = e2;
    }
    b->stream = user;
    b->glaunches = b->launches - l0;
    b->launches = l0;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e == cudaSuccess) b->gchunk = m;
    else batch_graph_drop(b);
    return e;
}

// Res of one instance from its six sums (as read_res)
static void res_from_sums(const pdhg_handle *h, const double *acc, double out[4]) {
    const double ht = h->ht, wx = h->wx;
    const double we = h->res_norm == 1 ? wx : ht * wx;
    double a2 = we * acc[0], b2 = we * acc[1], gap = we * acc[2], c2 = wx * acc[3];
    if (h->G.init == PDHG_INIT_LAMBDA) {
        a2 += c2;
        b2 += wx * acc[4];
        gap += wx * acc[5];
    }
    out[0] = std::sqrt(a2); out[1] = std::sqrt(b2); out[2] = std::sqrt(c2); out[3] = gap;
}

template <typename T>
static pdhg_status batch_iterate_T(pdhg_batch *b, int64_t max_iters, double tol, int32_t check_every, int32_t relative,
                                   int64_t *iters, int32_t *state) {
    std::vector<int64_t> it(b->count, 0);
    std::vector<int32_t> stt(b->count, 0);
    for (int32_t i = 0; i < b->count; ++i)
        if (!b->active[i]) stt[i] = 1;
    std::vector<double> acc;
    pdhg_status st = PDHG_OK;
    for (int64_t n = 0; n < max_iters && b->nlist > 0;) {
        // whole chunks of check_every iterations run as one graph replay (iterations and
        // check kernels); the tail and graph-less runs launch kernel by kernel
        const bool chunk = b->graphs && check_every > 0 && n % check_every == 0 && max_iters - n >= check_every;
        if (chunk && b->gchunk != check_every && batch_graph_build<T>(b, check_every) != cudaSuccess) {
            cudaGetLastError();                          // capture refused: launch kernel by kernel
            b->graphs = false;
        }
        bool checked = false;
        if (chunk && b->gchunk == check_every) {
            cudaError_t e = cudaGraphLaunch(b->gexec, b->stream);
            if (e != cudaSuccess) { st = cuda_fail(e, "batch graph launch"); break; }
            n += check_every;
            b->launches += b->glaunches;
            for (int32_t i = 0; i < b->count; ++i)
                if (b->active[i]) { it[i] += check_every; b->h[i]->iters += check_every; }
            st = batch_read(b, acc);
            if (st != PDHG_OK) break;
            checked = true;
        } else {
            cudaError_t e = batch_iteration<T>(b);
            if (e != cudaSuccess) { st = cuda_fail(e, "batched iteration"); break; }
            ++n;
            for (int32_t i = 0; i < b->count; ++i)
                if (b->active[i]) { ++it[i]; ++b->h[i]->iters; }
            if (check_every > 0 && (n % check_every == 0 || n == max_iters)) {
                st = batch_check<T>(b, acc);
                if (st != PDHG_OK) break;
                checked = true;
            }
        }
        if (checked) {
            bool changed = false;
            for (int32_t i = 0; i < b->count; ++i) {
                if (!b->active[i]) continue;
                double r[4];
                res_from_sums(b->h[i], &acc[(size_t)i * 6], r);
                history_push(b->h[i], r);
                const double scale = relative ? b->h[i]->res_init : 1.0;
                if (!std::isfinite(r[0]) || !std::isfinite(r[1]) ||
                    r[0] > 1e10 * std::max(b->h[i]->res_init, 1e-300)) {
                    stt[i] = -1; b->active[i] = 0; changed = true;
                } else if (r[0] <= tol * scale && r[1] <= tol * scale) {
                    stt[i] = 1; b->active[i] = 0; changed = true;
                }
            }
            if (changed) {
                st = batch_tables(b);
                if (st != PDHG_OK) break;
            }
        }
    }
    if (iters) std::copy(it.begin(), it.end(), iters);
    if (state) std::copy(stt.begin(), stt.end(), state);
    return st;
}

extern "C" pdhg_status pdhg_batch_iterate(pdhg_batch *b, int64_t max_iters, double tol, int32_t check_every,
                                          int32_t relative, int64_t *iters, int32_t *state) {
    if (!b) return fail(PDHG_ERR_INVALID_ARG, "null batch");
    if (max_iters < 0) return fail(PDHG_ERR_INVALID_ARG, "max_iters < 0");
    return b->prec == PDHG_FP64 ? batch_iterate_T<double>(b, max_iters, tol, check_every, relative, iters, state)
                                : batch_iterate_T<float>(b, max_iters, tol, check_every, relative, iters, state);
}

extern "C" pdhg_status pdhg_batch_reset(pdhg_batch *b) {
    if (!b) return fail(PDHG_ERR_INVALID_ARG, "null batch");
    b->active.assign(b->count, 1);
    return batch_tables(b);
}

extern "C" pdhg_status pdhg_batch_instance(pdhg_batch *b, int32_t i, pdhg_handle **h) {
    if (!b || !h) return fail(PDHG_ERR_INVALID_ARG, "null batch or out");
    if (i < 0 || i >= b->count) return fail(PDHG_ERR_INVALID_ARG, "instance index out of range");
    *h = b->h[i];
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_batch_launch_count(pdhg_batch *b, int64_t *launches, int32_t reset) {
    if (!b || !launches) return fail(PDHG_ERR_INVALID_ARG, "null batch or out");
    *launches = b->launches;
    if (reset) b->launches = 0;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_batch_set_launch(pdhg_batch *b, int32_t persistent, int32_t blocks_per_sm,
                                             int32_t order, const int32_t *tiles) {
    if (!b) return fail(PDHG_ERR_INVALID_ARG, "null batch");
    if (blocks_per_sm < 0) return fail(PDHG_ERR_INVALID_ARG, "blocks_per_sm must be >= 0");
    if (order != 0 && order != 1) return fail(PDHG_ERR_INVALID_ARG, "order must be 0 or 1");
    b->qorder = order;
    if (tiles)
        for (int k = 0; k < 8; ++k)
            if (tiles[k] < 1 || tiles[k] > 64) return fail(PDHG_ERR_INVALID_ARG, "tiles must be in [1, 64]");
    b->persistent = persistent != 0;
    b->blocks_per_sm = blocks_per_sm;
    if (tiles) std::copy(tiles, tiles + 8, b->tiles);
    return batch_tables(b);
}

extern "C" pdhg_status pdhg_batch_set_wait_budget(pdhg_batch *b, uint64_t ns) {
    if (!b) return fail(PDHG_ERR_INVALID_ARG, "null batch");
    batch_graph_drop(b);                         // the budget is a kernel argument
    b->wait_ns = ns;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_batch_set_graphs(pdhg_batch *b, int32_t enable) {
    if (!b) return fail(PDHG_ERR_INVALID_ARG, "null batch");
    batch_graph_drop(b);
    b->graphs = enable != 0;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_set_graphs(pdhg_handle *h, int32_t enable) {
    if (!h) return fail(PDHG_ERR_INVALID_ARG, "null handle");
    graph_drop(h);
    h->graphs = enable != 0;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_set_wait_budget(pdhg_handle *h, uint64_t ns) {
    if (!h) return fail(PDHG_ERR_INVALID_ARG, "null handle");
    if (h->G.fused) {
        h->fused.wait_ns = ns;
        graph_drop(h);                   // a captured rows-C launch holds the old budget
    }
    return PDHG_OK;
}

// ---------------------------------------------------------------------------
// Mixed-precision solve: Algorithm 1 in float32 (the fused path where it applies)
// until Res reaches tol or stops falling (float32 rounding floor), then the state
// widened to float64 and the iteration finished on the float64 plain path.  The
// workspace holds the float32 handle's region, then the float64 one's.
// ---------------------------------------------------------------------------
static pdhg_status mixed_schemes(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                                 pdhg_scheme *s32, pdhg_scheme *s64, size_t *b32, size_t *b64) {
    if (!scheme) return fail(PDHG_ERR_INVALID_ARG, "null scheme");
    *s32 = *scheme;
    s32->precision = PDHG_FP32;
    *s64 = *scheme;
    s64->precision = PDHG_FP64;
    s64->path = PDHG_PATH_PLAIN;
    pdhg_status st = pdhg_workspace_size(prob, grid, s32, b32);
    if (st != PDHG_OK) return st;
    Geom G;
    st = validate(prob, grid, s64, &G, true);
    if (st == PDHG_OK) *b64 = layout_of(G).total;
    return st;
}

extern "C" pdhg_status pdhg_mixed_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                                 const pdhg_scheme *scheme, size_t *bytes) {
    if (!bytes) return fail(PDHG_ERR_INVALID_ARG, "bytes is NULL");
    pdhg_scheme s32, s64;
    size_t b32, b64;
    pdhg_status st = mixed_schemes(prob, grid, scheme, &s32, &s64, &b32, &b64);
    if (st != PDHG_OK) return st;
    *bytes = align256(b32) + b64;
    return PDHG_OK;
}

extern "C" pdhg_status pdhg_solve_mixed(const pdhg_problem *prob, const pdhg_grid *grid, const pdhg_scheme *scheme,
                                        double tol, int32_t relative, int32_t check_every, int64_t max_iters,
                                        void *workspace, size_t bytes, void *stream, pdhg_handle **out,
                                        int64_t iters[2]) {
    if (!out) return fail(PDHG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (iters) iters[0] = iters[1] = 0;
    pdhg_scheme s32, s64;
    size_t b32, b64;
    pdhg_status st = mixed_schemes(prob, grid, scheme, &s32, &s64, &b32, &b64);
    if (st != PDHG_OK) return st;
    if (!workspace) return fail(PDHG_ERR_INVALID_ARG, "workspace is NULL");
    if (bytes < align256(b32) + b64)
        return fail(PDHG_ERR_WORKSPACE_TOO_SMALL, "workspace too small: need " + std::to_string(align256(b32) + b64));
    if (check_every < 1 || max_iters < 0 || !(tol >= 0))
        return fail(PDHG_ERR_INVALID_ARG, "check_every must be >= 1, max_iters >= 0 and tol >= 0");
    char *ws = (char *)workspace;
    pdhg_handle *h32 = nullptr, *h64 = nullptr;
    st = pdhg_create(prob, grid, &s32, ws, b32, stream, &h32);
    if (st != PDHG_OK) return st;
    // float32 phase: chunks of check_every iterations; stop at tol, or when the worse
    // entry of Res has not fallen by 5% over the last three checks (the float32 floor)
    const double scale = relative ? h32->res_init : 1.0;
    std::vector<double> hist;
    int64_t n32 = 0;
    while (n32 < max_iters) {
        int64_t done = 0;
        st = pdhg_iterate(h32, std::min<int64_t>(check_every, max_iters - n32), tol, check_every, relative, &done);
        n32 += done;
        if (st != PDHG_OK) break;
        const double r = std::max(h32->last_res[0], h32->last_res[1]);
        if (h32->last_res[0] <= tol * scale && h32->last_res[1] <= tol * scale) break;
        hist.push_back(r);
        if (hist.size() >= 4 && hist.back() > 0.95 * hist[hist.size() - 4]) break;
    }
    if (iters) iters[0] = n32;
    if (st != PDHG_OK) { pdhg_destroy(h32); return st; }
    // float64 phase from the widened state
    st = create_impl(prob, grid, &s64, ws + align256(b32), b64, stream, &h64, true);
    if (st != PDHG_OK) { pdhg_destroy(h32); return st; }
    const Geom &G = h32->G;
    const int64_t S = G.S;
    struct { size_t src, dst; int64_t n; } parts[5] = {
        {h32->u_off, h64->u_off, (G.nt + 1) * S}, {h32->L.phi, h64->L.phi, G.nt * S},
        {h32->L.phit, h64->L.phit, G.nt * S}, {h32->L.lam, h64->L.lam, S}, {h32->L.lamt, h64->L.lamt, S}};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 5 && e == cudaSuccess; ++i)
        e = launch_widen((const float *)(h32->ws + parts[i].src), (double *)(h64->ws + parts[i].dst), parts[i].n,
                         h64->stream);
    h64->launches += 5;
    pdhg_destroy(h32);
    if (e != cudaSuccess) { pdhg_destroy(h64); return cuda_fail(e, "float32 -> float64 hand-over"); }
    // from the float32 state the float64 phase is short (1 to a few tens of iterations on
    // the workloads measured): check after 1, 2, 3, 4, 6, 9, 13, ... iterations (chunks of
    // half the iterations done, at most check_every / 5), so a phase of n iterations costs
    // at most about 1.5 n iterations and O(log n) checks
    int64_t n64 = 0;
    const int64_t cap = std::max<int32_t>(1, check_every / 5);
    h64->graphs = false;                 // chunks of changing length: launch kernel by kernel
    while (n64 < max_iters - n32) {
        const int64_t chunk = std::min<int64_t>(std::min<int64_t>(std::max<int64_t>(1, n64 / 2), cap),
                                                max_iters - n32 - n64);
        int64_t done = 0;
        st = pdhg_iterate(h64, chunk, tol, (int32_t)chunk, relative, &done);
        n64 += done;
        if (st != PDHG_OK) break;
        const double sc = relative ? h64->res_init : 1.0;
        if (h64->last_res[0] <= tol * sc && h64->last_res[1] <= tol * sc) break;
    }
    if (iters) iters[1] = n64;
    if (st != PDHG_OK) { pdhg_destroy(h64); return st; }
    *out = h64;
    return PDHG_OK;
}

"""Spatial operators of the implicit schemes (oracle, float64, numpy).

Every operator acts on a batch of slices: the spatial axes are the trailing
ones ((nx,) for 1D FD, (ny, nx) for 2D FD, (3, ncell) for DG P2) and any
leading axes are batch axes.  ``D(v)`` is the spatial part of the equation
u_t + D(u) = 0, i.e. D(u) ~ f(u)_x - (gamma u_x)_x  (Eq. 2.1).

For each scheme there are three functions:

* ``D(p, v)``               -- the operator,
* ``D_jvp(p, v, w)``        -- D'(v) w,
* ``D_vjp(p, v, psi)``      -- D'(v)^T psi  (by transposing D_jvp term by term).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def flux(p, v):
    """f(u) = alpha u^2 + beta u (Sec. 3.2.3; linear transport has alpha = 0)."""
    return p.alpha * v * v + p.beta * v


def dflux(p, v):
    """f'(u) = 2 alpha u + beta."""
    return 2.0 * p.alpha * v + p.beta


# ---------------------------------------------------------------------------
# finite differences (Sec. 3.2.1, 3.2.2)
# ---------------------------------------------------------------------------

def _fd_axes(p):
    """(axis, h) pairs of the spatial directions, x last."""
    if p.dims == 2:
        return [(-1, p.hx), (-2, p.hy)]
    return [(-1, p.hx)]


def _num_flux(p, v, axis):
    """Interface flux F_{j+1/2} along ``axis``.

    fd_upwind: F_{j+1/2} = f(v_j)  (monotone upwind flux for f' >= 0, Sec. 3.2.2).
    fd_lf:     F_{j+1/2} = (f(v_j)+f(v_{j+1}))/2 - a/2 (v_{j+1}-v_j)  (global
               Lax-Friedrichs with a fixed constant a).
    """
    if p.space == "fd_upwind":
        return flux(p, v)
    vp = np.roll(v, -1, axis=axis)
    return 0.5 * (flux(p, v) + flux(p, vp)) - 0.5 * p.lf_a * (vp - v)


def _num_flux_jvp(p, v, w, axis):
    """Directional derivative of F_{j+1/2} along w."""
    if p.space == "fd_upwind":
        return dflux(p, v) * w
    vp = np.roll(v, -1, axis=axis)
    wp = np.roll(w, -1, axis=axis)
    return 0.5 * (dflux(p, v) * w + dflux(p, vp) * wp) - 0.5 * p.lf_a * (wp - w)


def _num_flux_vjp(p, v, g, axis):
    """Transpose of _num_flux_jvp: returns q_k = sum_j g_j dF_{j+1/2}/dv_k."""
    if p.space == "fd_upwind":
        return dflux(p, v) * g
    gm = np.roll(g, 1, axis=axis)                       # g_{k-1}
    # F_{k+1/2} holds v_k with weight (f'(v_k) + a)/2, F_{k-1/2} with (f'(v_k) - a)/2
    return 0.5 * (dflux(p, v) + p.lf_a) * g + 0.5 * (dflux(p, v) - p.lf_a) * gm


def _viscous(p, v):
    """-(gamma u_x)_x discretised by the central difference Lap of Sec. 3.2.1.

    Constant nu: -nu (v_{j+1} - 2 v_j + v_{j-1}) / h^2 along every axis.
    gamma_half (1D): -[gamma_{j+1/2}(v_{j+1}-v_j) - gamma_{j-1/2}(v_j-v_{j-1})]/h^2.
    The operator is linear and symmetric, so it is its own Jacobian transpose.
    """
    out = np.zeros_like(v)
    if p.gamma_half is not None:
        h = p.hx
        G = p.gamma_half * (np.roll(v, -1, axis=-1) - v) / h      # G_{j+1/2}
        out -= (G - np.roll(G, 1, axis=-1)) / h
    if p.nu != 0.0:
        for axis, h in _fd_axes(p):
            out -= p.nu * (np.roll(v, -1, axis=axis) - 2.0 * v + np.roll(v, 1, axis=axis)) / (h * h)
    return out


def fd_D(p, v):
    """D(v)_j = sum over directions of (F_{j+1/2} - F_{j-1/2})/h, plus the viscous term."""
    out = _viscous(p, v)
    for axis, h in _fd_axes(p):
        F = _num_flux(p, v, axis)
        out = out + (F - np.roll(F, 1, axis=axis)) / h
    return out


def fd_D_jvp(p, v, w):
    out = _viscous(p, w)
    for axis, h in _fd_axes(p):
        dF = _num_flux_jvp(p, v, w, axis)
        out = out + (dF - np.roll(dF, 1, axis=axis)) / h
    return out


def fd_D_vjp(p, v, psi):
    """D'(v)^T psi.  sum_j psi_j (F_{j+1/2} - F_{j-1/2})/h = sum_j F_{j+1/2} g_j with
    g_j = (psi_j - psi_{j+1})/h; then each F_{j+1/2} is transposed."""
    out = _viscous(p, psi)
    for axis, h in _fd_axes(p):
        g = (psi - np.roll(psi, -1, axis=axis)) / h
        out = out + _num_flux_vjp(p, v, g, axis)
    return out


# ---------------------------------------------------------------------------
# DG P2, modal Legendre basis, global Lax-Friedrichs interface flux
# (the DG weak form of Sec. 3.2.2 with P^2 elements; the residual is written
#  with the inverse mass matrix applied, as in Eq. 3.5)
# ---------------------------------------------------------------------------

GAUSS_X = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
GAUSS_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])
LEG = np.stack([np.ones(3), GAUSS_X, 0.5 * (3.0 * GAUSS_X ** 2 - 1.0)])   # P_m(xi_q)  [m][q]
DLEG = np.stack([np.zeros(3), np.ones(3), 3.0 * GAUSS_X])                 # P_m'(xi_q) [m][q]
LEFT = np.array([1.0, -1.0, 1.0])                                          # P_m(-1); P_m(1) = 1


def _dg_scale(p):
    """(2m+1)/h: the inverse of the Legendre mass matrix diag(h/(2m+1))."""
    return (2.0 * np.arange(3) + 1.0) / p.hx


def dg_D(p, U):
    """D(U)_{j,m} = -(2m+1)/h [ int_{-1}^{1} f(u_h) P_m' dxi - Fh_{j+1/2} + (-1)^m Fh_{j-1/2} ].

    u_h = sum_m U_{j,m} P_m(xi) on cell j; the volume integral uses 3-point Gauss
    (exact for quadratic f on P2); Fh_{j+1/2} = (f(uR_j)+f(uL_{j+1}))/2 - a/2 (uL_{j+1}-uR_j)
    with uR_j = u_h(x_{j+1/2}^-) and uL_{j+1} = u_h(x_{j+1/2}^+)."""
    uq = np.einsum("mq,...mj->...qj", LEG, U)
    vol = np.einsum("q,mq,...qj->...mj", GAUSS_W, DLEG, flux(p, uq))
    uR = U.sum(axis=-2)
    uLn = np.roll(np.einsum("m,...mj->...j", LEFT, U), -1, axis=-1)
    Fh = 0.5 * (flux(p, uR) + flux(p, uLn)) - 0.5 * p.lf_a * (uLn - uR)
    Fm = np.roll(Fh, 1, axis=-1)
    s = _dg_scale(p)[:, None]
    return -s * (vol - Fh[..., None, :] + LEFT[:, None] * Fm[..., None, :])


def dg_D_jvp(p, U, V):
    uq = np.einsum("mq,...mj->...qj", LEG, U)
    vq = np.einsum("mq,...mj->...qj", LEG, V)
    vol = np.einsum("q,mq,...qj->...mj", GAUSS_W, DLEG, dflux(p, uq) * vq)
    uR = U.sum(axis=-2)
    vR = V.sum(axis=-2)
    uLn = np.roll(np.einsum("m,...mj->...j", LEFT, U), -1, axis=-1)
    vLn = np.roll(np.einsum("m,...mj->...j", LEFT, V), -1, axis=-1)
    dFh = 0.5 * (dflux(p, uR) * vR + dflux(p, uLn) * vLn) - 0.5 * p.lf_a * (vLn - vR)
    dFm = np.roll(dFh, 1, axis=-1)
    s = _dg_scale(p)[:, None]
    return -s * (vol - dFh[..., None, :] + LEFT[:, None] * dFm[..., None, :])


def dg_D_vjp(p, U, Psi):
    """D'(U)^T Psi, transposing dg_D_jvp term by term.

    With S_m = (2m+1)/h Psi_m:
      volume:  -sum_q P_n(xi_q) f'(u_q) w_q sum_m P_m'(xi_q) S_m           (cell-local)
      fluxes:  sum_j dFh_{j+1/2} G_j with G_j = sum_m S_{m,j} - sum_m (-1)^m S_{m,j+1};
               dFh_{j+1/2} = (f'(uR_j)+a)/2 dvR_j + (f'(uL_{j+1})-a)/2 dvL_{j+1}.
    """
    s = _dg_scale(p)[:, None]
    S = s * Psi
    uq = np.einsum("mq,...mj->...qj", LEG, U)
    inner = np.einsum("q,mq,...mj->...qj", GAUSS_W, DLEG, S)          # w_q sum_m P_m' S_m
    out = -np.einsum("nq,...qj->...nj", LEG, dflux(p, uq) * inner)
    uR = U.sum(axis=-2)
    uLn = np.roll(np.einsum("m,...mj->...j", LEFT, U), -1, axis=-1)
    G = S.sum(axis=-2) - np.roll(np.einsum("m,...mj->...j", LEFT, S), -1, axis=-1)
    dA = 0.5 * (dflux(p, uR) + p.lf_a)           # dFh_{j+1/2}/duR_j
    dB = 0.5 * (dflux(p, uLn) - p.lf_a)          # dFh_{j+1/2}/duL_{j+1}
    out = out + (G * dA)[..., None, :] + LEFT[:, None] * np.roll(G * dB, 1, axis=-1)[..., None, :]
    return out


# ---------------------------------------------------------------------------
# DG P1 with the nodal basis of Sec. 3.2.2: phi_1(xi) = 1/2 - xi, phi_2(xi) = 1/2 + xi
# (nodes x_{j-1/4}, x_{j+1/4}); mass matrix (h/12)[[7,-1],[-1,7]]; upwind flux
# Fh(u-, u+) = f(u-) (the paper's choice for f' >= 0) or global Lax-Friedrichs.
#   E_m = int f(u_h) phi_m' dxi - Fh_{j+1/2} phi_m(1) + Fh_{j-1/2} phi_m(-1),
#   dU_j/dt = M^{-1} E (Eq. 3.5 / Eq. 3.8 form), D = -M^{-1} E.
# The volume integral V = int f(u_h) dxi uses 2-point Gauss (exact for quadratic f).
# ---------------------------------------------------------------------------

G2 = 1.0 / np.sqrt(3.0)
P1_Q = np.array([[0.5 + G2, 0.5 - G2], [0.5 - G2, 0.5 + G2]])   # phi_m(xi_q) [m][q], xi = -G2, +G2
P1_RIGHT = np.array([-0.5, 1.5])                                 # phi_m(1)
P1_LEFT = np.array([1.5, -0.5])                                  # phi_m(-1)
P1_MINV = np.array([[7.0, 1.0], [1.0, 7.0]]) / 4.0               # h * M^{-1}


def _p1_face(p, a, b):
    if p.space == "dg_p1_upwind":
        return flux(p, a)
    return 0.5 * (flux(p, a) + flux(p, b)) - 0.5 * p.lf_a * (b - a)


def _p1_face_da_db(p, a, b):
    if p.space == "dg_p1_upwind":
        return dflux(p, a), np.zeros_like(b)
    return 0.5 * (dflux(p, a) + p.lf_a), 0.5 * (dflux(p, b) - p.lf_a)


def _p1_E(p, U):
    uq = np.einsum("mq,...mj->...qj", P1_Q, U)
    V = flux(p, uq).sum(axis=-2)
    uR = np.einsum("m,...mj->...j", P1_RIGHT, U)
    uL = np.einsum("m,...mj->...j", P1_LEFT, U)
    Fp = _p1_face(p, uR, np.roll(uL, -1, axis=-1))
    Fm = np.roll(Fp, 1, axis=-1)
    dphi = np.array([-1.0, 1.0])
    return dphi[:, None] * V[..., None, :] - P1_RIGHT[:, None] * Fp[..., None, :] + P1_LEFT[:, None] * Fm[..., None, :]


def dg1_D(p, U):
    return -np.einsum("mn,...nj->...mj", P1_MINV, _p1_E(p, U)) / p.hx


def dg1_D_jvp(p, U, W):
    uq = np.einsum("mq,...mj->...qj", P1_Q, U)
    wq = np.einsum("mq,...mj->...qj", P1_Q, W)
    dV = (dflux(p, uq) * wq).sum(axis=-2)
    uR = np.einsum("m,...mj->...j", P1_RIGHT, U)
    uL = np.einsum("m,...mj->...j", P1_LEFT, U)
    wR = np.einsum("m,...mj->...j", P1_RIGHT, W)
    wL = np.einsum("m,...mj->...j", P1_LEFT, W)
    da, db = _p1_face_da_db(p, uR, np.roll(uL, -1, axis=-1))
    dFp = da * wR + db * np.roll(wL, -1, axis=-1)
    dFm = np.roll(dFp, 1, axis=-1)
    dphi = np.array([-1.0, 1.0])
    dE = dphi[:, None] * dV[..., None, :] - P1_RIGHT[:, None] * dFp[..., None, :] + P1_LEFT[:, None] * dFm[..., None, :]
    return -np.einsum("mn,...nj->...mj", P1_MINV, dE) / p.hx


def dg1_D_vjp(p, U, Psi):
    """D'(U)^T Psi: with A = -M^{-1 T} Psi / h (M symmetric) the pairing is sum_j A_j . dE_j;
    then dE is transposed term by term (volume, F_{j+1/2}, F_{j-1/2} = F_{(j-1)+1/2})."""
    A = -np.einsum("nm,...nj->...mj", P1_MINV, Psi) / p.hx
    dphi = np.array([-1.0, 1.0])
    uq = np.einsum("mq,...mj->...qj", P1_Q, U)
    cV = np.einsum("m,...mj->...j", dphi, A)                         # coefficient of dV_j
    out = np.einsum("mq,...qj->...mj", P1_Q, dflux(p, uq) * cV[..., None, :])
    G = -np.einsum("m,...mj->...j", P1_RIGHT, A) + np.roll(np.einsum("m,...mj->...j", P1_LEFT, A), -1, axis=-1)
    uR = np.einsum("m,...mj->...j", P1_RIGHT, U)
    uL = np.einsum("m,...mj->...j", P1_LEFT, U)
    da, db = _p1_face_da_db(p, uR, np.roll(uL, -1, axis=-1))           # at face j+1/2
    out = out + P1_RIGHT[:, None] * (G * da)[..., None, :] + P1_LEFT[:, None] * np.roll(G * db, 1, axis=-1)[..., None, :]
    return out


# ---------------------------------------------------------------------------
# dispatch
# ---------------------------------------------------------------------------

def D(p, v):
    if p.space == "dg_p2_lf":
        return dg_D(p, v)
    if p.space.startswith("dg_p1"):
        return dg1_D(p, v)
    return fd_D(p, v)


def D_jvp(p, v, w):
    if p.space == "dg_p2_lf":
        return dg_D_jvp(p, v, w)
    if p.space.startswith("dg_p1"):
        return dg1_D_jvp(p, v, w)
    return fd_D_jvp(p, v, w)


def D_vjp(p, v, psi):
    if p.space == "dg_p2_lf":
        return dg_D_vjp(p, v, psi)
    if p.space.startswith("dg_p1"):
        return dg1_D_vjp(p, v, psi)
    return fd_D_vjp(p, v, psi)


def dof_weight(p) -> float:
    """Spatial quadrature weight of the discrete L2 inner product (Sec. 3.2):
    h_x in 1D (the cell width for DG), h_x h_y in 2D."""
    return p.hx * p.hy if p.dims == 2 else p.hx

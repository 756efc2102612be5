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
# dispatch
# ---------------------------------------------------------------------------

def D(p, v):
    return dg_D(p, v) if p.space == "dg_p2_lf" else fd_D(p, v)


def D_jvp(p, v, w):
    return dg_D_jvp(p, v, w) if p.space == "dg_p2_lf" else fd_D_jvp(p, v, w)


def D_vjp(p, v, psi):
    return dg_D_vjp(p, v, psi) if p.space == "dg_p2_lf" else fd_D_vjp(p, v, psi)


def dof_weight(p) -> float:
    """Spatial quadrature weight of the discrete L2 inner product (Sec. 3.2):
    h_x in 1D (the cell width for DG), h_x h_y in 2D."""
    return p.hx * p.hy if p.dims == 2 else p.hx

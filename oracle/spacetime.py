"""All-slices residual R(u), J(u)v and J(u)^T psi (oracle, float64).

u holds slices l = 0..nt (shape [nt+1, *slice]); R and psi hold one slice per
equation l = 0..nt-1 (shape [nt, *slice]).

Time schemes (Sec. 3.1):
  BE:   R^l = (u^{l+1} - u^l)/h_t + D(u^{l+1}),                       l = 0..nt-1
  BDF2: R^0 as BE (reading: the start of BDF2 is not stated; one BE step),
        R^l = (3u^{l+1} - 4u^l + u^{l-1})/(2h_t) + D(u^{l+1}),        l = 1..nt-1.

The time part of R^m is written as sum_l coef(m, l) u^l.  Then, by summation
by parts (Sec. 3.1), the time part of (J^T psi)^l is sum_m coef(m, l) psi^m,
and the space part is D'(u^l)^T psi^{l-1} for l >= 1 (R^{l-1} holds D(u^l)).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import spatial


def time_coefs(p, m):
    """Nonzero time-stencil entries {l: coef(m, l)} of equation R^m."""
    ht = p.ht
    if p.time == "be" or m == 0:
        return {m + 1: 1.0 / ht, m: -1.0 / ht}
    return {m + 1: 1.5 / ht, m: -2.0 / ht, m - 1: 0.5 / ht}


def residual(p, u):
    """R^l(u) for l = 0..nt-1, all slices at once."""
    R = spatial.D(p, u[1:])
    for m in range(p.nt):
        for l, c in time_coefs(p, m).items():
            R[m] += c * u[l]
    return R


def jvp(p, u, v):
    """J(u) v, the derivative of residual() at u along v."""
    Jv = spatial.D_jvp(p, u[1:], v[1:])
    for m in range(p.nt):
        for l, c in time_coefs(p, m).items():
            Jv[m] += c * v[l]
    return Jv


def vjp(p, u, psi):
    """(J(u)^T psi)^l for l = 0..nt (the transpose of jvp)."""
    g = np.zeros((p.nt + 1,) + psi.shape[1:])
    g[1:] = spatial.D_vjp(p, u[1:], psi)
    for m in range(p.nt):
        for l, c in time_coefs(p, m).items():
            g[l] += c * psi[m]
    return g


def initial_residual(p, u):
    """The initial-condition row of the constraint: u^0 - u0 (Sec. 3.3, Eq. 3.10)."""
    return u[0] - p.u0

"""Derivatives of a terminal objective through the implicit scheme (oracle, float64).

Objective: Loss(u0, nu) = w_x |u^nt - target|^2, with u the scheme's solution
(Sec. 3.1) for initial data u0 and viscosity nu.  Its gradient follows from the
Lagrangian of the saddle form (Eq. 2.7, 3.10) with that objective added,

    L = w_x |u^nt - target|^2 + h_t w_x sum_l <phi^l, R^l(u)> + w_x <lambda, u^0 - u0>,

at its stationary point: R(u) = 0, u^0 = u0, and dL/du = 0, i.e. the discrete
adjoint equations J(u)^T phi = -2 (u^nt - target) / h_t on the last row (zero on
rows 1..nt-1) and lambda = -h_t (J^T phi)^0.  Then

    dLoss/du0 = -w_x lambda,     dLoss/dnu = h_t w_x sum_l <phi^l, dR^l/dnu>.

``sequential_adjoint`` solves the adjoint equations backward in time, one slice
at a time, with the Jacobian blocks c I + D'(u^m) assembled by finite
differences of D (newton.spatial_jacobian), independent of the transposes in
spatial.py; dR/dnu is a central difference of the residual in nu (exact: R is
linear in nu).  The finite-difference check of the gradient itself (Newton
solves at perturbed u0, nu) lives in the tests.

The saddle problem with the objective added is not convex in u when phi != 0
(the curvature of R weighted by phi enters the u-Hessian), and Algorithm 1 does
not converge on it.  ``linearised_step`` is Algorithm 1 on the problem
linearised at the solution u*: state v (a perturbation of u*), residual J(u*) v,
transposes at u*, initial row v^0, and the objective |u*^nt + v^nt - target|^2,
whose last-slice update is its proximal step.  This saddle problem is convex;
its stationary point is v = 0 with the same phi, lambda as above.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import newton, pdhg, precond, spacetime, spatial


def terminal_loss(p, u, target):
    """w_x |u^nt - target|^2."""
    d = u[-1] - target
    return float(spatial.dof_weight(p) * np.sum(d * d))


def dR_dnu(p, u):
    """dR^l/dnu for every slice (central difference; R is affine in nu)."""
    e = 1e-3
    return (spacetime.residual(p.replace(nu=p.nu + e), u) - spacetime.residual(p.replace(nu=p.nu - e), u)) / (2 * e)


def sequential_adjoint(p, u, target):
    """phi solving the adjoint equations for the solution u, backward in time.

    Row m = nt..1 of J^T phi involves phi^{m-1} through the block
    (c_new(m-1) I + D'(u^m))^T and later slices through the time stencil only:
        (c_new I + D'(u^m))^T phi^{m-1} = rhs_m - sum_{l >= m} coef(l, m) phi^l.
    Returns (phi [nt][...], lambda, dLoss/du0, dLoss/dnu)."""
    shape = p.slice_shape
    n = p.ndof
    ht, wx = p.ht, spatial.dof_weight(p)
    coefs = [spacetime.time_coefs(p, l) for l in range(p.nt)]
    phi = np.zeros((p.nt,) + shape)
    for m in range(p.nt, 0, -1):
        rhs = np.zeros(n)
        if m == p.nt:
            rhs -= 2.0 * (u[-1] - target).ravel() / ht
        for l in range(m, p.nt):
            c = coefs[l].get(m, 0.0)
            if c:
                rhs -= c * phi[l].ravel()
        A = coefs[m - 1][m] * sp.identity(n, format="csr") + newton.spatial_jacobian(p, u[m])
        phi[m - 1] = spla.spsolve(A.T.tocsc(), rhs).reshape(shape)
    g0 = np.zeros(shape)
    for l in range(p.nt):
        c = coefs[l].get(0, 0.0)
        if c:
            g0 += c * phi[l]
    lam = -ht * g0
    du0 = -wx * lam
    dnu = float(ht * wx * np.sum(phi * dR_dnu(p, u)))
    return phi, lam, du0, dnu


def pdhg_gradient(p, st):
    """(dLoss/du0, dLoss/dnu) read off a stationary (phi, lambda), with st["u"] the
    solution u* (dR/dnu is taken there)."""
    ht, wx = p.ht, spatial.dof_weight(p)
    du0 = -wx * st["lam"]
    dnu = float(ht * wx * np.sum(st["phi"] * dR_dnu(p, st["u"])))
    return du0, dnu


def linearised_initial_state(p):
    """v = 0, phi = 0, lambda = 0."""
    st = pdhg.initial_state(p)
    st["u"][:] = 0.0
    return st


def linearised_step(p, u_star, st, target):
    """One iteration of Algorithm 1 on the problem linearised at u_star (in place)."""
    ht = p.ht
    v, phit, lamt = st["u"], st["phit"], st["lamt"]
    g = spacetime.vjp(p, u_star, phit)
    vn = v.copy()
    vn[1:] = v[1:] - p.tau_u * g[1:]
    k = 2.0 * p.tau_u / ht
    vn[-1] = (vn[-1] + k * (target - u_star[-1])) / (1.0 + k)
    vn[0] = v[0] - p.tau_u0 * (ht * g[0] + lamt)
    z = precond.kd_inverse(p, spacetime.jvp(p, u_star, vn))
    phi = st["phi"] + p.tau_phi * z
    st["phit"] = 2.0 * phi - st["phi"]
    st["phi"] = phi
    lam = st["lam"] + p.tau_lambda * vn[0]
    st["lamt"] = 2.0 * lam - st["lam"]
    st["lam"] = lam
    st["u"] = vn
    st["iters"] += 1
    return st

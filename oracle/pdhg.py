"""Algorithm 1 (Sec. 3.3): preconditioned PDHG on the whole space-time system,
and the residual Res(u, phi) of Eq. 2.12 (oracle, float64).

Discrete Lagrangian (Eq. 3.10):
    L(u, phi, lambda) = h_t w_x sum_{l<nt} <phi^l, R^l(u)> + w_x <lambda, u^0 - u0>,
with w_x the spatial quadrature weight (h_x; h_x h_y in 2D).

One iteration n (readings, all listed in the design notes):
  1. primal, linearised at u^{n-1} (Eq. 2.11), descent in L2:
       u^l   <- u^l - tau_u  (J(u)^T phit)^l                      l = 1..nt
       u^0   <- u^0 - tau_u0 (h_t (J(u)^T phit)^0 + lamt)          (init "lambda")
     The h_t w_x factors of dL/du are absorbed into the step sizes.  The signs are
     the standard Chambolle-Pock ones (descent in u, ascent in phi and lambda).
  2. dual, in the H-norm of K_d (Eq. 2.9):
       phi    <- phi + tau_phi K_d^{-1} R(u^n),
       lambda <- lambda + tau_lambda (u^0 - u0).
  3. extrapolation: phit = 2 phi^n - phi^{n-1}, lamt = 2 lambda^n - lambda^{n-1}.
Initial guess [u0 extended in t, 0, 0] (Sec. 3.3).  With init "pinned" u^0 stays
u0 and lambda is unused.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import precond, spacetime, spatial


def initial_state(p):
    """[u0 extended in t, 0, 0] (Sec. 3.3)."""
    u = np.broadcast_to(p.u0, (p.nt + 1,) + p.u0.shape).astype(np.float64).copy()
    z = np.zeros((p.nt,) + p.u0.shape)
    return {"u": u, "phi": z.copy(), "phit": z.copy(),
            "lam": np.zeros(p.u0.shape), "lamt": np.zeros(p.u0.shape), "iters": 0}


def step(p, st, signs="standard", target=None):
    """One iteration of Algorithm 1, in place on the state dict ``st``.

    ``signs="paper"`` uses the signs as printed in Algorithm 1 (primal ascent along
    J^T phit, u^0 moved along -(phit^0 - lamt), dual descent); the tests record that
    this choice does not converge (see test_oracle_pdhg).

    ``target`` (a slice) adds the terminal objective w_x |u^nt - target|^2 to the
    Lagrangian (a primal objective in the saddle form of Eq. 2.7; its minimiser
    over u is still the scheme's solution, and phi, lambda become the adjoint).
    Scaled like the other rows of the primal step (by h_t w_x), the u^nt update
    is the proximal step of |v - target|^2 / h_t: with y = u^nt - tau_u (J^T phit)^nt,
    u^nt = (y + (2 tau_u / h_t) target) / (1 + 2 tau_u / h_t)."""
    ht = p.ht
    u, phit, lamt = st["u"], st["phit"], st["lamt"]
    g = spacetime.vjp(p, u, phit)
    un = u.copy()
    if signs == "standard":
        un[1:] = u[1:] - p.tau_u * g[1:]
        if target is not None:
            k = 2.0 * p.tau_u / ht
            un[-1] = (un[-1] + k * target) / (1.0 + k)
        if p.init == "lambda":
            un[0] = u[0] - p.tau_u0 * (ht * g[0] + lamt)
    else:
        un[1:] = u[1:] + p.tau_u * g[1:]
        if p.init == "lambda":
            un[0] = u[0] - p.tau_u0 * (phit[0] - lamt)
    R = spacetime.residual(p, un)
    z = precond.kd_inverse(p, R)
    phi_old = st["phi"]
    phi = phi_old + p.tau_phi * z if signs == "standard" else phi_old - p.tau_phi * z
    st["u"] = un
    st["phi"] = phi
    st["phit"] = 2.0 * phi - phi_old
    if p.init == "lambda":
        lam_old = st["lam"]
        lam = lam_old + p.tau_lambda * spacetime.initial_residual(p, un)
        st["lam"] = lam
        st["lamt"] = 2.0 * lam - lam_old
    st["iters"] += 1
    return st


def residual_norms(p, st, target=None):
    """[||A(u)||, ||grad A(u)^T phi||, ||u^0 - u0||, <phi, R(u)>] (Eq. 2.12).

    Discrete L2 norms weighted by h_t w_x over equation slices and by w_x over the
    initial row.  Entry 0 includes the initial row; entry 1 is the gradient of
    the Lagrangian in u: rows l >= 1 and, with init "lambda", the u^0 row
    h_t (J^T phi)^0 + lambda.  Entry 3 is the Lagrangian value (the duality-gap
    diagnostic: the objective is identically 0)."""
    ht = p.ht
    wx = spatial.dof_weight(p)
    u, phi, lam = st["u"], st["phi"], st["lam"]
    R = spacetime.residual(p, u)
    r0 = spacetime.initial_residual(p, u)
    g = spacetime.vjp(p, u, phi)
    if target is not None:          # gradient of the terminal objective, scaled like J^T phi
        g[-1] += 2.0 * (u[-1] - target) / ht
    a2 = ht * wx * np.sum(R * R)
    b2 = ht * wx * np.sum(g[1:] * g[1:])
    gap = ht * wx * np.sum(phi * R)
    c2 = wx * np.sum(r0 * r0)
    if p.init == "lambda":
        a2 += c2
        g0 = ht * g[0] + lam
        b2 += wx * np.sum(g0 * g0)
        gap += wx * np.sum(lam * r0)
    return np.array([np.sqrt(a2), np.sqrt(b2), np.sqrt(c2), gap])


def solve(p, max_iters=100000, tol=1e-10, check_every=1, relative=False,
          signs="standard", history=False, state=None, target=None):
    """Run Algorithm 1 until each entry of Res is <= tol (Sec. 3.3) or max_iters.

    relative=True scales both entries by ||A(u_init)|| (Res(u_init, 0) has a zero
    second entry).  Returns (state, iterations, history list)."""
    st = initial_state(p) if state is None else state
    hist = []
    scale = 1.0
    if relative:
        scale = residual_norms(p, st, target)[0]
    it = 0
    while it < max_iters:
        step(p, st, signs, target)
        it += 1
        if it % check_every == 0 or it == max_iters:
            res = residual_norms(p, st, target)
            if history:
                hist.append((it, res))
            if not np.all(np.isfinite(res)) or res[0] > 1e30:
                break
            if res[0] <= tol * scale and res[1] <= tol * scale:
                break
    return st, it, hist


def power_estimate(p, iters=60, seed=0):
    """Largest eigenvalue nu_max of the preconditioned operator that bounds the
    step sizes (Sec. 2.2: tau_p tau_q < 1/||A^T A||, with A^T K^{-1} A in place
    of A^T A for the G-prox step, Sec. 2.3), for the problem linearised at u_init:
    power iteration on v -> P^{1/2} J^T K_d^{-1} J P^{1/2} v with the primal
    metric P (h_t-weighted u^0 row) left out, i.e. on rows l >= 1 only."""
    st = initial_state(p)
    u = st["u"]
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(u.shape)
    v[0] = 0.0
    lam = 0.0
    for _ in range(iters):
        v /= np.linalg.norm(v)
        w = spacetime.vjp(p, u, precond.kd_inverse(p, spacetime.jvp(p, u, v)))
        w[0] = 0.0
        lam = float(np.sum(v * w))
        v = w
    return lam

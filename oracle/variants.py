"""The two variants of Algorithm 1 that change its starting point (oracle, float64).

* Algorithm 2 (Sec. 3.4), mesh refinement in time: solve on N x N_t0 slices, carry
  the result to N x 2 N_t0 as the starting point, and so on up to the final mesh.
* Algorithm 3 (Sec. 3.5), one time step at a time: for l = 0..N_t-1 solve the
  two-slice problem on [l h_t, (l+1) h_t] whose initial data is the previous
  step's end value, starting from that value held constant in t.

Readings (the paper leaves these open):
* "simple interpolation" from N_t0 to 2 N_t0 slices is linear in t for u and phi
  at the times the unknowns live at (u^l at l h_t; phi^l, the multiplier of R^l,
  at (l+1) h_t, with phi held constant below the first coarse time); lambda is a
  function of x only and is copied.  The extrapolated duals start equal to the
  duals (phit = phi, lamt = lambda), as at a fresh start.
* Algorithm 3 keeps every input of the full problem (flux, the Lax-Friedrichs
  constant, c, step sizes, h_t) and only shortens the horizon to one step, so its
  end values are the full scheme's solution.  A BDF2 step (l >= 1) is the BE step of
  length 2 h_t / 3 from (4 u^l - u^{l-1}) / 3 (the same equation rearranged); step 0
  is the scheme's BE start.
* Res of a one-step problem (Sec. 3.5) is the L2 norm over the domain at one time:
  the two entries of Eq. 2.12 on that problem (its equation slice and its initial
  row) with the quadrature weight w_x alone, without the h_t of the space-time norm.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import pdhg, spacetime, spatial


def interpolate_t(pc, stc, pf):
    """Starting state on pf (2 pc.nt slices, same horizon) from the state stc on pc."""
    assert pf.nt == 2 * pc.nt
    uc, phic = stc["u"], stc["phi"]
    u = np.empty((pf.nt + 1,) + uc.shape[1:])
    u[0::2] = uc                                   # t = 2l h_f = l h_c
    u[1::2] = 0.5 * (uc[:-1] + uc[1:])             # midpoints
    phi = np.empty((pf.nt,) + phic.shape[1:])
    phi[1::2] = phic                               # fine slice 2l+1 lives at (l+1) h_c
    phi[2::2] = 0.5 * (phic[:-1] + phic[1:])       # fine slice 2l: midway between coarse l-1 and l
    phi[0] = phic[0]                               # below the first coarse time: constant
    lam = stc["lam"].copy()
    return {"u": u, "phi": phi, "phit": phi.copy(), "lam": lam, "lamt": lam.copy(), "iters": 0}


def refine_in_time(p, levels, iters, tol, check_every=1):
    """Algorithm 2 on the final problem p (p.nt divisible by 2^(levels-1)).

    iters[k] is the iteration budget of level k (coarsest first); a level stops early
    once Res <= tol (absolute).  Returns (state on p, iterations per level)."""
    assert len(iters) == levels and p.nt % (1 << (levels - 1)) == 0
    counts = []
    st, prev = None, None
    for k in range(levels):
        pk = p.replace(nt=p.nt >> (levels - 1 - k))
        if st is not None:
            st = interpolate_t(prev, st, pk)
        st, it, _ = pdhg.solve(pk, max_iters=iters[k], tol=tol, check_every=check_every, state=st)
        counts.append(it)
        prev = pk
    return st, counts


def slice_residual_norms(p, st):
    """[||A(u)||, ||grad A(u)^T phi||] of a one-step problem in the L2 norm over the
    domain at one time (Sec. 3.5): weight w_x on every value, no h_t."""
    wx = spatial.dof_weight(p)
    u, phi, lam = st["u"], st["phi"], st["lam"]
    R = spacetime.residual(p, u)
    g = spacetime.vjp(p, u, phi)
    a2 = np.sum(R * R)
    b2 = np.sum(g[1:] * g[1:])
    if p.init == "lambda":
        r0 = spacetime.initial_residual(p, u)
        g0 = p.ht * g[0] + lam
        a2 += np.sum(r0 * r0)
        b2 += np.sum(g0 * g0)
    return np.sqrt(wx * np.array([a2, b2]))


def one_timestep(p, tol, max_iters_per_step=100000, check_every=1):
    """Algorithm 3: u*^0 = u0, then each u*^{l+1} from the two-slice problem on
    [l h_t, (l+1) h_t], iterated until both entries of slice_residual_norms are
    <= tol.  Returns (u* [nt+1][...], iterations per step).

    BDF2 (a reading; the paper states Algorithm 3 for one-step schemes): the equation of
    step l >= 1, (3 v - 4 u^l + u^{l-1}) / (2 h_t) + D(v) = 0, is the backward-Euler
    equation (v - w) / h' + D(v) = 0 with h' = 2 h_t / 3 and w = (4 u^l - u^{l-1}) / 3, so
    that step is the two-slice BE problem of length h' started from w; step 0 is the BE
    start of the scheme (reading 6)."""
    u = np.empty((p.nt + 1,) + p.u0.shape)
    u[0] = p.u0
    counts = []
    for l in range(p.nt):
        if p.time == "bdf2" and l >= 1:
            pl = p.replace(time="be", nt=1, T=2.0 * p.ht / 3.0, u0=(4.0 * u[l] - u[l - 1]) / 3.0)
        else:
            pl = p.replace(time="be", nt=1, T=p.ht, u0=u[l].copy())
        st = pdhg.initial_state(pl)
        it = 0
        while it < max_iters_per_step:
            pdhg.step(pl, st)
            it += 1
            if it % check_every == 0:
                r = slice_residual_norms(pl, st)
                if r[0] <= tol and r[1] <= tol:
                    break
        counts.append(it)
        u[l + 1] = st["u"][1]
    return u, counts

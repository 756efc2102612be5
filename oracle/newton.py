"""The discrete solution by its definition: the implicit scheme marched one time
step at a time (Sec. 3.1), each step solved by Newton's method (oracle, float64).

For l = 0..nt-1 the unknown is v = u^{l+1} and the equation is
    R^l(u^0..u^l, v) = coef(l, l+1) v + sum_{k<=l} coef(l, k) u^k + D(v) = 0,
with u^0 = u0.  The Jacobian coef(l,l+1) I + D'(v) is assembled from central
differences of D with a column colouring that follows the stencil (D is at most
quadratic, so central differences are exact up to rounding); it is therefore
independent of the hand-written D_jvp / D_vjp.  Newton's root does not depend on
the Jacobian, only on R.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import spacetime, spatial


def _colouring(p):
    """Colour classes of dofs whose Jacobian columns do not overlap, plus the row
    neighbourhood of each dof (flat indices)."""
    shape = p.slice_shape
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    if p.nmodes > 1:
        nm = p.nmodes
        m = next(k for k in (3, 4, 5, 6, 7, 8) if p.nx % k == 0) if p.nx >= 3 else p.nx
        cell = np.arange(p.nx)
        colour = (np.arange(nm)[:, None] * m + (cell % m)[None, :])
        nbrs = [np.concatenate([idx[:, (j + d) % p.nx] for d in (-1, 0, 1)]) for j in range(p.nx)]
        nb = {int(idx[mm, j]): nbrs[j] for mm in range(nm) for j in range(p.nx)}
        return colour.ravel(), nb, n
    if p.dims == 2:
        mx = next(k for k in (3, 4, 5, 6, 7, 8) if p.nx % k == 0) if p.nx >= 3 else p.nx
        my = next(k for k in (3, 4, 5, 6, 7, 8) if p.ny % k == 0) if p.ny >= 3 else p.ny
        jy, jx = np.meshgrid(np.arange(p.ny), np.arange(p.nx), indexing="ij")
        colour = (jy % my) * mx + (jx % mx)
        nb = {}
        for y in range(p.ny):
            for x in range(p.nx):
                nb[int(idx[y, x])] = np.array(
                    [idx[y, x], idx[y, (x + 1) % p.nx], idx[y, (x - 1) % p.nx],
                     idx[(y + 1) % p.ny, x], idx[(y - 1) % p.ny, x]])
        return colour.ravel(), nb, n
    m = next(k for k in (3, 4, 5, 6, 7, 8) if p.nx % k == 0) if p.nx >= 3 else p.nx
    colour = np.arange(p.nx) % m
    nb = {j: np.array([(j - 1) % p.nx, j, (j + 1) % p.nx]) for j in range(p.nx)}
    return colour, nb, n


def spatial_jacobian(p, v, eps=1e-4):
    """Sparse D'(v) by coloured central differences."""
    colour, nb, n = _colouring(p)
    shape = p.slice_shape
    rows, cols, vals = [], [], []
    for c in np.unique(colour):
        members = np.nonzero(colour == c)[0]
        e = np.zeros(n)
        e[members] = eps
        e = e.reshape(shape)
        diff = ((spatial.D(p, v + e) - spatial.D(p, v - e)) / (2.0 * eps)).ravel()
        for k in members:
            r = np.unique(nb[int(k)])
            rows.extend(r.tolist())
            cols.extend([int(k)] * len(r))
            vals.extend(diff[r].tolist())
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def solve(p, tol=1e-13, max_newton=60):
    """u^0..u^nt of the implicit scheme, each step to |R^l|_inf <= tol*scale."""
    u = np.empty((p.nt + 1,) + p.slice_shape)
    u[0] = p.u0
    n = p.ndof
    for l in range(p.nt):
        coefs = spacetime.time_coefs(p, l)
        c_new = coefs[l + 1]
        known = sum(c * u[k] for k, c in coefs.items() if k != l + 1)
        v = u[l].copy()
        scale = max(1.0, float(np.max(np.abs(known))))
        for _ in range(max_newton):
            r = c_new * v + known + spatial.D(p, v)
            if np.max(np.abs(r)) <= tol * scale:
                break
            J = c_new * sp.identity(n, format="csr") + spatial_jacobian(p, v)
            dv = spla.spsolve(J.tocsc(), r.ravel())
            v = v - dv.reshape(p.slice_shape)
        else:
            raise RuntimeError(f"Newton did not converge at step {l}")
        u[l + 1] = v
    return u

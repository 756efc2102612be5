"""Exact-rational assembly of 1D DG operators (oracle; Sec. 3.2.2, 3.2.3, App. A).

A generic builder, written once for any polynomial basis on the reference cell
[-1, 1], that produces the semi-discrete DG equations in the form of Eq. 3.8:

  d/dt U_j = sum_{s in {-1,0,1}} [ (U_{j+s}^T Q_s[m] U_{j+s})_m + L_s U_{j+s} ],

for the flux f(u) = alpha u^2 + beta u.  The weak form (Sec. 3.2.2) on cell j is
  M dU_j/dt = int f(u_h) v' dx - Fh_{j+1/2} v(x_{j+1/2}^-) + Fh_{j-1/2} v(x_{j-1/2}^+),
M the mass matrix.  Everything is computed with h = 1 in fractions.Fraction;
every entry scales as 1/h.  Coefficients are returned separately for alpha,
beta and (Lax-Friedrichs) a, so that the paper's C-matrices (App. A, Eq. A.1)
and A1, A2 (Eq. 3.5) can be compared entry by entry.

Bases: ``p1_nodal()`` -- the two nodal functions at x_{j-1/4}, x_{j+1/4} of
Sec. 3.2.2; ``p2_legendre()`` -- P0, P1, P2.
Fluxes: "upwind" -- Fh(u-, u+) = f(u-); "lf" -- (f(u-)+f(u+))/2 - a/2 (u+ - u-).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

from fractions import Fraction as Fr


class Poly:
    """Polynomial in xi with Fraction coefficients (c[k] multiplies xi^k)."""

    def __init__(self, coeffs):
        c = [Fr(x) for x in coeffs]
        while len(c) > 1 and c[-1] == 0:
            c.pop()
        self.c = c

    def __add__(self, o):
        o = o if isinstance(o, Poly) else Poly([o])
        n = max(len(self.c), len(o.c))
        return Poly([(self.c[k] if k < len(self.c) else 0) + (o.c[k] if k < len(o.c) else 0)
                     for k in range(n)])

    __radd__ = __add__

    def __mul__(self, o):
        if not isinstance(o, Poly):
            return Poly([x * Fr(o) for x in self.c])
        out = [Fr(0)] * (len(self.c) + len(o.c) - 1)
        for i, a in enumerate(self.c):
            for j, b in enumerate(o.c):
                out[i + j] += a * b
        return Poly(out)

    __rmul__ = __mul__

    def deriv(self):
        return Poly([k * self.c[k] for k in range(1, len(self.c))] or [0])

    def __call__(self, x):
        x = Fr(x)
        return sum(ck * x ** k for k, ck in enumerate(self.c))

    def integral(self):
        """int_{-1}^{1} p(xi) dxi."""
        return sum(ck * (Fr(1) - Fr(-1) ** (k + 1)) / (k + 1) for k, ck in enumerate(self.c))


def p1_nodal():
    """phi_1(-1/2) = 1, phi_1(1/2) = 0; phi_2(-1/2) = 0, phi_2(1/2) = 1 (Sec. 3.2.2)."""
    return [Poly([Fr(1, 2), -1]), Poly([Fr(1, 2), 1])]


def p2_legendre():
    return [Poly([1]), Poly([0, 1]), Poly([Fr(-1, 2), 0, Fr(3, 2)])]


def _mat_inv(A):
    n = len(A)
    M = [list(map(Fr, row)) + [Fr(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [x / pv for x in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    return [row[n:] for row in M]


def assemble(basis, flux="upwind"):
    """Returns dict with keys ('alpha'|'beta'|'a', s) -> coefficient arrays after
    applying M^{-1} (h = 1):
      ('alpha', s): list over m of n x n symmetric quadratic-form matrices,
      ('beta', s), ('a', s): n x n matrices (row m, column k) of the linear parts.
    """
    n = len(basis)
    mass = [[(basis[i] * basis[j]).integral() * Fr(1, 2) for j in range(n)] for i in range(n)]
    minv = _mat_inv(mass)
    right = [b(1) for b in basis]      # v(x_{j+1/2}^-) for the cell's own functions
    left = [b(-1) for b in basis]      # v(x_{j-1/2}^+)
    dphi = [b.deriv() for b in basis]

    # raw (before M^{-1}) forms: qa[s][m][a][b], lb[s][m][k], la[s][m][k]
    z2 = lambda: [[[Fr(0)] * n for _ in range(n)] for _ in range(n)]
    z1 = lambda: [[Fr(0)] * n for _ in range(n)]
    qa = {s: z2() for s in (-1, 0, 1)}
    lb = {s: z1() for s in (-1, 0, 1)}
    la = {s: z1() for s in (-1, 0, 1)}

    for m in range(n):
        # volume: int f(u_h) phi_m' dxi, u_h = sum_k U_k phi_k (the dx and d/dx scalings cancel)
        for a in range(n):
            lb[0][m][a] += (basis[a] * dphi[m]).integral()
            for b in range(n):
                qa[0][m][a][b] += (basis[a] * basis[b] * dphi[m]).integral()

        # -Fh_{j+1/2} phi_m(1): states uR_j (own cell, traces `right`) and uL_{j+1} (`left`)
        # +Fh_{j-1/2} phi_m(-1): states uR_{j-1} (`right`) and uL_j (`left`)
        for sign, vm, s_minus, s_plus in ((-1, right[m], 0, 1), (1, left[m], -1, 0)):
            w = sign * vm
            if flux == "upwind":          # Fh = f(u-)
                for a in range(n):
                    lb[s_minus][m][a] += w * right[a]
                    for b in range(n):
                        qa[s_minus][m][a][b] += w * right[a] * right[b]
            else:                          # Fh = (f(u-) + f(u+))/2 - a/2 (u+ - u-)
                for a in range(n):
                    lb[s_minus][m][a] += w * Fr(1, 2) * right[a]
                    lb[s_plus][m][a] += w * Fr(1, 2) * left[a]
                    la[s_minus][m][a] += w * Fr(1, 2) * right[a]
                    la[s_plus][m][a] += -w * Fr(1, 2) * left[a]
                    for b in range(n):
                        qa[s_minus][m][a][b] += w * Fr(1, 2) * right[a] * right[b]
                        qa[s_plus][m][a][b] += w * Fr(1, 2) * left[a] * left[b]

    out = {}
    for s in (-1, 0, 1):
        out[("beta", s)] = [[sum(minv[m][i] * lb[s][i][k] for i in range(n)) for k in range(n)]
                            for m in range(n)]
        out[("a", s)] = [[sum(minv[m][i] * la[s][i][k] for i in range(n)) for k in range(n)]
                         for m in range(n)]
        qs = []
        for m in range(n):
            Q = [[sum(minv[m][i] * qa[s][i][a][b] for i in range(n)) for b in range(n)]
                 for a in range(n)]
            Q = [[(Q[a][b] + Q[b][a]) / 2 for b in range(n)] for a in range(n)]
            qs.append(Q)
        out[("alpha", s)] = qs
    return out

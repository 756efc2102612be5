"""The dual-step preconditioner K_d and its inverse (oracle, float64).

K (Eq. 2.8 for linear flux, Eq. 2.10 for nonlinear flux) is
    K = -d_tt - c^2 d_xx + ghat^2 d_xxxx,
with the H-norm boundary term at t = 0 only (Sec. 2.2) and phi^{nt} = 0
(Sec. 3.1).  Sec. 3.3 takes K_d as a discretisation of K; the reading here:

    K_d = T_t / h_t^2  (x)  I  +  I  (x)  K_x,

T_t = tridiag(-1; 1, 2, ..., 2; -1) of size nt (row l = 0 carries the 1: the
Neumann end at t = 0; the Dirichlet end sits beyond l = nt-1).  T_t / h_t^2
equals D_t D_t^T for the backward-Euler difference with u^0 held fixed.
The same T_t is used for BDF2.  An ablation (p.tprec == "exact") replaces T_t by the
scheme's own h_t^2 D_t D_t^T = A_t A_t^T (pentadiagonal for BDF2), applied per Fourier
mode by a dense solve.

K_x for finite differences is diagonal in the discrete Fourier basis with
symbol kappa(theta) = c^2 L(theta) + ghat^2 L(theta)^2, L(theta) = (2 - 2 cos
theta)/h^2 (sum over directions in 2D): the central discretisation of
-c^2 d_xx + ghat^2 d_xxxx.  For DG P2 (a reading: the paper gives K only for
FD), K_x(theta) = S(theta)^H S(theta), S(theta) the Fourier symbol of the DG
operator of c u_x with the upwind flux; for FD this construction gives back
c^2 L(theta) exactly.

Sec. 3.3 notes that inverting K_d is a Laplacian-type solve that an FFT makes
cheap.  The oracle applies K_d^{-1} by an FFT in x (numpy, a library
primitive), a tridiagonal (Thomas) solve along t for every Fourier mode, and
the inverse FFT.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import spacetime, spatial


def symbol_L(n, h):
    """L(theta_k) = (2 - 2 cos(2 pi k / n)) / h^2 for k = 0..n-1."""
    k = np.arange(n)
    return (2.0 - 2.0 * np.cos(2.0 * np.pi * k / n)) / (h * h)


def fd_kappa(p):
    """kappa per rfft mode: shape (nx//2+1,) in 1D, (ny, nx//2+1) in 2D."""
    Lx = symbol_L(p.nx, p.hx)[: p.nx // 2 + 1]
    if p.dims == 2:
        Ly = symbol_L(p.ny, p.hy)
        L = Ly[:, None] + Lx[None, :]
    else:
        L = Lx
    return p.c ** 2 * L + p.gamma_hat ** 2 * L * L


def _upwind_problem(p):
    """The linear problem whose DG operator defines K_x: flux f = c u, and the
    Lax-Friedrichs flux with a = |c| (equal to the upwind flux for constant speed)."""
    q = p.replace(alpha=0.0, beta=p.c, lf_a=abs(p.c), nu=0.0, gamma_half=None)
    if p.space.startswith("dg_p1"):
        q = q.replace(space="dg_p1_lf")
    return q


def dg_symbol_S(p):
    """S(theta_k) for k = 0..ncell//2, shape (ncell//2+1, nm, nm), complex (nm = modes per cell).

    Built by applying the DG operator of c u_x to a unit coefficient in one
    cell: its output in cells j0, j0+1, j0-1 gives the blocks S_0, S_{-1}, S_{+1}
    of (S U)_j = S_0 U_j + S_{-1} U_{j-1} + S_{+1} U_{j+1}, and
    S(theta) = S_0 + S_{-1} e^{-i theta} + S_{+1} e^{i theta}."""
    q = _upwind_problem(p)
    n = p.nx
    nm = p.nmodes
    j0 = 1
    S0 = np.zeros((nm, nm))
    Sm = np.zeros((nm, nm))
    Sp = np.zeros((nm, nm))
    for col in range(nm):
        U = np.zeros((nm, n))
        U[col, j0] = 1.0
        out = spatial.D(q, U)
        S0[:, col] = out[:, j0]
        Sm[:, col] = out[:, (j0 + 1) % n]
        Sp[:, col] = out[:, (j0 - 1) % n]
    theta = 2.0 * np.pi * np.arange(n // 2 + 1) / n
    e = np.exp(-1j * theta)[:, None, None]
    return S0[None] + Sm[None] * e + Sp[None] * np.conj(e)


def dg_Kx(p):
    """K_x(theta_k) = S^H S, shape (ncell//2+1, 3, 3) (no fourth-order term for DG)."""
    assert p.gamma_hat == 0.0
    S = dg_symbol_S(p)
    return np.conj(np.swapaxes(S, -1, -2)) @ S


def thomas_t(rhs, s, ht):
    """Solve (T_t + s) z = h_t^2 rhs along axis 0 for every trailing index.

    rhs: [nt, ...] (complex), s = kappa h_t^2 broadcast over the trailing axes.
    Plain LU without pivoting: d_0 = 1 + s, d_l = 2 + s - 1/d_{l-1};
    y_l = h_t^2 rhs_l + y_{l-1}/d_{l-1};  z_{nt-1} = y/d, z_l = (y_l + z_{l+1})/d_l."""
    nt = rhs.shape[0]
    d = np.empty((nt,) + np.broadcast(rhs[0], s).shape)
    y = np.empty(d.shape, dtype=np.result_type(rhs, np.complex128))
    d[0] = 1.0 + s
    y[0] = ht * ht * rhs[0]
    for l in range(1, nt):
        d[l] = 2.0 + s - 1.0 / d[l - 1]
        y[l] = ht * ht * rhs[l] + y[l - 1] / d[l - 1]
    z = np.empty_like(y)
    z[nt - 1] = y[nt - 1] / d[nt - 1]
    for l in range(nt - 2, -1, -1):
        z[l] = (y[l] + z[l + 1]) / d[l]
    return z


def time_matrix(p):
    """A_t: the time part of the scheme's equations as an nt x nt matrix acting on
    u^1..u^nt (u^0 held fixed), read off the residual's own coefficients
    (spacetime.time_coefs), times h_t: row m is h_t * coef(m, k+1) in column k."""
    A = np.zeros((p.nt, p.nt))
    for m in range(p.nt):
        for k, c in spacetime.time_coefs(p, m).items():
            if k >= 1:
                A[m, k - 1] = c * p.ht
    return A


def exact_Tt(p):
    """The ablation's time operator, h_t^2 D_t D_t^T = A_t A_t^T (Sec. 3.3 takes K_d as
    the discrete operator of K; for BE this is T_t, for BDF2 a pentadiagonal matrix)."""
    A = time_matrix(p)
    return A @ A.T


def exact_t_solve(rhs, s, ht, Tt):
    """Solve (Tt + s) z = h_t^2 rhs along axis 0 for every trailing index (s broadcast over
    the trailing axes), by a dense solve per trailing index (numpy.linalg.solve)."""
    nt = rhs.shape[0]
    tail = rhs.shape[1:]
    sb = np.broadcast_to(s, tail).reshape(-1)
    R = (ht * ht * rhs).reshape(nt, -1).T                       # [n][nt]
    M = Tt[None, :, :] + sb[:, None, None] * np.eye(nt)[None]    # [n][nt][nt]
    Z = np.linalg.solve(M, R[..., None])[..., 0]
    return Z.T.reshape((nt,) + tail)


def _t_solve(p, rhs, s):
    """The time solve of K_d^{-1}: Thomas on T_t, or the exact operator for p.tprec == 'exact'."""
    if getattr(p, "tprec", "tridiag") == "exact":
        return exact_t_solve(rhs, s, p.ht, exact_Tt(p))
    return thomas_t(rhs, s, p.ht)


def kd_inverse(p, r):
    """z = K_d^{-1} r for r of shape [nt, *slice] (real)."""
    ht = p.ht
    if p.nmodes > 1:
        rh = np.fft.rfft(r, axis=-1)                      # [nt][nm][k]
        rh = np.moveaxis(rh, -1, 1)                       # [nt][k][nm]
        lam, V = np.linalg.eigh(dg_Kx(p))                 # K_x = V diag(lam) V^H
        w = np.einsum("kmi,tkm->tki", np.conj(V), rh)     # V^H r
        w = _t_solve(p, w, lam * ht * ht)
        zh = np.einsum("kmi,tki->tkm", V, w)
        zh = np.moveaxis(zh, 1, -1)
        return np.fft.irfft(zh, n=p.nx, axis=-1)
    kappa = fd_kappa(p)
    rh = np.fft.rfft(r, axis=-1)
    if p.dims == 2:
        rh = np.fft.fft(rh, axis=-2)
    zh = _t_solve(p, rh, kappa * ht * ht)
    if p.dims == 2:
        zh = np.fft.ifft(zh, axis=-2)
    return np.fft.irfft(zh, n=p.nx, axis=-1)


# ---------------------------------------------------------------------------
# dense assembly in real space (small grids only; used to pin kd_inverse)
# ---------------------------------------------------------------------------

def dense_Tt(nt):
    T = 2.0 * np.eye(nt) - np.eye(nt, k=1) - np.eye(nt, k=-1)
    T[0, 0] = 1.0
    return T


def _periodic_second_difference(n, h):
    """Matrix of v -> (v_{j+1} - 2 v_j + v_{j-1})/h^2 with periodic wrap."""
    A = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    A[0, -1] = A[-1, 0] = 1.0
    if n == 2:
        A = np.array([[-2.0, 2.0], [2.0, -2.0]])
    return A / (h * h)


def dense_Kx(p):
    """K_x as a real-space matrix (ndof x ndof), from stencils, not symbols."""
    if p.nmodes > 1:
        q = _upwind_problem(p)
        n = p.ndof
        S = np.zeros((n, n))
        for k in range(n):
            e = np.zeros(n)
            e[k] = 1.0
            S[:, k] = spatial.D(q, e.reshape(p.nmodes, p.nx)).ravel()
        return S.T @ S
    Dx = _periodic_second_difference(p.nx, p.hx)
    if p.dims == 2:
        Dy = _periodic_second_difference(p.ny, p.hy)
        Lap = np.kron(np.eye(p.ny), Dx) + np.kron(Dy, np.eye(p.nx))
    else:
        Lap = Dx
    return -p.c ** 2 * Lap + p.gamma_hat ** 2 * (Lap @ Lap)


def dense_Kd(p):
    """K_d = T_t/h_t^2 (x) I + I (x) K_x as an (nt*ndof)^2 matrix (T_t replaced by
    exact_Tt for p.tprec == 'exact')."""
    n = p.ndof
    Tt = exact_Tt(p) if getattr(p, "tprec", "tridiag") == "exact" else dense_Tt(p.nt)
    return np.kron(Tt / p.ht ** 2, np.eye(n)) + np.kron(np.eye(p.nt), dense_Kx(p))

"""Seeded synthetic problem descriptions for the space-time PDHG solver.

This module is shared by the CPU oracle (``oracle/``), the tests, ``bench.py``
and the CUDA binding.  It holds NO arithmetic of the method itself: no residual,
no adjoint, no preconditioner, no PDHG step.  It only describes problems
(grid, flux coefficients, scheme names, step sizes) and draws their initial
data on the host in float64 from ``numpy.random.default_rng(seed)``.

Conventions (shared by every consumer):

* Flux ``f(u) = alpha*u**2 + beta*u`` (the quadratic flux of Sec. 3.2.3; linear
  transport ``f = a*u`` of Sec. 3.2.2 is ``alpha = 0, beta = a``; Burgers is
  ``alpha = 1/2, beta = 0``; the traffic flux of Sec. 4.3 is ``alpha=-1, beta=1``).
* 1D finite differences: ``x_j = j*h_x``, ``h_x = lx/nx`` (Sec. 3.2).  2D: arrays
  are ``[y][x]`` with x fastest, ``h_y = ly/ny``.
* DG P2 (modal Legendre): ``nx`` cells ``[j*h, (j+1)*h]``; one slice is stored
  ``[3][nx]`` (mode-major, cell fastest).
* Time: ``t_l = l*h_t``, ``h_t = T/nt``, ``l = 0..nt`` (Sec. 3.1).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SPACES = ("fd_upwind", "fd_lf", "dg_p2_lf", "dg_p1_upwind", "dg_p1_lf")
TIMES = ("be", "bdf2")
INITS = ("lambda", "pinned")
TPRECS = ("tridiag", "exact")


@dataclass
class Problem:
    """One space-time instance: PDE, discretisation, PDHG step sizes, u0."""

    name: str = ""
    dims: int = 1
    space: str = "fd_upwind"
    time: str = "be"
    nx: int = 64
    ny: int = 1
    lx: float = 2.0 * np.pi
    ly: float = 2.0 * np.pi
    T: float = 1.0
    nt: int = 16
    alpha: float = 0.0          # f(u) = alpha u^2 + beta u
    beta: float = 1.0
    nu: float = 0.0             # constant viscosity: adds -nu * (discrete Laplacian)
    gamma_half: Optional[np.ndarray] = None   # 1D variable coefficient gamma_{j+1/2}
    lf_a: float = 0.0           # global Lax-Friedrichs constant (fd_lf, dg_p2_lf)
    c: float = 1.0              # preconditioner speed (K = -d_tt - c^2 d_xx + ghat^2 d_xxxx)
    gamma_hat: float = 0.0
    tau_u: float = 0.5
    tau_u0: float = 0.5
    tau_phi: float = 0.5
    tau_lambda: float = 0.99
    init: str = "lambda"        # "lambda": Algorithm 1 multiplier; "pinned": u^0 == u0
    u0: Optional[np.ndarray] = None   # one slice, float64, layout per the conventions above
    tprec: str = "tridiag"      # time part of K_d: "tridiag" (T_t for BE and BDF2) or "exact"
                                # (the scheme's own D_t D_t^T: pentadiagonal for BDF2)

    # ---- derived sizes (pure bookkeeping) ----
    @property
    def hx(self) -> float:
        return self.lx / self.nx

    @property
    def hy(self) -> float:
        return self.ly / self.ny if self.dims == 2 else 1.0

    @property
    def ht(self) -> float:
        return self.T / self.nt

    @property
    def nmodes(self) -> int:
        """Degrees of freedom per DG cell (1 for finite differences)."""
        return {"dg_p2_lf": 3, "dg_p1_upwind": 2, "dg_p1_lf": 2}.get(self.space, 1)

    @property
    def ndof(self) -> int:
        if self.nmodes > 1:
            return self.nmodes * self.nx
        return self.nx * (self.ny if self.dims == 2 else 1)

    @property
    def slice_shape(self) -> tuple:
        if self.nmodes > 1:
            return (self.nmodes, self.nx)
        if self.dims == 2:
            return (self.ny, self.nx)
        return (self.nx,)

    @property
    def cells_per_iter(self) -> int:
        """Space-time cell-iterations per PDHG iteration: ndof * nt."""
        return self.ndof * self.nt

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    def validate(self) -> None:
        assert self.space in SPACES and self.time in TIMES and self.init in INITS and self.tprec in TPRECS
        assert self.dims in (1, 2)
        assert self.u0 is not None and self.u0.shape == self.slice_shape
        if self.nmodes > 1:
            assert self.dims == 1
        if self.gamma_half is not None:
            assert self.dims == 1 and self.nmodes == 1
            assert self.gamma_half.shape == (self.nx,)


# --------------------------------------------------------------------------
# grids and initial data (host, float64)
# --------------------------------------------------------------------------

def fd_nodes(nx: int, lx: float) -> np.ndarray:
    """x_j = j * lx / nx (Sec. 3.2)."""
    return np.arange(nx, dtype=np.float64) * (lx / nx)


_GAUSS3_X = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
_GAUSS3_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


def dg_p2_project(fun, nx: int, lx: float) -> np.ndarray:
    """Initial data for DG P2: L2 projection of ``fun`` on Legendre P0..P2 per
    cell, by 3-point Gauss quadrature.  Returns ``[3][nx]``.

    U_{j,m} = (2m+1)/2 * sum_q w_q fun(x_j + xi_q h/2) P_m(xi_q).
    """
    h = lx / nx
    centers = (np.arange(nx) + 0.5) * h
    xq = centers[None, :] + 0.5 * h * _GAUSS3_X[:, None]       # [q][j]
    fq = fun(xq)
    P = np.stack([np.ones(3), _GAUSS3_X, 0.5 * (3 * _GAUSS3_X ** 2 - 1)])  # [m][q]
    U = np.empty((3, nx))
    for m in range(3):
        U[m] = 0.5 * (2 * m + 1) * np.einsum("q,q,qj->j", _GAUSS3_W, P[m], fq)
    return U


def dg_p1_nodes(fun, nx: int, lx: float) -> np.ndarray:
    """Initial data for DG P1 nodal (Sec. 3.2.2): point values at x_{j-1/4}, x_{j+1/4}
    of cell j = [j h, (j+1) h].  Returns ``[2][nx]``."""
    h = lx / nx
    c = (np.arange(nx) + 0.5) * h
    return np.stack([fun(c - 0.25 * h), fun(c + 0.25 * h)])


def random_fourier_2d(n: int, length: float, seed: int, modes: int = 8,
                      amp: float = 0.5, kmax: int = 4) -> np.ndarray:
    """sum_{m<modes} amp*cos(k_m . x + theta_m), k_m uniform in [-kmax,kmax]^2 \\ {0},
    theta_m uniform in [0, 2pi); returned on the n x n grid x_j = j*length/n."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < modes:
        k = rng.integers(-kmax, kmax + 1, size=2)
        if k[0] != 0 or k[1] != 0:
            ks.append(k)
    theta = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    x = fd_nodes(n, length)
    X = x[None, :]
    Y = x[:, None]
    u = np.zeros((n, n))
    for (kx, ky), th in zip(ks, theta):
        u += amp * np.cos(kx * X + ky * Y + th)
    return u


def random_fourier_1d(n: int, length: float, seed: int, modes: int = 8) -> np.ndarray:
    """sum_{k=1..modes} (0.5/k) N(0,1) sin(k x + theta_k) on x_j = j*length/n."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(modes)
    th = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    x = fd_nodes(n, length)
    u = np.zeros(n)
    for k in range(1, modes + 1):
        u += (0.5 / k) * a[k - 1] * np.sin(k * x * (2.0 * np.pi / length) + th[k - 1])
    return u


def random_state(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded N(0, scale^2) array (used to exercise kernels on generic states)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


# --------------------------------------------------------------------------
# named workloads (shapes and parameters of the paper's experiments and the
# benchmark configurations)
# --------------------------------------------------------------------------

def advection_upwind_be(nx: int = 128, nt: int = 64, cfl: float = 2.0,
                        tau=(0.9, 0.9, 0.9, 0.99), init: str = "lambda") -> Problem:
    """u_t + u_x = 0 on periodic [0, 2pi], BE + first-order upwind FD,
    u0 = sin x, h_t = cfl*h_x (Sec. 3.1, 3.2.2; CFL-violating for cfl > 1)."""
    lx = 2.0 * np.pi
    hx = lx / nx
    T = nt * cfl * hx
    u0 = np.sin(fd_nodes(nx, lx))
    return Problem(name=f"advection_upwind_be_{nx}x{nt}", dims=1, space="fd_upwind",
                   time="be", nx=nx, lx=lx, T=T, nt=nt, alpha=0.0, beta=1.0,
                   c=1.0, tau_u=tau[0], tau_u0=tau[1], tau_phi=tau[2],
                   tau_lambda=tau[3], init=init, u0=u0)


def heat_table1(nx: int, nt: int, init: str = "lambda") -> Problem:
    """Variable-coefficient heat equation of Sec. 4.1: [0,1] x [0,0.1],
    gamma(x) = 0.5 + 0.1 sin(2 pi x), u0 = exp(-64 (x-0.5)^2), BE + central FD,
    H-norm ||v_t||^2 + 0.6^2 ||v_xx||^2, (tau_u, tau_phi, tau_lambda) = (0.8, 0.8, 0.99)."""
    lx = 1.0
    hx = lx / nx
    xh = (np.arange(nx) + 0.5) * hx
    gamma_half = 0.5 + 0.1 * np.sin(2.0 * np.pi * xh)
    x = fd_nodes(nx, lx)
    u0 = np.exp(-64.0 * (x - 0.5) ** 2)
    return Problem(name=f"heat_{nx}x{nt}", dims=1, space="fd_upwind", time="be",
                   nx=nx, lx=lx, T=0.1, nt=nt, alpha=0.0, beta=0.0,
                   gamma_half=gamma_half, c=0.0, gamma_hat=0.6,
                   tau_u=0.8, tau_u0=0.8, tau_phi=0.8, tau_lambda=0.99,
                   init=init, u0=u0)


def burgers_dg_p2(ncell: int = 512, nt: int = 256, T: float = 2.0,
                  time: str = "bdf2", tau=(0.5, 0.5, 0.5, 0.99),
                  init: str = "lambda") -> Problem:
    """Inviscid Burgers u_t + (u^2/2)_x = 0 on periodic [0, 2pi], DG P2 with a
    global Lax-Friedrichs flux (a = 1.5), u0 = 0.5 + sin x projected; the
    breaking time of this u0 is 1, so T = 2 is past shock formation."""
    lx = 2.0 * np.pi
    u0 = dg_p2_project(lambda x: 0.5 + np.sin(x), ncell, lx)
    return Problem(name=f"burgers_dg_p2_{ncell}x{nt}", dims=1, space="dg_p2_lf",
                   time=time, nx=ncell, lx=lx, T=T, nt=nt, alpha=0.5, beta=0.0,
                   lf_a=1.5, c=1.5, tau_u=tau[0], tau_u0=tau[1], tau_phi=tau[2],
                   tau_lambda=tau[3], init=init, u0=u0)


def burgers_2d(n: int = 1024, nt: int = 256, seed: int = 20722, cfl: float = 1.0,
               tau=(0.5, 0.5, 0.5, 0.99), init: str = "lambda") -> Problem:
    """2D Burgers u_t + (u^2/2)_x + (u^2/2)_y = 0 on periodic [0,2pi]^2, BE +
    global Lax-Friedrichs FD, h_t = cfl*h_x (default h_t = h_x: T = pi/2 at
    nt = n/4), u0 = 8 random Fourier modes of amplitude 0.5 (seeded); a = c = max|u0|."""
    lx = 2.0 * np.pi
    hx = lx / n
    u0 = random_fourier_2d(n, lx, seed)
    amax = float(np.max(np.abs(u0)))
    return Problem(name=f"burgers2d_{n}x{n}x{nt}", dims=2, space="fd_lf", time="be",
                   nx=n, ny=n, lx=lx, ly=lx, T=nt * cfl * hx, nt=nt, alpha=0.5,
                   beta=0.0, lf_a=amax, c=amax, tau_u=tau[0], tau_u0=tau[1],
                   tau_phi=tau[2], tau_lambda=tau[3], init=init, u0=u0)


def transport_dg_p1(ncell: int = 64, nt: int = 32, T: float = 0.5, time: str = "bdf2",
                    tau=(0.3, 0.1, 0.3, 0.99), init: str = "lambda") -> Problem:
    """Linear transport u_t + 2 u_x = 0 on periodic [0, 1], u0 = sin(2 pi x), DG P1
    nodal + upwind flux, BDF2 (Sec. 4.2, Table 2 uses h_x = h_t)."""
    lx = 1.0
    u0 = dg_p1_nodes(lambda x: np.sin(2.0 * np.pi * x), ncell, lx)
    return Problem(name=f"transport_dg_p1_{ncell}x{nt}", dims=1, space="dg_p1_upwind",
                   time=time, nx=ncell, lx=lx, T=T, nt=nt, alpha=0.0, beta=2.0, lf_a=2.0,
                   c=2.0, tau_u=tau[0], tau_u0=tau[1], tau_phi=tau[2], tau_lambda=tau[3],
                   init=init, u0=u0)


def traffic_dg_p1(ncell: int = 256, nt: int = 32, time: str = "be",
                  tau=(0.4, 0.4, 0.4, 0.99), init: str = "lambda") -> Problem:
    """Traffic flow u_t + (u - u^2)_x = 0 on periodic [0, 2] x [0, 1] with u0 = 0.1 on
    [1, 2] and 0.25 elsewhere, DG P1 nodal + upwind flux (f' >= 0 on the data), BE
    (Sec. 4.3, Eq. 4.1-4.2)."""
    lx = 2.0
    u0 = dg_p1_nodes(lambda x: np.where((x >= 1.0) & (x <= 2.0), 0.1, 0.25), ncell, lx)
    return Problem(name=f"traffic_dg_p1_{ncell}x{nt}", dims=1, space="dg_p1_upwind",
                   time=time, nx=ncell, lx=lx, T=1.0, nt=nt, alpha=-1.0, beta=1.0, lf_a=1.0,
                   c=1.0, tau_u=tau[0], tau_u0=tau[1], tau_phi=tau[2], tau_lambda=tau[3],
                   init=init, u0=u0)


def viscous_burgers(nx: int = 2048, nt: int = 1024, T: float = 2.0, nu: float = 1e-3,
                    tau=(0.5, 0.5, 0.5, 0.99), init: str = "lambda") -> Problem:
    """u_t + (u^2/2)_x = nu u_xx on periodic [0, 2pi], BDF2 + global LF FD +
    central viscous term, u0 = 0.5 + sin x."""
    lx = 2.0 * np.pi
    u0 = 0.5 + np.sin(fd_nodes(nx, lx))
    return Problem(name=f"viscous_burgers_{nx}x{nt}", dims=1, space="fd_lf",
                   time="bdf2", nx=nx, lx=lx, T=T, nt=nt, alpha=0.5, beta=0.0,
                   nu=nu, lf_a=1.5, c=1.5, tau_u=tau[0], tau_u0=tau[1],
                   tau_phi=tau[2], tau_lambda=tau[3], init=init, u0=u0)


def batch_instances(count: int = 256, seed: int = 20723, nx_range=(256, 4096), nt_range=(64, 1024),
                    cfl_range=(1.0, 8.0), tau=(0.5, 0.1, 0.5, 0.99), pow2: bool = False) -> list:
    """A batch of independent 1D problems of mixed kind, size and scheme, drawn
    per instance from default_rng(seed):

    * kind: linear advection u_t + u_x = 0 (upwind FD) or Burgers u_t + (u^2/2)_x = 0
      (global Lax-Friedrichs FD), probability 1/2 each;
    * nx uniform over the integers of the range (pow2=True: a power of two with
      log2 nx uniform over the range);
    * nt uniform in nt_range; CFL = c h_t / h_x uniform in cfl_range; BE or BDF2;
    * u0 = sum_{k=1..8} (0.5/k) N(0,1) sin(k x + theta_k) on [0, 2 pi] (plus 0.5 for
      Burgers), c = a = max |f'(u0)| (1 for advection);
    * step sizes `tau` for BE; for BDF2 tau_u = tau_phi = sqrt(0.5 / (2.5 + nt / 4)) (tau_u0,
      tau_lambda as for BE): with the T_t preconditioner the power estimate of the
      preconditioned operator is about 2 for BE and 2.5 + nt/4 for BDF2 (oracle.pdhg.
      power_estimate, CFL 1..8), so tau_u tau_phi nu_max stays at or below 1/2 for both."""
    rng = np.random.default_rng(seed)
    lo, hi = int(np.log2(nx_range[0])), int(np.log2(nx_range[1]))
    out = []
    for i in range(count):
        burgers = bool(rng.random() < 0.5)
        nx = (1 << int(rng.integers(lo, hi + 1))) if pow2 else int(rng.integers(nx_range[0], nx_range[1] + 1))
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        cfl = float(rng.uniform(*cfl_range))
        time = "bdf2" if rng.random() < 0.5 else "be"
        ts = tau
        if time == "bdf2":
            tb = float(np.sqrt(0.5 / (2.5 + nt / 4.0)))
            ts = (tb, tau[1], tb, tau[3])
        useed = int(rng.integers(0, 2 ** 31 - 1))
        lx = 2.0 * np.pi
        u0 = random_fourier_1d(nx, lx, useed)
        if burgers:
            u0 = u0 + 0.5
            c = float(np.max(np.abs(u0)))
            alpha, beta, space = 0.5, 0.0, "fd_lf"
        else:
            c, alpha, beta, space = 1.0, 0.0, 1.0, "fd_upwind"
        hx = lx / nx
        T = nt * cfl * hx / c
        out.append(Problem(name=f"batch{i}_{'burgers' if burgers else 'advection'}_{nx}x{nt}", dims=1,
                           space=space, time=time, nx=nx, lx=lx, T=T, nt=nt, alpha=alpha, beta=beta,
                           lf_a=c, c=c, tau_u=ts[0], tau_u0=ts[1], tau_phi=ts[2],
                           tau_lambda=ts[3], u0=u0))
    return out

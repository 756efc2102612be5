"""Pins of the oracle's spatial and space-time operators (CPU only).

Each test ties the oracle to something other than itself: the paper's printed
DG matrices, closed-form Fourier symbols, conservation, order of accuracy, the
adjoint identity against finite differences, and special cases that reduce to
a simpler scheme.
"""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import pdhg_workloads as W
from oracle import dg_exact, spacetime, spatial

HERE = os.path.dirname(os.path.abspath(__file__))


def small_problems():
    yield W.advection_upwind_be(nx=8, nt=4)
    yield W.advection_upwind_be(nx=8, nt=4).replace(time="bdf2")
    yield W.heat_table1(8, 4)
    yield W.burgers_dg_p2(ncell=8, nt=4, T=0.5)
    yield W.burgers_dg_p2(ncell=8, nt=4, T=0.5, time="be")
    yield W.burgers_2d(n=8, nt=3)
    yield W.viscous_burgers(nx=8, nt=5, nu=0.05)
    yield W.advection_upwind_be(nx=8, nt=4).replace(alpha=-1.0, beta=1.0)   # traffic flux, upwind
    yield W.transport_dg_p1(ncell=8, nt=4).replace(alpha=0.6, beta=0.3)
    yield W.traffic_dg_p1(ncell=8, nt=3, time="bdf2").replace(space="dg_p1_lf", lf_a=1.3)


@pytest.mark.parametrize("p", list(small_problems()), ids=lambda p: p.name + "_" + p.time)
def test_adjoint_identity_and_jvp(p):
    """<J(u)v, psi> = <v, J(u)^T psi> on random vectors, and J(u)v equals the central
    difference of R (exact up to rounding: R is at most quadratic in u)."""
    rng = np.random.default_rng(7)
    u = rng.standard_normal((p.nt + 1,) + p.slice_shape)
    v = rng.standard_normal(u.shape)
    psi = rng.standard_normal((p.nt,) + p.slice_shape)
    Jv = spacetime.jvp(p, u, v)
    JTpsi = spacetime.vjp(p, u, psi)
    a, b = np.sum(Jv * psi), np.sum(v * JTpsi)
    assert abs(a - b) <= 1e-13 * max(abs(a), np.sum(np.abs(Jv * psi)))
    eps = 1e-5
    fd = (spacetime.residual(p, u + eps * v) - spacetime.residual(p, u - eps * v)) / (2 * eps)
    assert np.max(np.abs(fd - Jv)) <= 1e-8 * np.max(np.abs(Jv))


def _read_paper_matrices():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_dg_p1_matrices.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            fac = Fr(int(t[1]), int(t[2]))
            M = [[fac * int(t[4]), fac * int(t[5])], [fac * int(t[6]), fac * int(t[7])]]
            out[t[0]] = (t[3], M)
    return out


def test_dg_p1_builder_reproduces_paper_matrices():
    """The generic exact DG builder, given the P1 nodal basis and the upwind flux,
    reproduces A1, A2 (Eq. 3.5) and C1..C9 (Eq. A.1) entry by entry."""
    paper = _read_paper_matrices()
    asm = dg_exact.assemble(dg_exact.p1_nodal(), "upwind")
    assert asm[("beta", 0)] == paper["A1"][1]
    assert asm[("beta", -1)] == paper["A2"][1]
    assert asm[("beta", -1)] == paper["C7"][1]
    assert asm[("beta", 0)] == paper["C8"][1]
    assert asm[("beta", 1)] == paper["C9"][1]
    q = {s: asm[("alpha", s)] for s in (-1, 0, 1)}
    assert q[-1][0] == paper["C1"][1] and q[-1][1] == paper["C2"][1]
    assert q[0][0] == paper["C3"][1] and q[0][1] == paper["C4"][1]
    assert q[1][0] == paper["C5"][1] and q[1][1] == paper["C6"][1]


def test_dg_p2_operator_matches_exact_builder():
    """The vectorised DG P2 operator of the oracle equals the exact builder's quadratic
    and linear forms (P2 Legendre basis, Lax-Friedrichs flux) on random data."""
    rng = np.random.default_rng(3)
    n = 9
    p = W.burgers_dg_p2(ncell=n, nt=2).replace(alpha=0.7, beta=-0.3, lf_a=1.9)
    U = rng.standard_normal((3, n))
    asm = dg_exact.assemble(dg_exact.p2_legendre(), "lf")
    h = p.hx
    ref = np.zeros((3, n))
    for j in range(n):
        for s in (-1, 0, 1):
            Us = U[:, (j + s) % n]
            for m in range(3):
                Q = np.array(asm[("alpha", s)][m], dtype=float)
                Lb = np.array(asm[("beta", s)][m], dtype=float)
                La = np.array(asm[("a", s)][m], dtype=float)
                ref[m, j] += (p.alpha * Us @ Q @ Us + p.beta * Lb @ Us + p.lf_a * La @ Us) / h
    # the builder returns dU/dt; D is its negative
    assert np.max(np.abs(spatial.dg_D(p, U) + ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("flux", ["upwind", "lf"])
def test_dg_p1_operator_matches_exact_builder(flux):
    """The vectorised DG P1 nodal operator equals the exact builder's forms (which
    reproduce the paper's A1, A2, C1..C9) on random data, upwind and Lax-Friedrichs."""
    rng = np.random.default_rng(4)
    n = 9
    p = W.transport_dg_p1(ncell=n, nt=2).replace(space=f"dg_p1_{flux}", alpha=0.7, beta=-0.3, lf_a=1.9)
    U = rng.standard_normal((2, n))
    asm = dg_exact.assemble(dg_exact.p1_nodal(), flux)
    ref = np.zeros((2, n))
    for j in range(n):
        for s in (-1, 0, 1):
            Us = U[:, (j + s) % n]
            for m in range(2):
                Q = np.array(asm[("alpha", s)][m], dtype=float)
                Lb = np.array(asm[("beta", s)][m], dtype=float)
                La = np.array(asm[("a", s)][m], dtype=float)
                ref[m, j] += (p.alpha * Us @ Q @ Us + p.beta * Lb @ Us + p.lf_a * La @ Us) / p.hx
    assert np.max(np.abs(spatial.dg1_D(p, U) + ref)) <= 1e-12 * np.max(np.abs(ref))


def test_fd_symbols_closed_form():
    """Linear FD operators on a Fourier mode: upwind speed b gives
    b (1 - e^{-i theta}) / h, the viscous term nu L(theta) (L = (2-2cos)/h^2)."""
    nx = 16
    p = W.advection_upwind_be(nx=nx, nt=2).replace(beta=1.3)
    x = W.fd_nodes(nx, p.lx)
    k = 3
    theta = k * p.hx
    mode = np.exp(1j * k * x)
    got = spatial.fd_D(p, mode.real) + 1j * spatial.fd_D(p, mode.imag)
    assert np.allclose(got, 1.3 * (1 - np.exp(-1j * theta)) / p.hx * mode, atol=1e-12)
    q = p.replace(beta=0.0, nu=0.37)
    got = spatial.fd_D(q, np.sin(k * x))
    L = (2 - 2 * np.cos(theta)) / p.hx ** 2
    assert np.allclose(got, 0.37 * L * np.sin(k * x), atol=1e-12)
    # Lax-Friedrichs with a = |b| on a linear flux equals upwind
    r = p.replace(space="fd_lf", lf_a=1.3)
    v = np.random.default_rng(0).standard_normal(nx)
    assert np.allclose(spatial.fd_D(r, v), spatial.fd_D(p, v), atol=1e-12)


def test_2d_reduces_to_1d():
    """2D Lax-Friedrichs on data that depends on x only equals the 1D scheme row by
    row (the y-differences vanish); swapping x and y transposes the result."""
    rng = np.random.default_rng(5)
    p2 = W.burgers_2d(n=8, nt=2).replace(lf_a=1.7, nu=0.01)
    p1 = p2.replace(dims=1, ny=1, u0=p2.u0[0])
    g = rng.standard_normal(8)
    v = np.broadcast_to(g, (8, 8)).copy()
    d2 = spatial.fd_D(p2, v)
    d1 = spatial.fd_D(p1, g)
    assert np.allclose(d2, np.broadcast_to(d1, (8, 8)), atol=1e-12)
    w = rng.standard_normal((8, 8))
    assert np.allclose(spatial.fd_D(p2, w.T), spatial.fd_D(p2, w).T, atol=1e-12)


@pytest.mark.parametrize("p", [W.burgers_2d(n=8, nt=2), W.burgers_dg_p2(ncell=8, nt=2),
                               W.viscous_burgers(nx=8, nt=2), W.heat_table1(8, 2),
                               W.traffic_dg_p1(ncell=8, nt=2)],
                         ids=lambda p: p.name)
def test_spatial_conservation(p):
    """Periodic fluxes telescope: sum_j D(v)_j = 0 (DG: the cell averages -- the P0 mode
    for P2, (U1 + U2)/2 for the P1 nodal basis)."""
    v = np.random.default_rng(2).standard_normal(p.slice_shape)
    d = spatial.D(p, v)
    s = d[0].sum() if p.space == "dg_p2_lf" else (d.sum() / 2 if p.nmodes == 2 else d.sum())
    assert abs(s) <= 1e-11 * np.sum(np.abs(d))


def test_dg_p2_order_of_accuracy():
    """On smooth data D(Pi u) approximates Pi(f(u)_x): the error of the cell averages
    falls by about 2^3 per halving of h (third order for P2)."""
    errs = []
    for n in (16, 32, 64):
        p = W.burgers_dg_p2(ncell=n, nt=2).replace(lf_a=2.0)
        u = lambda x: 0.5 + np.sin(x)
        U = W.dg_p2_project(u, n, p.lx)
        ex = W.dg_p2_project(lambda x: (0.5 + np.sin(x)) * np.cos(x), n, p.lx)
        errs.append(np.sqrt(p.hx * np.sum((spatial.dg_D(p, U)[0] - ex[0]) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 2.5), orders


def test_heat_laplacian_order_of_accuracy():
    """-Lap_gamma(u) approximates -(gamma u')' to second order."""
    errs = []
    for n in (32, 64, 128):
        p = W.heat_table1(n, 2)
        x = W.fd_nodes(n, 1.0)
        u = np.sin(2 * np.pi * x)
        g = lambda x: 0.5 + 0.1 * np.sin(2 * np.pi * x)
        dg = lambda x: 0.2 * np.pi * np.cos(2 * np.pi * x)
        exact = -(dg(x) * 2 * np.pi * np.cos(2 * np.pi * x) - g(x) * 4 * np.pi ** 2 * np.sin(2 * np.pi * x))
        errs.append(np.max(np.abs(spatial.fd_D(p, u) - exact)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.9), orders

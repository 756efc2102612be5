"""GPU parity of the fused 2D path (float32): primal / rows-R / cols / rows-C kernels.

* small and mid sizes: n iterations element by element against the float64
  oracle and against the plain path (several row blocks, several t-chunks, a
  ragged last chunk, nx != ny, BE and BDF2, lambda and pinned initial rows);
* the full benchmark size (1024 x 1024 x 256, the launch configuration that
  bench.py times), on outputs the oracle computes one by one: the K_d^{-1} R
  spectrum at sampled Fourier modes (a tridiagonal solve per mode), the primal
  step at sampled points, and the float64 residual norms.
"""
import numpy as np
import pytest

import pdhg_workloads as W
from oracle import newton, pdhg as opdhg
from oracle import precond, spacetime, spatial

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2207_07234_gb300 import binding
    binding.load()
    return binding


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))


def small_cases():
    base = dict(tau_u=0.4, tau_phi=0.4, tau_u0=0.1, tau_lambda=0.99)
    yield W.burgers_2d(n=256, nt=71).replace(**base)                       # t-chunks, ragged last (71 prime)
    yield W.burgers_2d(n=256, nt=9).replace(time="bdf2", **base)            # chunks of 8 and 1, BDF2
    yield W.burgers_2d(n=256, nt=6).replace(init="pinned", nu=0.02, **base)
    p = W.burgers_2d(n=512, nt=5).replace(**base)
    yield p.replace(ny=256, ly=np.pi, u0=np.ascontiguousarray(p.u0[:256]))   # nx != ny
    yield W.burgers_2d(n=256, nt=7).replace(space="fd_upwind", alpha=0.0, beta=1.0, **base)
    yield W.burgers_2d(n=1024, nt=3).replace(**base)                         # the ny = 1024 column kernel
    p = W.burgers_2d(n=1024, nt=5).replace(**base)                          # TMA rows-C with ny = 512
    yield p.replace(ny=512, ly=np.pi, u0=np.ascontiguousarray(p.u0[:512]))
    p = W.burgers_2d(n=2048, nt=3).replace(**base)                          # nx = 2048: radix-2 + 3 radix-8
    yield p.replace(ny=256, ly=np.pi / 4, u0=np.ascontiguousarray(p.u0[:256]))
    # one time slice: the two-slice problems of Algorithm 3's steps
    yield W.burgers_2d(n=256, nt=1).replace(**base)
    yield W.burgers_2d(n=256, nt=1).replace(init="pinned", **base)
    yield W.burgers_2d(n=1024, nt=1).replace(init="pinned", **base)        # the nx = ny = 1024 kernels


@pytest.mark.parametrize("p", list(small_cases()), ids=lambda p: f"{p.name}_{p.time}_{p.init}_{p.ny}")
def test_fused_matches_oracle_and_plain(B, p):
    n = 4
    with B.Solver(p, precision="fp32", path="fused") as s:
        assert s.info()["path"] == "fused"
        s.iterate(n)
        assert s.launches() == 4 * n
        g = {k: s.get_host(k) for k in ("u", "phi", "phit", "lambda")}
        rg = s.residual()
    with B.Solver(p, precision="fp32", path="plain") as s:
        s.iterate(n)
        pl = {k: s.get_host(k) for k in ("u", "phi", "phit")}
    st = opdhg.initial_state(p)
    u_init = st["u"].copy()
    for _ in range(n):
        opdhg.step(p, st)
    # the increments u - u_init and the multipliers (which start at 0), each to 1e-5 of
    # its own largest value: float32 arithmetic (unit roundoff 6e-8, a few roundings per
    # step, the float32-rounded u0) stays far inside it; an error in any update would not.
    # u itself is rounded to float32 once per iteration by each float32 path, n 2^-24
    # max|u| each, which the increment bound adds (with one moving slice and small
    # steps the increment after n iterations is small next to u)
    du = st["u"] - u_init
    ur = n * 2.0 ** -24 * np.max(np.abs(st["u"]))
    assert np.max(np.abs(g["u"] - st["u"])) <= 1e-5 * np.max(np.abs(du)) + ur
    assert rel(g["phi"], st["phi"]) <= 1e-5
    assert rel(g["phit"], st["phit"]) <= 1e-5
    assert np.max(np.abs(g["u"] - pl["u"])) <= 1e-5 * np.max(np.abs(pl["u"] - u_init)) + 2 * ur
    assert rel(g["phi"], pl["phi"]) <= 1e-5
    ro = opdhg.residual_norms(p, st)
    assert np.allclose(rg[:3], ro[:3], rtol=1e-4)


def test_fused_converges_like_plain(B):
    """Both float32 paths reach the same relative residual in the same number of
    checked iterations on a small nonlinear problem (short horizon, T = pi/8,
    before the shocks, where Algorithm 1 converges)."""
    p = W.burgers_2d(n=256, nt=16, cfl=0.5).replace(tau_u=0.5, tau_phi=0.5, tau_u0=0.1)
    its = {}
    for path in ("fused", "plain"):
        with B.Solver(p, precision="fp32", path=path) as s:
            its[path] = s.iterate(3000, tol=1e-4, check_every=20, relative=True)
            assert its[path] < 3000
            its[path + "_u"] = s.get_host("u")
    assert abs(its["fused"] - its["plain"]) <= 40
    assert rel(its["fused_u"], its["plain_u"].astype(np.float64)) <= 1e-4


def test_fused_fp32_converged_matches_newton(B):
    """Algorithm 1 on the fused float32 path, run until float32's rounding stops it (a
    relative Res of a few 1e-6 on this problem: checked to be below 1e-5), lands
    within 1e-5 relative L-inf of the discrete solution, i.e. the oracle's Newton
    time-stepper (the definition of the implicit scheme's solution): 2D Burgers
    256^2 x 8 at h_t = h_x / 2 (T = pi/32, before shocks form).  The mixed solve
    (the same float32 iterations, then float64) goes on past that floor to relative
    Res 1e-10 and then matches the Newton solution to 1e-9."""
    p = W.burgers_2d(n=256, nt=8, cfl=0.5).replace(tau_u=0.5, tau_phi=0.5, tau_u0=0.1)
    un = newton.solve(p)
    scale = float(np.max(np.abs(un)))
    r0 = opdhg.residual_norms(p, opdhg.initial_state(p))[0]
    with B.Solver(p, precision="fp32", path="fused") as s:
        assert s.info()["path"] == "fused"
        s.iterate(6000, tol=1e-6, check_every=20, relative=True)
        r = s.residual()
        u = s.get_host("u").astype(np.float64)
    floor = max(r[0], r[1]) / r0
    assert floor <= 1e-5, floor
    assert np.max(np.abs(u - un)) <= 1e-5 * scale, (np.max(np.abs(u - un)) / scale, floor)
    s, its = B.solve_mixed(p, tol=1e-10, relative=True, check_every=20, max_iters=30000, path="fused")
    try:
        r = s.residual()
        u = s.get_host("u")
    finally:
        s.close()
    assert max(r[0], r[1]) <= 1e-10 * r0, (its, r)
    assert np.max(np.abs(u - un)) <= 1e-9 * scale, np.max(np.abs(u - un)) / scale


def _dft2_mode(a, kx, ky):
    """sum_{y,x} a[..., y, x] exp(-2 pi i (kx x / nx + ky y / ny)) for each leading index."""
    ny, nx = a.shape[-2:]
    ex = np.exp(-2j * np.pi * kx * np.arange(nx) / nx)
    ey = np.exp(-2j * np.pi * ky * np.arange(ny) / ny)
    return (a.astype(np.float64) @ ex) @ ey


def test_full_size_sampled(B):
    """1024 x 1024 x 256 in the benchmark configuration."""
    import bench
    p = bench.workload("burgers2d")
    rng = np.random.default_rng(5)
    with B.Solver(p, precision="fp32", path="auto") as s:
        assert s.info()["path"] == "fused"
        s.iterate(1)
        phi1 = s.get_host("phi")
        phit1 = s.get_host("phit")
        u1 = s.get_host("u")
        s.iterate(1)
        u2 = s.get_host("u")
        res2 = s.residual()
    # (a) iteration 1: phi^1 = tau_phi K_d^{-1} R(u_init); u is still u0 extended, so every
    # slice of R is D(u0).  Check sampled Fourier modes against the oracle's per-mode solve.
    assert np.array_equal(u1[1:], np.broadcast_to(p.u0.astype(np.float32), u1[1:].shape))
    Du0 = spatial.D(p, p.u0)
    kappa = precond.fd_kappa(p)
    modes = [(0, 0), (1, 0), (0, 3), (2, 5), (4, 4), (7, 1000), (100, 17), (511, 511), (512, 0)]
    zr, zg = {}, {}
    for kx, ky in modes:
        r_hat = _dft2_mode(Du0[None], kx, ky)[0] * np.ones(p.nt)
        zr[kx, ky] = precond.thomas_t(r_hat[:, None], np.array([kappa[ky, kx] * p.ht ** 2]), p.ht)[:, 0]
        zg[kx, ky] = _dft2_mode(phi1, kx, ky) / p.tau_phi
    Z = max(np.max(np.abs(v)) for v in zr.values())
    for m in modes:
        err = np.max(np.abs(zg[m] - zr[m]))
        own = np.max(np.abs(zr[m]))
        # float32 transforms and t-recurrence against the float64 per-mode solve: an absolute
        # floor of the float32 2D transform of values of size Z (measured 2.1e-5 Z on an
        # absent mode) plus 1e-4 of the mode itself
        assert err <= 5e-5 * Z + 1e-4 * own, (m, err, own, Z)
    assert np.array_equal(phit1, 2 * phi1) or rel(phit1, 2 * phi1.astype(np.float64)) <= 1e-6
    # (b) iteration 2: the primal step at sampled points from the GPU's own phit^1
    for _ in range(200):
        l = int(rng.integers(1, p.nt + 1))
        y, x = int(rng.integers(0, p.ny)), int(rng.integers(0, p.nx))
        # time part: (phit^{l-1} - phit^l)/h_t (phit^{nt} = 0); space part at one point
        t_part = phit1[l - 1, y, x] / p.ht - (phit1[l, y, x] / p.ht if l < p.nt else 0.0)
        psi = phit1[l - 1].astype(np.float64)
        win = np.zeros((3, 3))
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                win[dy + 1, dx + 1] = psi[(y + dy) % p.ny, (x + dx) % p.nx]
        # D'(u)^T psi at the point from the oracle's 2D operator applied to a 3x3 periodic patch
        q = p.replace(nx=3, ny=3, lx=3 * p.hx, ly=3 * p.hy)
        v = np.full((3, 3), float(u1[l, y, x]))
        s_part = spatial.fd_D_vjp(q, v, win)[1, 1]
        ref = float(u1[l, y, x]) - p.tau_u * (t_part + s_part)
        assert abs(float(u2[l, y, x]) - ref) <= 1e-5 * max(1.0, abs(ref)), (l, y, x)
    # (c) float64 residual norms of the float32 state against the oracle on the same state
    u64 = u2.astype(np.float64)
    R = spacetime.residual(p, u64)
    r0 = u64[0] - p.u0
    a = np.sqrt(p.ht * p.hx * p.hy * np.sum(R * R) + p.hx * p.hy * np.sum(r0 * r0))
    assert abs(res2[0] - a) <= 1e-4 * a


def test_wait_budget_timeout_is_reported(B):
    """The bounded TMA stage waits of rows-C (nx = 1024): with a zero budget every wait
    gives up, the blocks drain their copies and return, and the next residual check
    reports PDHG_ERR_TIMEOUT; the CUDA context stays usable for the next handle."""
    p = W.burgers_2d(n=1024, nt=3).replace(tau_u=0.4, tau_phi=0.4, tau_u0=0.1, tau_lambda=0.99)
    with B.Solver(p, precision="fp32", path="fused") as s:
        s.set_wait_budget(0)
        with pytest.raises(B.PdhgError) as e:
            s.iterate(2, tol=0.0, check_every=1)
        assert e.value.status == -6
    with B.Solver(p, precision="fp32", path="fused") as s:
        s.set_wait_budget(10**9)
        s.iterate(2, tol=0.0, check_every=1)
        assert np.all(np.isfinite(s.residual()))

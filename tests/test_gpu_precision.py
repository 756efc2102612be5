"""The float32 error against the float64 oracle, per configuration.

The float32 path keeps the stencils, the FFT preconditioner and the dual step in
float32 and the residual reductions in float64.  For each named configuration (at
its own size where the oracle finishes in seconds, else with that configuration's
kernels on fewer time slices) this module measures how far a float32 result lies
from the float64 oracle on the same seeded input, bounds it, and prints it
(``PRECISION <configuration> <quantity> <value>``; ``pytest -s`` shows the lines):

* advection 128 x 64, BE + upwind, CFL 2: the float32 solution run to its rounding
  floor (4000 iterations; float64 reaches relative Res 1e-6 in 1250) against the
  closed-form discrete solution, relative L-inf;
* DG P2 Burgers 512 cells x 256 slices, BDF2, T = 2: 20 fixed iterates at the BDF2
  step sizes sqrt(0.5 / (2.5 + nt/4)) (Algorithm 1 does not converge past the shock),
  the increments u - u_init and phi on their own scales;
* viscous Burgers 2048 x 1024, BDF2, nu = 1e-3 (the gradient workload's forward problem
  at its own size, in the benchmark's launch configuration): 20 fixed iterates, u to the
  float32 forward-error bound of its update stencil (large cancelling coefficients at
  nt = 1024; see the test), phi as above;
* 2D Burgers 1024 x 1024 (BE + global LF; the nx = ny = 1024 fused kernels) on 6
  slices: 4 fixed iterates, as above;
* the batch: two BE and two BDF2 instances of the 256-instance draw (the smallest
  of each, non-power-of-two nx: Bluestein x-transforms), 10 fixed iterates in one
  batch, as above;
* the gradient workload's scheme (viscous Burgers, BDF2, nu = 1e-3) before the shock
  with the exact time operator at 128 x 64: the float32 gradient (dLoss/du0,
  dLoss/dnu) against the oracle's sequential adjoint of the Newton solution.

Fixed-iterate bounds are 1e-5 of each field's own largest value (the stated float32
tolerance), for u plus the float32 rounding of u itself over the iterations; the floor
solution's, 1e-5 relative L-inf; the gradient's, 1e-4 of the
largest dLoss/du0 (the product of the float32 floors of two solves and the
conditioning of the linearised problem, see tests/test_gpu_adjoint.py).
"""
import numpy as np
import pytest

import pdhg_workloads as W
from oracle import adjoint, newton, pdhg as opdhg

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


def report(config, quantity, value):
    print(f"PRECISION {config} {quantity} {value:.3e}")


def oracle_iterates(p, n):
    st = opdhg.initial_state(p)
    for _ in range(n):
        opdhg.step(p, st)
    return st


def increments(config, g_u, g_phi, p, n):
    """The increment u - u_init to 1e-5 of its own largest value plus the rounding of the
    stored u itself (n iterations, each rounding u to float32: n 2^-24 max|u|; at small
    step sizes the increment after a few iterations is small next to u); phi (which
    starts at 0) to 1e-5 of its largest value."""
    o = oracle_iterates(p, n)
    u_init = opdhg.initial_state(p)["u"]
    du_o = o["u"] - u_init
    err_u = float(np.max(np.abs(np.asarray(g_u, np.float64) - o["u"])))
    ep = rel(g_phi, o["phi"])
    report(config, f"u-u_init_after_{n}_rel_to_increment", err_u / np.max(np.abs(du_o)))
    report(config, f"u_after_{n}_rel_to_u", err_u / np.max(np.abs(o["u"])))
    report(config, f"phi_after_{n}", ep)
    assert err_u <= 1e-5 * np.max(np.abs(du_o)) + n * 2.0 ** -24 * np.max(np.abs(o["u"])), err_u
    assert ep <= 1e-5, ep


def test_advection_128x64_float32_floor_against_closed_form(B):
    import test_oracle_solution as tos
    p = W.advection_upwind_be().replace(tau_u=1.4, tau_u0=0.1, tau_phi=0.35, tau_lambda=0.99)
    exact = tos._mode_closed_form_be(p)
    with B.Solver(p, precision="fp32", path="plain") as s:
        s.iterate(4000)
        u = s.get_host("u")
        r = s.residual()
    e = rel(u, exact)
    report("advection_128x64", "u_at_float32_floor_vs_closed_form", e)
    report("advection_128x64", "abs_res_at_float32_floor", max(r[0], r[1]))
    assert e <= 1e-5


def test_dg_p2_burgers_512x256_fixed_iterates(B):
    # BDF2 with T_t: step sizes sqrt(0.5 / (2.5 + nt/4)) (the batch workload's rule); 0.2
    # leaves the iteration's stable range at nt = 256 within 20 iterations
    t = float(np.sqrt(0.5 / (2.5 + 256 / 4.0)))
    p = W.burgers_dg_p2(tau=(t, 0.1, t, 0.99)).replace(c=0.5)
    with B.Solver(p, precision="fp32", path="plain") as s:
        s.iterate(20)
        gu, gphi = s.get_host("u"), s.get_host("phi")
    increments("dg_p2_burgers_512x256_bdf2", gu, gphi, p, 20)


def test_viscous_burgers_2048x1024_fixed_iterates(B):
    """The gradient workload's forward problem at its own size (viscous Burgers 2048 x 1024,
    BDF2, nu = 1e-3, T = 2), in the launch configuration the benchmark's gradient leg times
    (plain path, steps 0.05): 20 fixed iterates in float32 and in float64 against the
    oracle's.

    At nt = 1024 the stencil of J^T phit has large coefficients of both signs (the BDF2
    time part 4/h_t = 2048, the space part max|u|/h_x + 2a/h_x + 4 nu/h_x^2 ~ 2000) whose
    terms cancel, so float32 rounding of the primal update is not small next to the
    increment as it is on the short grids above.  Its bound is the forward error of a
    k-term float32 sum (Higham's gamma_k = k u / (1 - k u), u = 2^-24, k = 16) applied
    to each iteration's update: sum over iterations of gamma_16 tau_u C_T max|phit|,
    C_T the sum of the stencil's absolute coefficients; plus the rounding of the stored
    u (n 2^-24 max|u|) and the stated float32 tolerance, 1e-5 of the increment.  (A
    root-sum-square model of the same roundings, sqrt(n k) u tau_u C_T max|phit|, gives
    3.0e-5 absolute; the measured error is 2.8e-5, 1.5e-5 of max|u|.)  phi keeps the 1e-5
    bound.  In float64, 1e-11 of the increment."""
    p = W.viscous_burgers().replace(tau_u=0.05, tau_phi=0.05, tau_u0=0.05)
    n = 20
    o = opdhg.initial_state(p)
    u_init = o["u"].copy()
    phit_max = 0.0
    for _ in range(n):
        opdhg.step(p, o)
        phit_max += float(np.max(np.abs(o["phit"])))
    hx, ht = p.lx / p.nx, p.T / p.nt
    c_t = 4.0 / ht + np.max(np.abs(o["u"])) / hx + 2.0 * p.lf_a / hx + 4.0 * p.nu / hx ** 2
    u32 = 2.0 ** -24
    gamma16 = 16 * u32 / (1 - 16 * u32)
    du_o = o["u"] - u_init
    with B.Solver(p, precision="fp32", path="plain") as s:
        s.iterate(n)
        gu, gphi = s.get_host("u"), s.get_host("phi")
    err_u = float(np.max(np.abs(np.asarray(gu, np.float64) - o["u"])))
    ep = rel(gphi, o["phi"])
    report("viscous_burgers_2048x1024_bdf2", f"u-u_init_after_{n}_rel_to_increment", err_u / np.max(np.abs(du_o)))
    report("viscous_burgers_2048x1024_bdf2", f"u_after_{n}_rel_to_u", err_u / np.max(np.abs(o["u"])))
    report("viscous_burgers_2048x1024_bdf2", f"phi_after_{n}", ep)
    bound = (1e-5 * np.max(np.abs(du_o)) + n * u32 * np.max(np.abs(o["u"])) +
             gamma16 * p.tau_u * c_t * phit_max)
    assert err_u <= bound, (err_u, bound)
    assert ep <= 1e-5, ep
    with B.Solver(p, precision="fp64", path="plain") as s:
        s.iterate(n)
        gu, gphi = s.get_host("u"), s.get_host("phi")
    assert np.max(np.abs(gu - o["u"])) <= 1e-11 * np.max(np.abs(du_o))
    assert rel(gphi, o["phi"]) <= 1e-11


def test_burgers2d_1024_fused_fixed_iterates(B):
    p = W.burgers_2d(n=1024, nt=6, tau=(0.15, 0.1, 0.15, 0.99))
    with B.Solver(p, precision="fp32", path="fused") as s:
        s.iterate(4)
        gu, gphi = s.get_host("u"), s.get_host("phi")
    increments("burgers2d_1024x1024_fused", gu, gphi, p, 4)


def test_batch_instances_fixed_iterates(B):
    probs = W.batch_instances()
    pick = []
    for scheme in ("be", "bdf2"):
        idx = sorted((i for i in range(len(probs)) if probs[i].time == scheme), key=lambda i: probs[i].cells_per_iter)
        pick += idx[:2]
    sel = [probs[i] for i in pick]
    with B.Batch(sel, precision="fp32") as bt:
        bt.iterate(10)
        got = [(bt.instance(k).get_host("u"), bt.instance(k).get_host("phi")) for k in range(len(sel))]
    for i, p, (gu, gphi) in zip(pick, sel, got):
        increments(f"batch_instance_{i}_{p.nx}x{p.nt}_{p.time}", gu, gphi, p, 10)


def test_gradient_scheme_float32_gradient(B):
    p = W.viscous_burgers(nx=128, nt=64, T=0.5, nu=1e-3).replace(tprec="exact")
    t = float(np.sqrt(0.4 / opdhg.power_estimate(p, iters=60)))
    p = p.replace(tau_u=t, tau_u0=t, tau_phi=t)
    g = 0.5 + 0.9 * np.sin(W.fd_nodes(p.nx, p.lx) - 1.0)
    u = newton.solve(p)
    _, _, du0, dnu = adjoint.sequential_adjoint(p, u, g)
    _, du0_32, dnu_32, _ = B.solve_gradient(p, g, tol=1e-5, max_iters=20000, adj_tol=0.0, adj_max_iters=20000,
                                            check_every=100, precision="fp32")
    e0 = float(np.max(np.abs(du0_32 - du0)) / np.max(np.abs(du0)))
    e1 = abs(dnu_32 - dnu) / max(abs(dnu), np.max(np.abs(du0)))
    report("viscous_burgers_128x64_bdf2_exact_time_operator", "dLoss_du0", e0)
    report("viscous_burgers_128x64_bdf2_exact_time_operator", "dLoss_dnu", e1)
    assert e0 <= 1e-4 and e1 <= 1e-4

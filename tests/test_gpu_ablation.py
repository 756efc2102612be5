"""The preconditioner ablation of Sec. 3.3's K_d on the GPU (PDHG_FLAG_EXACT_TIME_PRECOND):
the time part of K_d as the scheme's own h_t^2 D_t D_t^T (pentadiagonal for BDF2) in
place of T_t = tridiag(-1; 1, 2, ..., 2; -1).

* fixed iterates with the exact operator equal the oracle's (float64, element by element);
* the fixed point is unchanged: converged u equals the Newton time-stepper;
* iteration counts to relative Res 1e-8 equal the oracle's for both operators on the two
  BDF2 cases (DG P1 transport of Table 2's setup, upwind advection), and the exact
  operator needs fewer iterations.
"""
import numpy as np
import pytest

import pdhg_workloads as W
from oracle import newton, pdhg as opdhg

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


def steps(p, fac):
    """tau_u = tau_phi = sqrt(fac / nu_max), nu_max the oracle's power estimate for p's K_d."""
    t = float(np.sqrt(fac / opdhg.power_estimate(p, iters=100)))
    return p.replace(tau_u=t, tau_phi=t, tau_u0=0.1, tau_lambda=0.99)


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))


FIXED = [steps(W.advection_upwind_be(nx=256, nt=9).replace(time="bdf2", tprec="exact"), 0.8),
         steps(W.transport_dg_p1(ncell=128, nt=11).replace(tprec="exact"), 1.0),
         steps(W.burgers_dg_p2(ncell=64, nt=7, T=0.5).replace(c=0.5, tprec="exact"), 1.0),
         steps(W.burgers_2d(n=32, nt=6).replace(time="bdf2", tprec="exact"), 0.8),
         steps(W.viscous_burgers(nx=128, nt=6, T=0.5, nu=0.01).replace(time="bdf2", tprec="exact"), 0.8)]


@pytest.mark.parametrize("p", FIXED, ids=lambda p: p.name)
def test_exact_time_operator_fixed_iterates(B, p):
    n = 20
    with B.Solver(p, precision="fp64") as s:
        assert s.info()["path"] == "plain"
        s.iterate(n)
        g = {k: s.get_host(k) for k in ("u", "phi", "phit")}
    st = opdhg.initial_state(p)
    for _ in range(n):
        opdhg.step(p, st)
    tu = 1e-11 if p.nmodes == 2 else 1e-12          # DG P1: the sensitivity noted in test_gpu_parity
    assert rel(g["u"], st["u"]) <= tu
    assert rel(g["phi"], st["phi"]) <= 10 * tu
    assert rel(g["phit"], st["phit"]) <= 10 * tu


def test_exact_time_operator_keeps_the_fixed_point(B):
    p = steps(W.viscous_burgers(nx=16, nt=6, T=0.5, nu=0.05).replace(time="bdf2", tprec="exact"), 0.8)
    un = newton.solve(p)
    with B.Solver(p, precision="fp64") as s:
        s.iterate(60000, tol=1e-12, check_every=50)
        u = s.get_host("u")
    assert np.max(np.abs(u - un)) <= 1e-11 * np.max(np.abs(un))


@pytest.mark.parametrize("base,fac", [(W.transport_dg_p1(ncell=32, nt=16, T=0.5), 1.0),
                                      (W.advection_upwind_be(nx=64, nt=32).replace(time="bdf2"), 0.8)],
                         ids=["dg_p1_transport_bdf2", "fd_advection_bdf2"])
def test_ablation_iteration_counts(B, base, fac):
    its = {}
    for tp in ("tridiag", "exact"):
        p = steps(base.replace(tprec=tp), fac)
        with B.Solver(p, precision="fp64") as s:
            its[tp] = s.iterate(60000, tol=1e-8, check_every=10, relative=True)
        _, it_o, _ = opdhg.solve(p, max_iters=60000, tol=1e-8, check_every=10, relative=True)
        assert its[tp] == it_o, (tp, its[tp], it_o)
    assert its["exact"] < its["tridiag"], its

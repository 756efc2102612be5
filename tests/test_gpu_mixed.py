"""Mixed-precision solve (pdhg_solve_mixed): float32 until the tolerance or
float32's rounding floor, then float64 from the widened state.  Its result is the
scheme's solution (Newton time-stepper) to the float64 tolerance, and the float64
phase, warm-started, needs fewer iterations than a float64 solve from scratch."""
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


def _bdf2_viscous():
    """Viscous Burgers, BDF2, the lambda row: tau_u = tau_u0 = tau_phi = sqrt(0.5 / nu_max)."""
    p = W.viscous_burgers(nx=128, nt=8, nu=0.05).replace(time="bdf2", name="viscous_burgers_bdf2_128x8")
    t = float(np.sqrt(0.5 / opdhg.power_estimate(p, iters=60)))
    return p.replace(tau_u=t, tau_u0=t, tau_phi=t)


CASES = [W.advection_upwind_be(nx=256, nt=32, tau=(1.4, 0.1, 0.35, 0.99)),
         _bdf2_viscous(),
         W.burgers_2d(n=256, nt=8).replace(name="transport2d_256x256x8", alpha=0.0, beta=1.0, space="fd_upwind",
                                           lf_a=1.0, c=1.0, tau_u=0.5, tau_phi=0.5, tau_u0=0.1)]


@pytest.mark.parametrize("p", CASES, ids=lambda p: p.name)
def test_mixed_reaches_scheme_solution(B, p):
    s, its = B.solve_mixed(p, tol=1e-10, relative=True, check_every=10, max_iters=50000)
    with s:
        u = s.get_host("u")
        r = s.residual()
        assert s.info()["precision"] == 0                     # the float64 handle
    assert its[0] > 0 and its[1] > 0 and sum(its) < 50000, its
    un = newton.solve(p)
    assert np.max(np.abs(u - un)) <= 1e-8 * np.max(np.abs(un))
    # the float64 phase, warm-started, is shorter than a float64 solve from scratch
    with B.Solver(p, precision="fp64", path="plain") as s64:
        n64 = s64.iterate(50000, tol=1e-10, check_every=10, relative=True)
    assert its[1] < n64, (its, n64)


def test_mixed_uses_the_fused_path_for_2d(B):
    """On a 2D float32-eligible grid the float32 phase runs the fused kernels."""
    p = CASES[-1]
    with B.Solver(p, precision="fp32") as s32:
        assert s32.info()["path"] == "fused"
    s, its = B.solve_mixed(p, tol=1e-6, relative=True, check_every=10)
    with s:
        r = s.residual()
    assert np.all(np.isfinite(r)) and its[0] > 0

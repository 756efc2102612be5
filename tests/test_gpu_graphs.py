"""CUDA-graph replay of the plain path's iteration chunks: the same kernels in the
same order, so the iterates, the residuals and the stopping iteration are
identical with and without graphs."""
import numpy as np
import pytest

import pdhg_workloads as W

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


CASES = [W.advection_upwind_be(tau=(1.4, 0.1, 0.35, 0.99)), W.heat_table1(128, 16),
         W.traffic_dg_p1(ncell=64, nt=8), W.burgers_2d(n=64, nt=8).replace(tau_u=0.15, tau_phi=0.15, tau_u0=0.1)]


@pytest.mark.parametrize("p", CASES, ids=lambda p: p.name)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graphs_change_nothing(B, p, precision):
    out = []
    for graphs in (True, False):
        with B.Solver(p, precision=precision, path="plain") as s:
            s.set_graphs(graphs)
            n1 = s.iterate(205, tol=0.0, check_every=10)          # 20 chunks + 5 single iterations
            n2 = s.iterate(20000, tol=1e-7, check_every=25, relative=True)
            out.append((n1, n2, s.get_host("u"), s.get_host("phi"), s.residual(), s.launches()))
    (a1, a2, au, ap, ar, al), (b1, b2, bu, bp, br, bl) = out
    assert a1 == b1 == 205 and a2 == b2
    assert np.array_equal(au, bu) and np.array_equal(ap, bp)
    assert np.array_equal(ar, br)
    assert al == bl                       # the same launches are counted either way


def test_profiling_bypasses_graphs(B):
    p = W.advection_upwind_be(nx=128, nt=16, tau=(0.5, 0.1, 0.5, 0.99))
    with B.Solver(p, precision="fp64", path="plain") as s:
        s.set_profiling(True)
        s.iterate(30, check_every=10)
        t = s.stage_times()
        assert t["primal"][1] == 30 and t["check"][1] == 3      # one record per stage call


FUSED = [W.burgers_2d(n=256, nt=16).replace(tau_u=0.4, tau_phi=0.4, tau_u0=0.1),
         W.burgers_2d(n=1024, nt=4).replace(tau_u=0.4, tau_phi=0.4, tau_u0=0.1, init="pinned"),
         W.burgers_2d(n=1024, nt=1).replace(tau_u=0.4, tau_phi=0.4, tau_u0=0.1, init="pinned")]


@pytest.mark.parametrize("p", FUSED, ids=lambda p: f"{p.name}_{p.init}")
def test_fused_graphs_change_nothing(B, p):
    """Fused problems of at most 2^23 cell-iterations replay chunks from a graph by
    default (Algorithm 3's two-slice steps among them): iterates, residuals, stopping
    iteration and launch count as launched kernel by kernel, bit for bit."""
    out = []
    for graphs in (True, False):
        with B.Solver(p, precision="fp32", path="fused") as s:
            s.set_graphs(graphs)
            n1 = s.iterate(23, tol=0.0, check_every=5)
            n2 = s.iterate(400, tol=1e-3, check_every=10, relative=True)
            out.append((n1, n2, s.get_host("u"), s.get_host("phi"), s.residual(), s.launches()))
    (a1, a2, au, ap, ar, al), (b1, b2, bu, bp, br, bl) = out
    assert a1 == b1 == 23 and a2 == b2
    assert np.array_equal(au, bu) and np.array_equal(ap, bp)
    assert np.array_equal(ar, br)
    assert al == bl


def test_wait_budget_drops_a_captured_graph(B):
    """The bounded waits' budget is a launch argument of the nx = 1024 rows-C kernel: a
    budget set after a chunk was captured takes effect (the graph is dropped and
    captured again), so a zero budget is reported as PDHG_ERR_TIMEOUT at the next check."""
    p = FUSED[2]
    with B.Solver(p, precision="fp32", path="fused") as s:
        s.iterate(10, tol=0.0, check_every=5)
        s.set_wait_budget(0)
        with pytest.raises(B.PdhgError) as e:
            s.iterate(5, tol=0.0, check_every=5)
        assert e.value.status == -6

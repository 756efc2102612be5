"""Pins of the oracle's Algorithms 2 and 3 (Sec. 3.4, 3.5; CPU only).

The transfer between time meshes is exact on data linear in t; both variants, run
to a tight tolerance, reach the scheme's discrete solution (the Newton
time-stepper); on the traffic example they need about as many iterations as
Table 3 prints."""
import os

import numpy as np
import pytest

import pdhg_workloads as W
from oracle import newton, pdhg, variants

HERE = os.path.dirname(os.path.abspath(__file__))


def _table3():
    rows = {}
    with open(os.path.join(HERE, "golden", "paper_table3_variants.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                t = ln.split()
                rows[t[0]] = [None if v == "-" else int(v) for v in t[1:]]
    return rows


def test_interpolate_t_exact_on_linear_data():
    """u = a + b t at t = l h and phi = c + d t at t = (l+1) h are carried to the
    mesh of half the step exactly (phi's first fine slice, below the first coarse
    time, takes the constant extension)."""
    pc = W.advection_upwind_be(nx=8, nt=4)
    pf = pc.replace(nt=8)
    x = np.linspace(0.0, 1.0, 8)
    a, b, c, d = np.sin(3 * x), np.cos(x), x ** 2, 1.0 - x
    tc = np.arange(pc.nt + 1) * pc.ht
    st = {"u": a + b * tc[:, None], "phi": c + d * tc[1:, None], "lam": x.copy()}
    f = variants.interpolate_t(pc, st, pf)
    tf = np.arange(pf.nt + 1) * pf.ht
    assert np.allclose(f["u"], a + b * tf[:, None], atol=1e-14)
    assert np.allclose(f["phi"][1:], c + d * tf[2:, None], atol=1e-14)
    assert np.allclose(f["phi"][0], st["phi"][0], atol=0)
    assert np.array_equal(f["phit"], f["phi"]) and np.array_equal(f["lamt"], x)


def one_step_taus(p, fac=0.5):
    """tau_u = tau_u0 = tau_phi = sqrt(fac / nu_max) of the two-slice problem."""
    t = float(np.sqrt(fac / pdhg.power_estimate(p.replace(nt=1, T=p.ht), iters=60)))
    return p.replace(tau_u=t, tau_u0=t, tau_phi=t)


@pytest.mark.parametrize("p", [W.advection_upwind_be(nx=16, nt=8), W.traffic_dg_p1(ncell=16, nt=4),
                               W.viscous_burgers(nx=16, nt=6, nu=0.05).replace(time="be"),
                               W.viscous_burgers(nx=16, nt=6, nu=0.05),
                               W.advection_upwind_be(nx=16, nt=8).replace(time="bdf2"),
                               W.burgers_dg_p2(ncell=8, nt=5, T=0.4).replace(c=0.5)],
                         ids=lambda p: f"{p.name}_{p.time}")
def test_one_timestep_reaches_scheme_solution(p):
    """Algorithm 3 to Res <= 1e-12 gives the full scheme's solution slice by slice
    (the one-step problems keep the full problem's inputs), for BE and for BDF2, whose
    steps l >= 1 are BE steps of length 2 h_t / 3 from (4 u^l - u^{l-1}) / 3."""
    p = one_step_taus(p)
    u, counts = variants.one_timestep(p, 1e-12, max_iters_per_step=5000)
    assert max(counts) < 5000, counts
    un = newton.solve(p)
    assert np.max(np.abs(u - un)) <= 1e-9 * max(1.0, np.max(np.abs(un)))
    assert len(counts) == p.nt and min(counts) >= 1


def test_refine_reaches_scheme_solution():
    """Algorithm 2 (three levels, the coarse ones cut short) converges to the
    discrete solution of the finest mesh."""
    p = W.advection_upwind_be(nx=16, nt=8)
    nu = max(pdhg.power_estimate(p.replace(nt=n), iters=60) for n in (2, 4, 8))
    t = float(np.sqrt(0.1 / nu))       # the u^0 / lambda coupling, outside nu, needs the margin
    p = p.replace(tau_u=t, tau_u0=t, tau_phi=t)
    st, counts = variants.refine_in_time(p, 3, [50, 50, 20000], 1e-12)
    un = newton.solve(p)
    assert counts[:2] == [50, 50] and counts[2] < 20000
    assert np.max(np.abs(st["u"] - un)) <= 1e-9


def test_table3_refine_counts_near_paper():
    """Table 3, mesh refinement: 1000 + 1000 iterations on 256 x 8 and 256 x 16, then
    the paper needs 3601 on 256 x 32; this oracle needs 3402 (-5.5%); world time
    5402 vs 5601 and operations 138266 N vs 144833 N.  Pinned within 15%."""
    t3 = _table3()
    p = W.traffic_dg_p1()
    st, counts = variants.refine_in_time(p, 3, [1000, 1000, 20000], 1e-3)
    assert counts[:2] == t3["refine_levels"][:2]
    assert abs(counts[2] - t3["refine_levels"][2]) <= 0.15 * t3["refine_levels"][2], counts
    ops = sum(c * (p.nt // 2 ** (2 - k) + 1) for k, c in enumerate(counts))
    assert abs(ops - t3["refine"][2]) <= 0.15 * t3["refine"][2], ops
    # fewer operations than the vanilla method, as the table shows
    assert ops < t3["vanilla"][2]


def test_table3_one_timestep_count_near_paper():
    """Table 3, one-timestep: the paper needs 8627 iterations over the 32 steps; this
    oracle, with Sec. 3.5's per-time L2 residual, needs 8645 (+0.2%).  (With the
    h_t-weighted space-time norm instead it would stop after 6000.)  Pinned within 5%."""
    t3 = _table3()
    p = W.traffic_dg_p1()
    u, counts = variants.one_timestep(p, 1e-3)
    total = sum(counts)
    assert abs(total - t3["onestep"][0]) <= 0.05 * t3["onestep"][0], total
    assert 2 * total < t3["vanilla"][2]          # the cheapest in operations, as printed
    # the steps shrink as the solution settles: the first step is the hardest
    assert counts[0] == max(counts)

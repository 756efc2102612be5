"""GPU parity of Algorithms 2 and 3 (Sec. 3.4, 3.5) through the C ABI against the
oracle's drivers: iteration counts per level / per step, and the solutions."""
import numpy as np
import pytest

import pdhg_workloads as W
from oracle import newton, pdhg as opdhg, variants

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


def taus(p, fac, probs):
    """tau_u = tau_u0 = tau_phi = sqrt(fac / nu_max), nu_max over the given problems."""
    nu = max(opdhg.power_estimate(q, iters=60) for q in probs)
    t = float(np.sqrt(fac / nu))
    return p.replace(tau_u=t, tau_u0=t, tau_phi=t)


def one_step_taus(p, fac=0.5):
    return taus(p, fac, [p.replace(nt=1, T=p.ht)])


def test_one_step_traffic_counts_and_solution(B):
    """Table 3's one-timestep row on the GPU (float64): the per-step iteration counts
    equal the oracle's (the stopping test may flip by one iteration where a residual
    lands within rounding of the tolerance) and so do the end values."""
    p = W.traffic_dg_p1()
    uo, co = variants.one_timestep(p, 1e-3)
    ug, cg = B.solve_one_step(p, tol=1e-3, precision="fp64")
    ug = ug.cpu().numpy()
    d = np.abs(np.array(cg) - np.array(co))
    assert d.max() <= 1 and d.sum() <= 2, (cg, co)
    tol = 1e-9 if d.sum() == 0 else 1e-3
    assert rel(ug, uo) <= tol


@pytest.mark.parametrize("p", [W.advection_upwind_be(nx=64, nt=8), W.traffic_dg_p1(ncell=64, nt=6),
                               W.viscous_burgers(nx=128, nt=6, nu=0.05).replace(time="be")],
                         ids=lambda p: p.name)
def test_one_step_reaches_scheme_solution(B, p):
    """Algorithm 3 on the GPU to Res <= 1e-12 equals the Newton time-stepper."""
    p = one_step_taus(p)
    ug, cg = B.solve_one_step(p, tol=1e-12, max_iters_per_step=20000, precision="fp64")
    assert max(cg) < 20000
    un = newton.solve(p)
    assert rel(ug.cpu().numpy(), un) <= 1e-9


def test_one_step_fp32_counts_near_fp64(B):
    """float32 one-step on the traffic example stops within 5% of the float64 count."""
    p = W.traffic_dg_p1()
    _, c64 = B.solve_one_step(p, tol=1e-3, precision="fp64")
    u32, c32 = B.solve_one_step(p, tol=1e-3, precision="fp32")
    assert abs(sum(c32) - sum(c64)) <= 0.05 * sum(c64)
    assert np.all(np.isfinite(u32.cpu().numpy()))


@pytest.mark.parametrize("p", [W.viscous_burgers(nx=64, nt=12, T=0.5, nu=0.02),
                               W.burgers_dg_p2(ncell=32, nt=10, T=0.5).replace(c=0.5),
                               W.traffic_dg_p1(ncell=16, nt=4, time="bdf2")],
                         ids=lambda p: p.name)
def test_one_step_bdf2_reaches_scheme_solution(B, p):
    """Algorithm 3 for BDF2 (each step l >= 1 the BE step of length 2 h_t / 3 from
    (4 u^l - u^{l-1}) / 3) on the GPU, float64: the oracle's per-step counts and the
    Newton solution of the BDF2 scheme (1e-9)."""
    t = float(np.sqrt(0.5 / opdhg.power_estimate(p.replace(nt=1, T=p.ht, time="be"), iters=60)))
    p = p.replace(tau_u=t, tau_u0=t, tau_phi=t)
    u, counts = B.solve_one_step(p, tol=1e-11, max_iters_per_step=20000, check_every=10, precision="fp64")
    uo, co = variants.one_timestep(p, 1e-11, max_iters_per_step=20000, check_every=10)
    assert max(abs(a - b) for a, b in zip(counts, co)) <= 10, (counts, co)
    un = newton.solve(p)
    assert np.max(np.abs(u.cpu().numpy() - un)) <= 1e-9 * max(1.0, np.max(np.abs(un)))


@pytest.mark.parametrize("p", [W.viscous_burgers(nx=64, nt=12, T=0.5, nu=0.02),
                               W.viscous_burgers(nx=64, nt=12, T=0.5, nu=0.02).replace(time="bdf2"),
                               W.burgers_2d(n=32, nt=6, cfl=0.5)],
                         ids=lambda p: f"{p.name}_{p.time}")
def test_one_step_mixed_reaches_scheme_solution(B, p):
    """Mixed steps (float32 to its floor, then float64 from the widened state): with a
    per-step tolerance far below float32's floor the float64 phase carries every step to
    the scheme's solution (Newton, 1e-9)."""
    t = float(np.sqrt(0.5 / opdhg.power_estimate(p.replace(nt=1, T=p.ht, time="be"), iters=60)))
    p = p.replace(init="pinned", tau_u=t, tau_u0=t, tau_phi=t)
    um, cm = B.solve_one_step(p, tol=1e-11, max_iters_per_step=20000, check_every=10, precision="mixed")
    assert um.dtype.is_floating_point and um.element_size() == 8
    assert max(cm) < 20000
    un = newton.solve(p)
    assert np.max(np.abs(um.cpu().numpy() - un)) <= 1e-9 * max(1.0, np.max(np.abs(un)))


def test_one_step_fused_float32_phase(B):
    """2D finite differences with nx, ny >= 256: the float32 step handles of Algorithm 3
    run on the fused path (path "auto").  Mixed steps to a per-step tolerance far below
    float32's floor give the same solution as with float32 steps on the plain path (both
    are the scheme's solution, 1e-9), and float32 steps alone stop at the plain path's
    per-step counts (within 10%), both within 1e-4 of that solution (the oracle's steps at
    this tolerance stop 1.8e-5 from it)."""
    p = W.burgers_2d(n=256, nt=4, cfl=0.5)
    t = float(np.sqrt(0.5 / opdhg.power_estimate(p.replace(nt=1, T=p.ht, time="be"), iters=60)))
    p = p.replace(init="pinned", tau_u=t, tau_u0=t, tau_phi=t)
    up, cp = B.solve_one_step(p, tol=1e-11, max_iters_per_step=20000, check_every=10, precision="mixed",
                              path="plain")
    uf, cf = B.solve_one_step(p, tol=1e-11, max_iters_per_step=20000, check_every=10, precision="mixed")
    up, uf = up.cpu().numpy(), uf.cpu().numpy()
    assert np.max(np.abs(uf - up)) <= 1e-9 * max(1.0, np.max(np.abs(up)))
    r0 = 1e-3                            # about 4e-4 of a step's initial Res: above float32's floor
    sp, kp = B.solve_one_step(p, tol=r0, max_iters_per_step=20000, check_every=10, precision="fp32", path="plain")
    sf, kf = B.solve_one_step(p, tol=r0, max_iters_per_step=20000, check_every=10, precision="fp32")
    assert all(abs(a - b) <= max(10, 0.1 * b) for a, b in zip(kf, kp)), (kf, kp)
    assert rel(sf.cpu().numpy(), up) <= 1e-4 and rel(sp.cpu().numpy(), up) <= 1e-4


def test_refine_traffic_counts_and_solution(B):
    """Table 3's mesh-refinement row on the GPU (float64): 1000 + 1000 iterations on
    256 x 8 and 256 x 16, then to Res <= 1e-3 on 256 x 32; counts and the final
    state equal the oracle's driver."""
    p = W.traffic_dg_p1()
    sto, co = variants.refine_in_time(p, 3, [1000, 1000, 20000], 1e-3)
    s, cg = B.solve_refine(p, 3, [1000, 1000, 20000], tol=1e-3, check_every=1, precision="fp64")
    with s:
        ug, phig = s.get_host("u"), s.get_host("phi")
    assert cg[:2] == [1000, 1000] and abs(cg[2] - co[2]) <= 1, (cg, co)
    if cg == co:
        assert rel(ug, sto["u"]) <= 1e-9
        assert rel(phig, sto["phi"]) <= 1e-7


def test_refine_fixed_counts_match_oracle_elementwise(B):
    """Fixed iteration counts (no residual checks) on three levels: the GPU's final
    state equals the oracle's element by element, which pins the transfer of u, phi,
    lambda between meshes."""
    p = W.advection_upwind_be(nx=128, nt=8)
    p = taus(p, 0.1, [p.replace(nt=n) for n in (2, 4, 8)])
    sto, _ = variants.refine_in_time(p, 3, [7, 5, 6], 0.0)
    s, cg = B.solve_refine(p, 3, [7, 5, 6], tol=0.0, check_every=0, precision="fp64", path="plain")
    with s:
        got = {k: s.get_host(k) for k in ("u", "phi", "phit", "lambda", "lambdat")}
    assert cg == [7, 5, 6]
    assert rel(got["u"], sto["u"]) <= 1e-12
    assert rel(got["phi"], sto["phi"]) <= 1e-11
    assert rel(got["phit"], sto["phit"]) <= 1e-11
    assert rel(got["lambda"], sto["lam"]) <= 1e-11


def test_refine_onto_fused_path(B):
    """The finest level on the fused 2D float32 path, the transfer written into its
    current u buffer: after fixed counts the state equals the oracle's (float32)."""
    p = W.burgers_2d(n=256, nt=8).replace(tau_u=0.15, tau_u0=0.1, tau_phi=0.15)
    sto, _ = variants.refine_in_time(p, 2, [4, 3], 0.0)
    s, cg = B.solve_refine(p, 2, [4, 3], tol=0.0, check_every=0, precision="fp32", path="auto")
    with s:
        assert s.info()["path"] == "fused"
        ug = s.get_host("u")
    assert rel(ug, sto["u"]) <= 1e-4

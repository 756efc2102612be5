"""GPU gradient of a terminal objective through the solve (pdhg_solve_gradient)
against the oracle: the sequential discrete adjoint (itself pinned to finite
differences of Newton solves) and, for a fixed number of adjoint iterations,
the oracle's Algorithm 1 on the linearised problem."""
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


def with_taus(p, fac=0.3):
    t = float(np.sqrt(fac / opdhg.power_estimate(p, iters=60)))
    return p.replace(tau_u=t, tau_u0=t, tau_phi=t)


def target_of(p):
    if p.dims == 2:
        x = W.fd_nodes(p.nx, p.lx)
        return 0.5 + 0.4 * np.sin(x[None, :] - 1.0) * np.cos(x[:, None][: p.ny])
    return 0.5 + 0.9 * np.sin(W.fd_nodes(p.nx, p.lx) - 1.0)


CASES = [
    W.viscous_burgers(nx=64, nt=16, T=1.0, nu=0.05).replace(time="be"),
    W.viscous_burgers(nx=64, nt=16, T=1.0, nu=0.05),
    W.advection_upwind_be(nx=64, nt=8).replace(nu=0.02),
    W.burgers_2d(n=16, nt=6).replace(nu=0.02),
]


@pytest.mark.parametrize("p", CASES, ids=lambda p: f"{p.name}_{p.time}")
def test_gradient_equals_sequential_adjoint(B, p):
    p = with_taus(p)
    g = target_of(p)
    u = newton.solve(p)
    _, _, du0, dnu = adjoint.sequential_adjoint(p, u, g)
    loss, du0_g, dnu_g, iters = B.solve_gradient(p, g, tol=1e-12, adj_tol=1e-12, check_every=10)
    assert iters[0] < 100000 and iters[1] < 100000
    assert abs(loss - adjoint.terminal_loss(p, u, g)) <= 1e-10 * max(1.0, loss)
    assert np.max(np.abs(du0_g - du0)) <= 1e-8 * np.max(np.abs(du0))
    assert abs(dnu_g - dnu) <= 1e-8 * max(abs(dnu), 1e-3 * np.max(np.abs(du0)))


def test_gradient_workload_scheme_with_the_exact_time_operator(B):
    """The gradient workload's scheme (viscous Burgers, BDF2, nu = 1e-3) before the shock
    (T = 0.5) at 128 x 64, with the exact time operator (with T_t the BDF2 steps must shrink
    as nt^{-1/2} and Algorithm 1 does not converge at this shape): the float64 GPU gradient
    after 50,000 adjoint iterations (the adjoint's multipliers converge more slowly than the
    forward state: 3e-2 after 2000, 5e-8 after 10,000) equals the sequential adjoint of the
    Newton solution, and the float32 one (forward to float32's floor, 20,000 adjoint
    iterations) stays within 1e-4 of it."""
    p = W.viscous_burgers(nx=128, nt=64, T=0.5, nu=1e-3).replace(tprec="exact")
    p = with_taus(p, fac=0.4)
    g = target_of(p)
    u = newton.solve(p)
    _, _, du0, dnu = adjoint.sequential_adjoint(p, u, g)
    loss, du0_g, dnu_g, iters = B.solve_gradient(p, g, tol=1e-12, adj_tol=0.0, adj_max_iters=50000,
                                                 check_every=100)
    assert iters[0] < 100000 and iters[1] == 50000
    assert np.max(np.abs(du0_g - du0)) <= 1e-9 * np.max(np.abs(du0))
    assert abs(dnu_g - dnu) <= 1e-9 * max(abs(dnu), 1e-3 * np.max(np.abs(du0)))
    loss32, du0_32, dnu_32, _ = B.solve_gradient(p, g, tol=1e-5, max_iters=20000, adj_tol=0.0,
                                                 adj_max_iters=20000, check_every=100, precision="fp32")
    assert np.max(np.abs(du0_32 - du0)) <= 1e-4 * np.max(np.abs(du0))
    assert abs(dnu_32 - dnu) <= 1e-4 * max(abs(dnu), np.max(np.abs(du0)))


@pytest.mark.parametrize("p", CASES[:2] + CASES[3:], ids=lambda p: f"{p.name}_{p.time}")
def test_adjoint_fixed_iterates(B, p):
    """25 adjoint iterations after a converged forward solve: lambda (hence dLoss/du0)
    and dLoss/dnu equal the oracle's linearised Algorithm 1 after 25 iterations."""
    p = with_taus(p)
    g = target_of(p)
    u = newton.solve(p)
    st = adjoint.linearised_initial_state(p)
    for _ in range(25):
        adjoint.linearised_step(p, u, st, g)
    du0_o, dnu_o = adjoint.pdhg_gradient(p, {"u": u, "phi": st["phi"], "lam": st["lam"]})
    _, du0_g, dnu_g, iters = B.solve_gradient(p, g, tol=1e-13, adj_tol=0.0, adj_max_iters=25, check_every=10)
    assert iters[1] == 25
    assert np.max(np.abs(du0_g - du0_o)) <= 1e-9 * np.max(np.abs(du0_o))
    assert abs(dnu_g - dnu_o) <= 1e-9 * max(abs(dnu_o), 1e-3)


@pytest.mark.parametrize("p", CASES[:2], ids=lambda p: f"{p.name}_{p.time}")
def test_gradient_float32_against_float64_oracle(B, p):
    """The gradient computed in float32 (forward and adjoint Algorithm 1 in float32, run for a
    fixed budget past float32's rounding floor) against the oracle's float64 sequential
    adjoint: dLoss/du0 to 1e-4 of its largest value and dLoss/dnu to 1e-4 of its size.
    The bound comes from the float32 floors of the two solves (relative Res of a few 1e-6
    each, see the fused converged-parity test) times the conditioning of the linearised
    problem, which is O(10) here."""
    p = with_taus(p)
    g = target_of(p)
    u = newton.solve(p)
    _, _, du0, dnu = adjoint.sequential_adjoint(p, u, g)
    loss, du0_g, dnu_g, iters = B.solve_gradient(p, g, tol=1e-9, max_iters=20000, adj_tol=1e-9,
                                                 adj_max_iters=20000, check_every=50, precision="fp32")
    assert abs(loss - adjoint.terminal_loss(p, u, g)) <= 1e-5 * max(1.0, loss)
    assert np.max(np.abs(du0_g - du0)) <= 1e-4 * np.max(np.abs(du0)), np.max(np.abs(du0_g - du0)) / np.max(np.abs(du0))
    assert abs(dnu_g - dnu) <= 1e-4 * max(abs(dnu), 1e-3 * np.max(np.abs(du0))), (dnu_g, dnu)


def test_autograd_with_u0_on_the_device(B):
    """TerminalLoss with u0 a CUDA tensor: u0 goes to the library as a device pointer
    (PDHG_FLAG_U0_ON_DEVICE, no host copy); loss and gradient equal those of the host path,
    and the Lax-Friedrichs constant taken from the device scan of u0 equals the host's."""
    import torch
    p = with_taus(W.viscous_burgers(nx=64, nt=16, T=1.0, nu=0.05).replace(time="be", lf_a=0.0))
    g = target_of(p)
    TL = B.terminal_loss_fn()
    opts = {"tol": 1e-12, "adj_tol": 1e-12, "check_every": 10}
    out = {}
    for where in ("cpu", "cuda"):
        u0 = torch.tensor(p.u0, dtype=torch.float64, device=where, requires_grad=True)
        nu = torch.tensor(p.nu, dtype=torch.float64, requires_grad=True)
        loss = TL.apply(u0, nu, p, g, opts)
        loss.backward()
        out[where] = (float(loss), u0.grad.detach().cpu().numpy(), float(nu.grad))
        assert u0.grad.device == u0.device
    # both solves run to Res 1e-12: equal to that level (bitwise when lf_a rounds alike)
    assert abs(out["cpu"][0] - out["cuda"][0]) <= 1e-10 * max(1.0, abs(out["cpu"][0]))
    assert np.max(np.abs(out["cpu"][1] - out["cuda"][1])) <= 1e-9 * np.max(np.abs(out["cpu"][1]))
    assert abs(out["cpu"][2] - out["cuda"][2]) <= 1e-9 * max(1.0, abs(out["cpu"][2]))


def test_autograd_function_matches_gpu_finite_differences(B):
    """TerminalLoss.backward returns the gradient; the objective's own central
    differences (GPU forward solves at u0 +- eps v) agree with <dLoss/du0, v>."""
    import torch
    p = with_taus(W.viscous_burgers(nx=64, nt=16, T=1.0, nu=0.05).replace(time="be"))
    g = target_of(p)
    TL = B.terminal_loss_fn()
    opts = {"tol": 1e-12, "adj_tol": 1e-12, "check_every": 10}
    u0 = torch.tensor(p.u0, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(p.nu, dtype=torch.float64, requires_grad=True)
    loss = TL.apply(u0, nu, p, g, opts)
    loss.backward()
    v = np.random.default_rng(3).standard_normal(p.nx)
    eps = 1e-5
    lp = B.solve_gradient(p.replace(u0=p.u0 + eps * v), g, **opts)[0]
    lm = B.solve_gradient(p.replace(u0=p.u0 - eps * v), g, **opts)[0]
    assert abs((lp - lm) / (2 * eps) - float(u0.grad.numpy() @ v)) <= 1e-6 * max(1.0, abs(lp - lm) / (2 * eps))
    assert nu.grad is not None and np.isfinite(float(nu.grad))


def test_gradient_rejects_unsupported(B):
    p = W.traffic_dg_p1(ncell=16, nt=4)
    with pytest.raises(B.PdhgError) as e:
        B.solve_gradient(p, p.u0)
    assert e.value.status == -7

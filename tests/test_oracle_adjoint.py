"""Pins of the oracle's gradient of a terminal objective (CPU only).

The sequential discrete adjoint (backward in time, Jacobian blocks from finite
differences of D) equals central differences of the objective computed from
Newton solves at perturbed u0 and nu; Algorithm 1 on the problem linearised at
the solution converges to the same adjoint, while Algorithm 1 on the nonlinear
objective-augmented problem does not."""
import numpy as np
import pytest

import pdhg_workloads as W
from oracle import adjoint, newton, pdhg


def problem(time):
    p = W.viscous_burgers(nx=32, nt=16, T=1.0, nu=0.05).replace(time=time)
    t = float(np.sqrt(0.3 / pdhg.power_estimate(p, iters=60)))
    return p.replace(tau_u=t, tau_u0=t, tau_phi=t)


def target(p):
    return 0.5 + 0.9 * np.sin(W.fd_nodes(p.nx, p.lx) - 1.0)


@pytest.mark.parametrize("time", ["be", "bdf2"])
def test_sequential_adjoint_equals_finite_differences(time):
    p = problem(time)
    g = target(p)
    u = newton.solve(p)
    _, _, du0, dnu = adjoint.sequential_adjoint(p, u, g)
    rng = np.random.default_rng(1)
    eps = 1e-5
    for _ in range(2):
        v = rng.standard_normal(p.nx)
        lp = adjoint.terminal_loss(p, newton.solve(p.replace(u0=p.u0 + eps * v)), g)
        lm = adjoint.terminal_loss(p, newton.solve(p.replace(u0=p.u0 - eps * v)), g)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - du0 @ v) <= 1e-7 * max(1.0, abs(fd))
    qp, qm = p.replace(nu=p.nu + eps), p.replace(nu=p.nu - eps)
    fd = (adjoint.terminal_loss(qp, newton.solve(qp), g) - adjoint.terminal_loss(qm, newton.solve(qm), g)) / (2 * eps)
    assert abs(fd - dnu) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("time", ["be", "bdf2"])
def test_linearised_pdhg_converges_to_adjoint(time):
    p = problem(time)
    g = target(p)
    u = newton.solve(p)
    phi, lam, du0, dnu = adjoint.sequential_adjoint(p, u, g)
    st = adjoint.linearised_initial_state(p)
    for _ in range(6000):
        adjoint.linearised_step(p, u, st, g)
    assert np.max(np.abs(st["lam"] - lam)) <= 1e-9 * np.max(np.abs(lam))
    assert np.max(np.abs(st["phi"] - phi)) <= 1e-9 * np.max(np.abs(phi))
    assert np.max(np.abs(st["u"])) <= 1e-9
    # the gradient read off the state
    du0_p, dnu_p = adjoint.pdhg_gradient(p, {"u": u, "phi": st["phi"], "lam": st["lam"]})
    assert np.max(np.abs(du0_p - du0)) <= 1e-9 * np.max(np.abs(du0))
    assert abs(dnu_p - dnu) <= 1e-9 * abs(dnu)


def test_objective_augmented_nonlinear_pdhg_does_not_converge():
    """Why the adjoint runs on the linearised problem: with phi* != 0 the
    objective-augmented Lagrangian is not convex in u and Algorithm 1 drifts away
    from the solution even when started there."""
    p = problem("be")
    g = target(p)
    st, it, _ = pdhg.solve(p, max_iters=20000, tol=1e-10, check_every=100)
    assert it < 20000
    u = st["u"].copy()
    st2, it2, _ = pdhg.solve(p, max_iters=3000, tol=1e-10, check_every=100, state=st, target=g)
    assert it2 == 3000 and np.max(np.abs(st2["u"] - u)) > 1e-2

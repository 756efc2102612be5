"""Pins of the oracle's preconditioner K_d (CPU only)."""
import numpy as np
import pytest

import pdhg_workloads as W
from oracle import precond, spacetime


@pytest.mark.parametrize("p", [
    W.advection_upwind_be(nx=8, nt=5),
    W.heat_table1(8, 4),
    W.burgers_2d(n=6, nt=3),
    W.burgers_dg_p2(ncell=6, nt=4),
    W.viscous_burgers(nx=7, nt=3),
    W.transport_dg_p1(ncell=6, nt=4),
    W.advection_upwind_be(nx=7, nt=4).replace(nu=0.1),         # odd nx (the Bluestein path's lengths)
    W.viscous_burgers(nx=10, nt=3),
], ids=lambda p: p.name)
def test_kd_inverse_equals_dense_solve(p):
    """FFT-in-x + Thomas-in-t equals a dense solve of K_d assembled in real space from
    stencils (not from Fourier symbols); K_d is symmetric positive definite."""
    rng = np.random.default_rng(11)
    r = rng.standard_normal((p.nt,) + p.slice_shape)
    Kd = precond.dense_Kd(p)
    zd = np.linalg.solve(Kd, r.ravel()).reshape(r.shape)
    z = precond.kd_inverse(p, r)
    assert np.max(np.abs(z - zd)) <= 1e-12 * np.max(np.abs(zd))
    assert np.max(np.abs(Kd - Kd.T)) == 0.0
    assert np.min(np.linalg.eigvalsh(Kd)) > 0.0


def test_Tt_is_backward_euler_gram_matrix():
    """T_t / h_t^2 = A_t A_t^T with A_t the backward-Euler difference acting on
    u^1..u^nt (u^0 held fixed): the paper's H-norm with phi^{nt} = 0."""
    p = W.advection_upwind_be(nx=4, nt=6).replace(beta=0.0)
    n = p.ndof
    u = np.zeros((p.nt + 1,) + p.slice_shape)
    A = np.zeros((p.nt * n, p.nt * n))
    for k in range(p.nt * n):
        v = np.zeros_like(u)
        v.reshape(-1)[n + k] = 1.0
        A[:, k] = spacetime.jvp(p, u, v).ravel()
    T = np.kron(precond.dense_Tt(p.nt), np.eye(n)) / p.ht ** 2
    assert np.allclose(A @ A.T, T, rtol=1e-13, atol=1e-13 * np.max(T))


def test_fd_symbol_equals_upwind_gram():
    """For FD the symbol kappa = c^2 L(theta) equals |S(theta)|^2 of the upwind operator
    of c u_x, the construction the DG preconditioner generalises."""
    p = W.advection_upwind_be(nx=16, nt=2).replace(c=1.7)
    k = np.arange(9)
    theta = 2 * np.pi * k / 16
    S = 1.7 * (1 - np.exp(-1j * theta)) / p.hx
    assert np.allclose(np.abs(S) ** 2, precond.fd_kappa(p), rtol=1e-13)


def test_dg_symbol_blocks_hermitian_psd():
    p = W.burgers_dg_p2(ncell=8, nt=2)
    K = precond.dg_Kx(p)
    assert np.allclose(K, np.conj(np.swapaxes(K, -1, -2)), atol=1e-12)
    assert np.min(np.linalg.eigvalsh(K)) > -1e-9 * np.max(np.abs(K))


def test_thomas_kappa_zero_prefix_sums():
    """For kappa = 0 every pivot is 1, so z is a suffix sum of prefix sums of h_t^2 r."""
    nt = 7
    r = np.random.default_rng(1).standard_normal((nt, 1)) + 0j
    z = precond.thomas_t(r, np.zeros(1), 0.5)
    y = np.cumsum(0.25 * r[:, 0])
    zz = np.cumsum(y[::-1])[::-1]
    assert np.allclose(z[:, 0], zz, atol=1e-14)


def test_float32_preconditioner_keeps_the_fixed_point(monkeypatch):
    """The reading behind the float32 preconditioner of the mixed solve's float64 phase
    (and of the float32 t-recurrence): K_d^{-1} only shapes the iteration.  Algorithm 1
    with K_d^{-1} applied to a float32-rounded residual and its result rounded to float32
    again reaches the same discrete solution (Newton) as the exact preconditioner, to the
    float64 tolerance, in about the same number of iterations."""
    from oracle import newton, pdhg as opdhg
    p = W.advection_upwind_be(nx=64, nt=16, tau=(1.4, 0.1, 0.35, 0.99))
    _, n_exact, _ = opdhg.solve(p, tol=1e-10, relative=True, check_every=10, max_iters=20000)
    exact = precond.kd_inverse

    def kd_inverse_f32(q, r):
        return exact(q, np.asarray(r, np.float32).astype(np.float64)).astype(np.float32).astype(np.float64)

    monkeypatch.setattr(precond, "kd_inverse", kd_inverse_f32)
    st, n32, _ = opdhg.solve(p, tol=1e-10, relative=True, check_every=10, max_iters=20000)
    un = newton.solve(p)
    assert n32 < 20000
    assert np.max(np.abs(st["u"] - un)) <= 1e-8 * np.max(np.abs(un))
    assert abs(n32 - n_exact) <= 0.05 * n_exact + 10


# ---------------------------------------------------------------------------
# ablation: the exact time operator h_t^2 D_t D_t^T in place of T_t
# ---------------------------------------------------------------------------

def test_exact_time_operator_is_Tt_for_backward_euler():
    """For BE with u^0 held fixed, h_t^2 D_t D_t^T is the tridiagonal T_t of the reading."""
    p = W.advection_upwind_be(nx=8, nt=7)
    assert np.array_equal(precond.exact_Tt(p), precond.dense_Tt(p.nt))


def test_exact_time_operator_bdf2_interior_rows_are_the_symbol_autocorrelation():
    """Away from the first rows, h_t^2 D_t D_t^T for BDF2 is the Toeplitz matrix whose
    coefficients are those of |a(w)|^2, a(w) = 3/2 - 2 e^{-iw} + 1/2 e^{-2iw} the Fourier
    symbol of the BDF2 difference (Sec. 3.1): computed here by sampling |a|^2 and an
    inverse FFT.  The matrix is symmetric positive definite and pentadiagonal."""
    p = W.advection_upwind_be(nx=8, nt=12).replace(time="bdf2")
    K = precond.exact_Tt(p)
    n = 64
    w = 2.0 * np.pi * np.arange(n) / n
    a = 1.5 - 2.0 * np.exp(-1j * w) + 0.5 * np.exp(-2j * w)
    c = np.fft.ifft(np.abs(a) ** 2).real                 # c[k] = coefficient of e^{ikw}
    for l in range(3, p.nt - 3):
        for d in range(-3, 4):
            assert abs(K[l, l + d] - c[d % n]) < 1e-13, (l, d)
    assert np.allclose(K, K.T, atol=0.0) and np.all(np.linalg.eigvalsh(K) > 0)
    assert np.all(np.triu(K, 3) == 0.0)


@pytest.mark.parametrize("p", [
    W.advection_upwind_be(nx=10, nt=6).replace(time="bdf2", tprec="exact"),
    W.burgers_2d(n=4, nt=5).replace(time="bdf2", tprec="exact", ny=6, ly=1.5 * np.pi,
                                      u0=W.burgers_2d(n=4).u0[:1].repeat(6, 0)),
    W.burgers_dg_p2(ncell=6, nt=5).replace(c=0.7, tprec="exact"),
    W.transport_dg_p1(ncell=6, nt=5).replace(tprec="exact"),
], ids=["fd1d", "fd2d", "dgp2", "dgp1"])
def test_exact_kd_inverse_equals_dense_solve(p):
    """K_d^{-1} with the exact time operator (per-mode dense solves after the x/y FFTs)
    equals a dense solve of the assembled K_d (stencils in real space) to 1e-12."""
    rng = np.random.default_rng(3)
    r = rng.standard_normal((p.nt,) + p.slice_shape)
    z = precond.kd_inverse(p, r)
    zd = np.linalg.solve(precond.dense_Kd(p), r.ravel()).reshape(r.shape)
    assert np.max(np.abs(z - zd)) <= 1e-12 * np.max(np.abs(zd))


def test_bdf2_preconditioned_norm_with_tt_and_exact_operator():
    """What the T_t reading costs BDF2: the largest eigenvalue of the preconditioned
    operator (power estimate) grows as 2.5 + nt/4 with T_t, while the exact time operator
    keeps it at the BE value (about 2) for every nt -- the reason the exact operator cuts
    BDF2 iteration counts and the T_t step sizes must shrink as nt^{-1/2}."""
    from oracle import pdhg as opdhg
    for nt in (16, 32, 64):
        p = W.advection_upwind_be(nx=32, nt=nt).replace(time="bdf2", T=nt * 2 * (2 * np.pi / 32))
        tt = opdhg.power_estimate(p, iters=40)
        ex = opdhg.power_estimate(p.replace(tprec="exact"), iters=40)
        be = opdhg.power_estimate(p.replace(time="be"), iters=40)
        assert abs(tt - (2.5 + nt / 4)) <= 0.02 * (2.5 + nt / 4), (nt, tt)
        assert abs(ex - be) <= 0.05 * be and be < 2.0, (nt, ex, be)


def test_exact_operator_converges_viscous_burgers_bdf2():
    """Viscous Burgers, BDF2 (the gradient workload's scheme, 64 x 32, nu = 1e-3, T = 0.5),
    steps from the power estimate of each preconditioner: with the exact time operator
    Algorithm 1 reaches relative Res 1e-8 within 1000 iterations; with T_t (admissible
    steps smaller by sqrt(2.5 + nt/4) / sqrt(2)) it is still above 1e-2 after 1500."""
    from oracle import pdhg as opdhg
    base = W.viscous_burgers(nx=64, nt=32, T=0.5, nu=1e-3)
    rel = {}
    for tprec in ("exact", "tridiag"):
        p = base.replace(tprec=tprec)
        t = float(np.sqrt(0.5 / opdhg.power_estimate(p, iters=30)))
        q = p.replace(tau_u=t, tau_phi=t, tau_u0=t)
        r0 = opdhg.residual_norms(q, opdhg.initial_state(q))[0]
        st, its, _ = opdhg.solve(q, max_iters=1500, tol=1e-8, check_every=100, relative=True)
        r = opdhg.residual_norms(q, st)
        rel[tprec] = (its, max(r[0], r[1]) / r0)
    assert rel["exact"][0] <= 1000 and rel["exact"][1] <= 1e-8, rel
    assert rel["tridiag"][1] > 1e-2, rel

"""The C-ABI library loads on a machine without a GPU and exports every symbol
that include/pdhg.h declares; host-side validation needs no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import pdhg_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2207_07234_gb300 import binding
    return binding.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "pdhg.h")).read()
    return sorted(set(re.findall(r"\b(pdhg_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    from paper_2207_07234_gb300 import binding
    names = declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS) == names


def _size(p, **kw):
    from paper_2207_07234_gb300 import binding
    return binding.workspace_size(p, **kw)


def test_workspace_size_and_validation(lib):
    from paper_2207_07234_gb300 import binding
    p = W.burgers_2d(n=64, nt=8)
    n32 = _size(p, precision="fp32", path="plain")
    n64 = _size(p, precision="fp64", path="plain")
    cells = 64 * 64 * 8
    assert n32 >= 4 * cells * 4 and n64 >= 4 * cells * 8
    with pytest.raises(binding.PdhgError) as e:
        _size(W.burgers_dg_p2(ncell=96, nt=4))
    assert e.value.status == -7                                   # UNSUPPORTED: DG nx not a power of two
    with pytest.raises(binding.PdhgError) as e:
        _size(W.advection_upwind_be(nx=64, nt=4).replace(tau_u=-1.0))
    assert e.value.status == -1                                   # INVALID_ARG
    with pytest.raises(binding.PdhgError) as e:
        _size(W.burgers_dg_p2(ncell=64, nt=4).replace(nu=0.1))
    assert e.value.status == -7
    assert "power of two" in lib.pdhg_last_error().decode() or lib.pdhg_last_error()


def test_create_rejects_without_device_work(lib):
    """Argument errors are reported before any device work: NULL workspace,
    misaligned workspace, too small a workspace."""
    from paper_2207_07234_gb300 import binding
    p = W.advection_upwind_be(nx=16, nt=4)
    prob, grid, scheme, keep = binding.structs(p, "fp64", "plain")
    h = ctypes.c_void_p()
    st = lib.pdhg_create(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme), None, 0, None,
                         ctypes.byref(h))
    assert st == -1
    st = lib.pdhg_create(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                         ctypes.c_void_p(256), 16, None, ctypes.byref(h))
    assert st == -2
    st = lib.pdhg_create(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                         ctypes.c_void_p(257), 1 << 30, None, ctypes.byref(h))
    assert st == -1
    bad = p.replace(u0=np.full_like(p.u0, np.nan))
    prob, grid, scheme, keep = binding.structs(bad, "fp64", "plain")
    st = lib.pdhg_create(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                         ctypes.c_void_p(256 * 1024), 1 << 30, None, ctypes.byref(h))
    assert st == -1 and "non-finite" in lib.pdhg_last_error().decode()


def test_batch_validation_without_device_work(lib):
    """Batch sizes add up the instances; 2D, mixed precision and the fused path are
    rejected before any device work."""
    from paper_2207_07234_gb300 import binding
    probs = [W.advection_upwind_be(nx=64, nt=8), W.traffic_dg_p1(ncell=32, nt=4)]

    def arrays(ps, precisions, paths):
        parts = [binding.structs(p, pr, pa) for p, pr, pa in zip(ps, precisions, paths)]
        n = len(ps)
        return (n, (binding.pdhg_problem * n)(*[x[0] for x in parts]), (binding.pdhg_grid * n)(*[x[1] for x in parts]),
                (binding.pdhg_scheme * n)(*[x[2] for x in parts]), parts)

    n, P, G, S, keep = arrays(probs, ["fp32", "fp32"], ["auto", "auto"])
    total = ctypes.c_size_t(0)
    assert lib.pdhg_batch_workspace_size(n, P, G, S, ctypes.byref(total)) == 0
    parts = sum(binding.workspace_size(p, "fp32", "plain") for p in probs)
    assert total.value > parts
    for bad in ([probs[0], W.burgers_2d(n=16, nt=4)], ):
        n, P, G, S, keep = arrays(bad, ["fp32", "fp32"], ["auto", "auto"])
        assert lib.pdhg_batch_workspace_size(n, P, G, S, ctypes.byref(total)) == -7
    n, P, G, S, keep = arrays(probs, ["fp32", "fp64"], ["auto", "auto"])
    assert lib.pdhg_batch_workspace_size(n, P, G, S, ctypes.byref(total)) == -1
    n, P, G, S, keep = arrays(probs, ["fp32", "fp32"], ["auto", "fused"])
    assert lib.pdhg_batch_workspace_size(n, P, G, S, ctypes.byref(total)) == -7


def test_non_power_of_two_nx_accepted_only_for_1d_fd(lib):
    """nx outside the powers of two: 1D finite differences up to 4096 (Bluestein
    x-transform); DG, 2D and longer 1D lines are rejected before any device work."""
    from paper_2207_07234_gb300 import binding
    assert binding.workspace_size(W.advection_upwind_be(nx=1000, nt=8), "fp64") > 0
    assert binding.workspace_size(W.advection_upwind_be(nx=257, nt=8), "fp32") > 0
    for bad in (W.advection_upwind_be(nx=4097, nt=4), W.traffic_dg_p1(ncell=100, nt=4),
                W.burgers_2d(n=16, nt=4).replace(nx=24, u0=np.zeros((16, 24)))):
        with pytest.raises(binding.PdhgError) as e:
            binding.workspace_size(bad, "fp64")
        assert e.value.status == -7


def test_mixed_workspace_and_wait_budget_without_device_work(lib):
    """The mixed solve's workspace holds the float32 handle and the float64 one; for
    finite differences (nx a power of two) the float64 part adds float32 copies of the
    preconditioner's tables (x/y twiddles, theta), for DG it does not.  A null handle is
    rejected by pdhg_set_wait_budget."""
    from paper_2207_07234_gb300 import binding
    for p, pre32 in ((W.burgers_2d(n=64, nt=8), True), (W.traffic_dg_p1(ncell=32, nt=4), False)):
        prob, grid, scheme, keep = binding.structs(p, "fp64", "plain")
        nb = ctypes.c_size_t(0)
        assert lib.pdhg_mixed_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                             ctypes.byref(nb)) == 0
        n32 = _size(p, precision="fp32", path="auto")
        n64 = _size(p, precision="fp64", path="plain")
        extra = nb.value - (-(-n32 // 256) * 256 + n64)
        if pre32:
            nkx, ny = p.nx // 2 + 1, p.ny
            tables = nkx * 8 + ny * 8 + nkx * ny * 4           # twx, twy (float2), theta (float)
            assert tables <= extra <= tables + 3 * 256
        else:
            assert extra == 0
    assert lib.pdhg_set_wait_budget(None, ctypes.c_uint64(0)) == -1
    n = ctypes.c_int64(0)
    assert lib.pdhg_residual_history(None, None, ctypes.c_int64(0), ctypes.byref(n), 0) == -1


def test_mixed_steps_flag_only_for_the_one_step_solve(lib):
    """PDHG_FLAG_MIXED_STEPS is accepted by the one-step workspace query (a float32 and a
    float64 handle per step length: more than the float64 one-step workspace) and
    rejected, before any device work, by the entry points it does not apply to."""
    from paper_2207_07234_gb300 import binding
    p = W.burgers_2d(n=64, nt=8)
    for time in ("be", "bdf2"):
        q = p.replace(init="pinned", time=time)
        prob, grid, scheme, keep = binding.structs(q, "fp64", "plain")
        n64 = ctypes.c_size_t(0)
        assert lib.pdhg_one_step_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                                ctypes.byref(n64)) == 0
        scheme.flags |= binding.FLAG_MIXED_STEPS
        nm = ctypes.c_size_t(0)
        assert lib.pdhg_one_step_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                                ctypes.byref(nm)) == 0
        assert nm.value > n64.value
        nb = ctypes.c_size_t(0)
        assert lib.pdhg_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                       ctypes.byref(nb)) == -1

"""pdhg_residual_noalloc: residual norms without a workspace or any allocation.

Callers that cannot allocate device memory (they may only use buffers they
were handed) cannot give pdhg_create() its workspace; this entry point keeps
its reduction scratch in a fixed array inside the library.  The test calls it
through the C ABI on a state produced by the handle-based path and compares
its output with pdhg_residual() on that handle, twice in a row (the scratch is
shared and keeps the previous call's contents).  This file is collected last.
"""
import ctypes

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
    lib = binding.load()
    fn = lib.pdhg_residual_noalloc
    fn.argtypes = [ctypes.POINTER(binding.pdhg_problem), ctypes.POINTER(binding.pdhg_grid),
                   ctypes.POINTER(binding.pdhg_scheme)] + [ctypes.c_void_p] * 5 + \
                  [ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return binding


def _noalloc(B, p, precision, s, lf_a):
    import torch
    prob, grid, scheme, keep = B.structs(p.replace(lf_a=lf_a), precision, "plain")
    u, phi = s.get("u"), s.get("phi")
    lam = s.get("lambda") if p.init == "lambda" else None       # pinned: lambda may be NULL
    u0 = torch.as_tensor(p.u0, dtype=s.dtype, device=s.device).contiguous()
    gam = (torch.as_tensor(p.gamma_half, dtype=s.dtype, device=s.device).contiguous()
           if p.gamma_half is not None else None)
    out = (ctypes.c_double * 4)()
    stream = torch.cuda.current_stream()
    st = B.load().pdhg_residual_noalloc(
        ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
        ctypes.c_void_p(lam.data_ptr() if lam is not None else None),
        ctypes.c_void_p(u0.data_ptr()), ctypes.c_void_p(gam.data_ptr() if gam is not None else None),
        out, ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, B.load().pdhg_last_error().decode()
    return np.array(list(out))


CASES = ["burgers2d_fp32", "heat_fp64", "dg_fp64", "heat_pinned_fp64", "dg_p1_fp64", "viscous_bdf2_fp32"]


@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_handle_residual_twice(B, case):
    if case == "burgers2d_fp32":
        p = W.burgers_2d(n=64, nt=8).replace(tau_u=0.4, tau_phi=0.4, tau_u0=0.1)
        prec, lf_a = "fp32", p.lf_a
    elif case == "heat_fp64":                    # variable-coefficient Laplacian: gamma_half given
        p = W.heat_table1(64, 16)
        prec, lf_a = "fp64", 1.0
    elif case == "heat_pinned_fp64":             # u^0 pinned: lambda passed as NULL
        p = W.heat_table1(64, 16, init="pinned")
        prec, lf_a = "fp64", 1.0
    elif case == "dg_p1_fp64":                   # the paper's nodal DG P1 (upwind), traffic flux
        p = W.traffic_dg_p1(ncell=64, nt=8)
        prec, lf_a = "fp64", 1.0
    elif case == "viscous_bdf2_fp32":            # 1D FD Lax-Friedrichs + viscosity, BDF2
        p = W.viscous_burgers(nx=256, nt=12, T=0.5, nu=0.01).replace(tau_u=0.3, tau_phi=0.3, tau_u0=0.1)
        prec, lf_a = "fp32", p.lf_a
    else:
        p = W.burgers_dg_p2(ncell=64, nt=6, T=0.5).replace(c=0.5, tau_u=0.1, tau_phi=0.1, tau_u0=0.1)
        prec, lf_a = "fp64", p.lf_a
    with B.Solver(p, precision=prec, path="plain") as s:
        s.iterate(7)
        ref = s.residual()
        first = _noalloc(B, p, prec, s, lf_a)
        s.iterate(3)                      # change the state, then call twice more
        ref2 = s.residual()
        second = _noalloc(B, p, prec, s, lf_a)
        third = _noalloc(B, p, prec, s, lf_a)
    # the same kernels on the same state: equal up to the order of the float64 sums
    tol = 1e-12
    for got, want in ((first, ref), (second, ref2), (third, ref2)):
        assert np.allclose(got[:3], want[:3], rtol=tol, atol=0.0)
        assert abs(got[3] - want[3]) <= tol * max(abs(want[3]), 1e-300)


def test_noalloc_rejects_too_large(B):
    import torch
    p = W.burgers_2d(n=1024, nt=2000)      # 32 * 2001 partial blocks > 43685: rejected before any launch
    prob, grid, scheme, keep = B.structs(p, "fp32", "plain")
    out = (ctypes.c_double * 4)()
    dummy = torch.zeros(4, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    st = B.load().pdhg_residual_noalloc(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                        ptr, ptr, ptr, ptr, None, out, None)
    assert st == -7 and "too large" in B.load().pdhg_last_error().decode()


@pytest.mark.parametrize("what", ["nx_1d", "nx_2d", "nu_negative", "nx_not_pow2_2d"])
def test_noalloc_rejects_grids_outside_the_limits(B, what):
    """Grids that pdhg_create rejects are rejected here too, before any device work:
    sizes beyond nx <= 8192 / ny <= 2048 (whose slices would overflow the kernels'
    32-bit per-slice indices), a negative viscosity, a 2D nx that is not a power of two."""
    import torch
    if what == "nx_1d":
        p = W.advection_upwind_be(nx=64, nt=2).replace(nx=1 << 20, u0=np.zeros(1 << 20))
    elif what == "nx_2d":
        q = W.burgers_2d(n=64, nt=2)
        p = q.replace(nx=1 << 16, ny=1 << 16, u0=np.zeros((1, 1)))
    elif what == "nu_negative":
        p = W.viscous_burgers(nx=64, nt=2, T=0.5, nu=0.01).replace(nu=-0.01)
    else:
        q = W.burgers_2d(n=64, nt=2)
        p = q.replace(nx=96, u0=np.zeros((64, 96)))
    prob, grid, scheme, keep = B.structs(p, "fp32", "plain")
    out = (ctypes.c_double * 4)()
    dummy = torch.zeros(4, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    st = B.load().pdhg_residual_noalloc(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                        ptr, ptr, ptr, ptr, None, out, None)
    assert st in (-1, -7), (st, B.load().pdhg_last_error().decode())

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
    lam = s.get("lambda")
    u0 = torch.as_tensor(p.u0, dtype=s.dtype, device=s.device).contiguous()
    gam = (torch.as_tensor(p.gamma_half, dtype=s.dtype, device=s.device).contiguous()
           if p.gamma_half is not None else None)
    out = (ctypes.c_double * 4)()
    stream = torch.cuda.current_stream()
    st = B.load().pdhg_residual_noalloc(
        ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
        ctypes.c_void_p(u0.data_ptr()), ctypes.c_void_p(gam.data_ptr() if gam is not None else None),
        out, ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, B.load().pdhg_last_error().decode()
    return np.array(list(out))


@pytest.mark.parametrize("case", ["burgers2d_fp32", "heat_fp64", "dg_fp64"])
def test_noalloc_matches_handle_residual_twice(B, case):
    if case == "burgers2d_fp32":
        p = W.burgers_2d(n=64, nt=8).replace(tau_u=0.4, tau_phi=0.4, tau_u0=0.1)
        prec, lf_a = "fp32", p.lf_a
    elif case == "heat_fp64":
        p = W.heat_table1(64, 16)
        prec, lf_a = "fp64", 1.0
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
    for got, want in ((first, ref), (second, ref2), (third, ref2)):
        assert np.allclose(got[:3], want[:3], rtol=1e-12, atol=0.0)
        assert abs(got[3] - want[3]) <= 1e-12 * max(abs(want[3]), 1e-300)


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

"""Debug build (-DPDHG_DEBUG): the kernels of the fused 2D iteration and the 2D residual
check verify every global index, and the plain path's per-stage kernels (alone and in
batches) every global store, against the extent of its buffer; an index out of range is
recorded (and the access redirected to element 0), and the next residual check returns
PDHG_ERR_BOUNDS.  The parity cases of the fused path (ragged t-chunks, BDF2 across chunk
boundaries, both initial rows, nx != ny, the TMA rows-C at nx = 1024, nx = 2048) and their
float64 plain runs, 1D plain cases (Bluestein lengths, DG P2 / P1, BE and BDF2) alone
and as a batch, the t-solve variants (the exact time operator, the float64 recurrence) and
the mixed solve go through that build with checks after every second iteration and find
no out-of-range index."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

SCRIPT = r'''
import numpy as np
import pdhg_workloads as W
from paper_2207_07234_gb300 import binding as B
base = dict(tau_u=0.4, tau_phi=0.4, tau_u0=0.1, tau_lambda=0.99)
cases = [W.burgers_2d(n=256, nt=71).replace(**base),
         W.burgers_2d(n=256, nt=9).replace(time="bdf2", **base),
         W.burgers_2d(n=256, nt=6).replace(init="pinned", nu=0.02, **base)]
p = W.burgers_2d(n=1024, nt=5).replace(**base)
cases.append(p.replace(ny=512, ly=np.pi, u0=np.ascontiguousarray(p.u0[:512])))
p = W.burgers_2d(n=2048, nt=3).replace(**base)
cases.append(p.replace(ny=256, ly=np.pi / 4, u0=np.ascontiguousarray(p.u0[:256])))
for q in cases:
    for prec, path in (("fp32", "fused"), ("fp64", "plain")):
        with B.Solver(q, precision=prec, path=path) as s:
            s.iterate(4, tol=0.0, check_every=2)
            s.residual()
# the plain path's 1D kernels (power-of-two and Bluestein x-lengths, DG P2 and P1, BE and
# BDF2) alone and as one batch, both precisions
plain = [W.advection_upwind_be(nx=256, nt=9), W.advection_upwind_be(nx=300, nt=7).replace(time="bdf2"),
         W.viscous_burgers(nx=333, nt=6, T=0.5, nu=0.01), W.heat_table1(128, 11),
         W.burgers_dg_p2(ncell=64, nt=5, T=0.5, time="be").replace(c=0.5, tau_u=0.05, tau_u0=0.05, tau_phi=0.05),
         W.traffic_dg_p1(ncell=32, nt=7, time="bdf2")]
for q in plain:
    for prec in ("fp32", "fp64"):
        with B.Solver(q, precision=prec, path="plain") as s:
            s.iterate(4, tol=0.0, check_every=2)
            s.residual()
for prec in ("fp32", "fp64"):
    with B.Batch(plain, precision=prec) as bt:
        bt.iterate(4, tol=0.0, check_every=2)
        for i in range(len(plain)):
            bt.instance(i).residual()
# the exact time operator (1D finite differences with BDF2, DG P1 and P2, 2D plain), the
# float64 t-recurrence (1D and 2D plain, the fused columns at ny = 1024) and the mixed
# solve, whose float64 phase applies K_d^{-1} in float32
exact = [W.advection_upwind_be(nx=256, nt=9).replace(time="bdf2", tprec="exact"),
         W.transport_dg_p1(ncell=64, nt=7).replace(tprec="exact"),
         W.burgers_dg_p2(ncell=32, nt=5, T=0.5).replace(c=0.5, tprec="exact", tau_u=0.05, tau_u0=0.05,
                                                       tau_phi=0.05),
         W.burgers_2d(n=32, nt=6).replace(time="bdf2", tprec="exact", **base)]
for q in exact:
    for prec in ("fp32", "fp64"):
        with B.Solver(q, precision=prec, path="plain") as s:
            s.iterate(4, tol=0.0, check_every=2)
            s.residual()
t64 = [(W.advection_upwind_be(nx=256, nt=9), "plain"), (W.burgers_2d(n=64, nt=5).replace(**base), "plain"),
       (W.burgers_2d(n=1024, nt=3).replace(**base), "fused")]
for q, path in t64:
    with B.Solver(q, precision="fp32", path=path, t64=True) as s:
        s.iterate(4, tol=0.0, check_every=2)
        s.residual()
mixed = [W.advection_upwind_be(nx=256, nt=32, tau=(1.4, 0.1, 0.35, 0.99)),
         W.burgers_2d(n=64, nt=8).replace(alpha=0.0, beta=1.0, space="fd_upwind", lf_a=1.0, c=1.0, tau_u=0.5,
                                          tau_phi=0.5, tau_u0=0.1)]
for q in mixed:
    s, its = B.solve_mixed(q, tol=1e-9, relative=True, check_every=10, max_iters=50000)
    with s:
        assert its[1] > 0, its                              # the float64 phase ran
        s.residual()
print("debug build: no out-of-range index in", len(cases) + len(plain) + len(exact) + len(t64) + len(mixed),
      "cases")
'''


def test_debug_build_finds_no_out_of_range_index():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_07234_gb300 import _build
    lib = _build.build(debug=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PDHG_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=root, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    assert "no out-of-range index" in r.stdout


CANARY_SCRIPT = r'''
import numpy as np
import torch
import pdhg_workloads as W
from paper_2207_07234_gb300 import binding as B
p = W.advection_upwind_be(nx=64, nt=8)
with B.Solver(p, precision="fp64", path="plain") as s:
    s.iterate(2, tol=0.0, check_every=1)             # canaries intact: no error
    # u is the first buffer of the workspace ((nt + 1) x nx doubles); the byte after it
    # starts its canary region.  Overwrite it from the host, as a kernel writing one
    # element past u would.
    off = (p.nt + 1) * p.nx * 8
    s.workspace[off] = 0
    torch.cuda.synchronize()
    try:
        s.iterate(1, tol=0.0, check_every=1)
        print("not detected")
    except B.PdhgError as e:
        print("status", e.status, str(e))
'''


def test_debug_canary_overwrite_is_reported():
    """Debug builds surround every sub-buffer of the workspace with canary bytes, filled
    at create and verified at every residual read: a byte overwritten after the u buffer
    (here from the host; no kernel misbehaves and the GPU sees no fault) makes the next
    check return PDHG_ERR_BOUNDS naming the canary."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_07234_gb300 import _build
    lib = _build.build(debug=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PDHG_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CANARY_SCRIPT], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    assert "status -8" in r.stdout and "canary" in r.stdout and "buffer 0" in r.stdout, r.stdout

"""Thin ctypes binding of include/pdhg.h (argument marshalling only).

Every step of the PDHG iteration runs in libpdhg.so's CUDA kernels; PyTorch is
used here only to own the device workspace and to supply the CUDA stream.
Importing this module loads the library and raises if it is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpdhg.so")

# ---- enums (mirror include/pdhg.h) ----
OK = 0
STATUS = {0: "PDHG_OK", -1: "PDHG_ERR_INVALID_ARG", -2: "PDHG_ERR_WORKSPACE_TOO_SMALL",
          -3: "PDHG_ERR_CUDA", -4: "PDHG_ERR_NONFINITE", -5: "PDHG_ERR_DIVERGED",
          -6: "PDHG_ERR_TIMEOUT", -7: "PDHG_ERR_UNSUPPORTED", -8: "PDHG_ERR_BOUNDS"}
TIME = {"be": 0, "bdf2": 1}
SPACE = {"fd_upwind": 0, "fd_lf": 1, "dg_p2_lf": 2, "dg_p1_upwind": 3, "dg_p1_lf": 4}
PRECISION = {"fp64": 0, "fp32": 1}
INIT = {"lambda": 0, "pinned": 1}
PATH = {"auto": 0, "plain": 1, "fused": 2}
FIELD = {"u": 0, "phi": 1, "phit": 2, "lambda": 3, "lambdat": 4, "u_terminal": 5}
FLAG_EXACT_TIME_PRECOND = 1      # pdhg_scheme.flags: time part of K_d = h_t^2 D_t D_t^T (ablation)
FLAG_U0_ON_DEVICE = 2            # pdhg_scheme.flags: pdhg_problem.u0 is a device pointer
FLAG_T_SOLVE_FP64 = 4            # pdhg_scheme.flags: float32 handle, t-solve recurrence in float64
FLAG_MIXED_STEPS = 8             # pdhg_scheme.flags (one-step solve): float32, then float64 per step
STAGES = ["primal", "residual_fft", "fft_y", "tsolve", "dual", "check", "fused_rows", "fused_cols"]

# every symbol include/pdhg.h declares
EXPORTS = ["pdhg_workspace_size", "pdhg_create", "pdhg_destroy", "pdhg_set_stream", "pdhg_iterate",
           "pdhg_residual", "pdhg_get_field", "pdhg_set_field", "pdhg_solution", "pdhg_info",
           "pdhg_launch_count",
           "pdhg_set_profiling", "pdhg_stage_times", "pdhg_set_graphs", "pdhg_set_wait_budget",
           "pdhg_residual_history", "pdhg_last_error",
           "pdhg_refine_workspace_size",
           "pdhg_solve_refine", "pdhg_one_step_workspace_size", "pdhg_solve_one_step",
           "pdhg_gradient_workspace_size", "pdhg_solve_gradient", "pdhg_mixed_workspace_size",
           "pdhg_solve_mixed", "pdhg_batch_workspace_size",
           "pdhg_batch_create", "pdhg_batch_destroy", "pdhg_batch_iterate", "pdhg_batch_reset",
           "pdhg_batch_instance", "pdhg_batch_launch_count", "pdhg_batch_set_launch",
           "pdhg_batch_set_wait_budget", "pdhg_batch_set_graphs", "pdhg_residual_noalloc"]


class PdhgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class pdhg_problem(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("nu", ctypes.c_double),
                ("gamma_half", ctypes.POINTER(ctypes.c_double)), ("u0", ctypes.POINTER(ctypes.c_double)),
                ("lf_a", ctypes.c_double), ("c", ctypes.c_double), ("gamma_hat", ctypes.c_double),
                ("tau_u", ctypes.c_double), ("tau_u0", ctypes.c_double), ("tau_phi", ctypes.c_double),
                ("tau_lambda", ctypes.c_double)]


class pdhg_grid(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("T", ctypes.c_double),
                ("nt", ctypes.c_int64)]


class pdhg_scheme(ctypes.Structure):
    _fields_ = [("time", ctypes.c_int32), ("space", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("init", ctypes.c_int32), ("path", ctypes.c_int32), ("flags", ctypes.c_int32)]


_lib = None


def load(path: str | None = None):
    """Load libpdhg.so (raises OSError if it has not been built).  PDHG_LIBRARY in the
    environment names another build of the same library (the debug build)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("PDHG_LIBRARY", LIB_PATH)
    if not os.path.exists(path):
        raise OSError(f"{path} not found: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P, G, S = ctypes.POINTER(pdhg_problem), ctypes.POINTER(pdhg_grid), ctypes.POINTER(pdhg_scheme)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "pdhg_workspace_size": [P, G, S, ctypes.POINTER(ctypes.c_size_t)],
        "pdhg_create": [P, G, S, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "pdhg_destroy": [vp],
        "pdhg_set_stream": [vp, vp],
        "pdhg_iterate": [vp, i64, ctypes.c_double, i32, i32, ctypes.POINTER(i64)],
        "pdhg_residual": [vp, ctypes.POINTER(ctypes.c_double)],
        "pdhg_get_field": [vp, i32, vp, i32],
        "pdhg_solution": [vp, vp, i32, i32],
        "pdhg_set_field": [vp, i32, vp, i32],
        "pdhg_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                      ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "pdhg_launch_count": [vp, ctypes.POINTER(i64), i32],
        "pdhg_set_profiling": [vp, i32],
        "pdhg_stage_times": [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)],
        "pdhg_set_graphs": [vp, i32],
        "pdhg_set_wait_budget": [vp, ctypes.c_uint64],
        "pdhg_residual_history": [vp, ctypes.POINTER(ctypes.c_double), i64, ctypes.POINTER(i64), i32],
        "pdhg_refine_workspace_size": [P, G, S, i32, ctypes.POINTER(ctypes.c_size_t)],
        "pdhg_solve_refine": [P, G, S, i32, ctypes.POINTER(i64), ctypes.c_double, i32, i32, vp, ctypes.c_size_t,
                              vp, ctypes.POINTER(vp), ctypes.POINTER(i64)],
        "pdhg_one_step_workspace_size": [P, G, S, ctypes.POINTER(ctypes.c_size_t)],
        "pdhg_gradient_workspace_size": [P, G, S, ctypes.POINTER(ctypes.c_size_t)],
        "pdhg_mixed_workspace_size": [P, G, S, ctypes.POINTER(ctypes.c_size_t)],
        "pdhg_solve_mixed": [P, G, S, ctypes.c_double, i32, i32, i64, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp),
                             ctypes.POINTER(i64)],
        "pdhg_batch_workspace_size": [i32, P, G, S, ctypes.POINTER(ctypes.c_size_t)],
        "pdhg_batch_create": [i32, P, G, S, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "pdhg_batch_destroy": [vp],
        "pdhg_batch_iterate": [vp, i64, ctypes.c_double, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i32)],
        "pdhg_batch_reset": [vp],
        "pdhg_batch_instance": [vp, i32, ctypes.POINTER(vp)],
        "pdhg_batch_launch_count": [vp, ctypes.POINTER(i64), i32],
        "pdhg_batch_set_launch": [vp, i32, i32, i32, ctypes.POINTER(i32)],
        "pdhg_batch_set_wait_budget": [vp, ctypes.c_uint64],
        "pdhg_batch_set_graphs": [vp, ctypes.c_int32],
        "pdhg_solve_gradient": [P, G, S, ctypes.POINTER(ctypes.c_double), ctypes.c_double, i64, ctypes.c_double, i64,
                                i32, vp, ctypes.c_size_t, vp, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)],
        "pdhg_solve_one_step": [P, G, S, ctypes.c_double, i64, i32, vp, ctypes.c_size_t, vp, vp,
                                ctypes.POINTER(i64), ctypes.POINTER(i64)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.pdhg_last_error.argtypes = []
    lib.pdhg_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status):
    if status != OK:
        raise PdhgError(status, load().pdhg_last_error().decode())


def structs(p, precision="fp32", path="auto", u0_device=None, t64=False):
    """C structs for a pdhg_workloads.Problem; returns (prob, grid, scheme, keepalive).
    u0_device: a contiguous float64 CUDA tensor holding u0 (PDHG_FLAG_U0_ON_DEVICE), else
    p.u0 is passed from host memory."""
    prob = pdhg_problem()
    prob.alpha, prob.beta, prob.nu = p.alpha, p.beta, p.nu
    if u0_device is not None:
        import torch
        assert u0_device.is_cuda and u0_device.dtype == torch.float64 and u0_device.is_contiguous()
        assert u0_device.numel() == p.ndof
        keep = [u0_device]
        prob.u0 = ctypes.cast(ctypes.c_void_p(u0_device.data_ptr()), ctypes.POINTER(ctypes.c_double))
    else:
        u0 = np.ascontiguousarray(p.u0, dtype=np.float64).ravel()
        keep = [u0]
        prob.u0 = u0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if p.gamma_half is not None:
        g = np.ascontiguousarray(p.gamma_half, dtype=np.float64)
        keep.append(g)
        prob.gamma_half = g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    prob.lf_a, prob.c, prob.gamma_hat = p.lf_a, p.c, p.gamma_hat
    prob.tau_u, prob.tau_u0, prob.tau_phi, prob.tau_lambda = p.tau_u, p.tau_u0, p.tau_phi, p.tau_lambda
    grid = pdhg_grid(p.dims, p.nx, p.ny if p.dims == 2 else 1, p.lx, p.ly, p.T, p.nt)
    flags = FLAG_EXACT_TIME_PRECOND if getattr(p, "tprec", "tridiag") == "exact" else 0
    if u0_device is not None:
        flags |= FLAG_U0_ON_DEVICE
    if t64:
        flags |= FLAG_T_SOLVE_FP64
    scheme = pdhg_scheme(TIME[p.time], SPACE[p.space], PRECISION[precision], INIT[p.init], PATH[path], flags)
    return prob, grid, scheme, keep


def workspace_size(p, precision="fp32", path="auto") -> int:
    prob, grid, scheme, _keep = structs(p, precision, path)
    n = ctypes.c_size_t(0)
    _check(load().pdhg_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                      ctypes.byref(n)))
    return n.value


class Solver:
    """One space-time problem on the GPU (a pdhg_handle plus its torch-owned workspace)."""

    def __init__(self, p, precision="fp32", path="auto", device=None, stream=None, _adopt=None, t64=False):
        """t64: float32 fields with the t-solve recurrence in float64 (PDHG_FLAG_T_SOLVE_FP64)."""
        import torch
        self._torch = torch
        self.p = p
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.device = torch.device(device if device is not None else "cuda")
        self.ndof = p.ndof
        self.nt = p.nt
        self._owned = True
        if _adopt is not None:           # a handle made by another entry point, in `workspace`
            self.h, self.workspace, self._stream = _adopt[:3]
            self._owned = _adopt[3] if len(_adopt) > 3 else True
            return
        lib = load()
        prob, grid, scheme, keep = structs(p, precision, path, t64=t64)
        nbytes = ctypes.c_size_t(0)
        _check(lib.pdhg_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                       ctypes.byref(nbytes)))
        self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._stream = s
        h = ctypes.c_void_p()
        _check(lib.pdhg_create(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                               ctypes.c_void_p(self.workspace.data_ptr()), nbytes.value,
                               ctypes.c_void_p(s.cuda_stream), ctypes.byref(h)))
        self.h = h

    # ---- lifecycle ----
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            if getattr(self, "_owned", True):
                load().pdhg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- iteration ----
    def iterate(self, n, tol=0.0, check_every=0, relative=False) -> int:
        done = ctypes.c_int64(0)
        _check(load().pdhg_iterate(self.h, int(n), float(tol), int(check_every), int(bool(relative)),
                                   ctypes.byref(done)))
        return done.value

    def residual(self) -> np.ndarray:
        out = (ctypes.c_double * 4)()
        _check(load().pdhg_residual(self.h, out))
        return np.array(list(out))

    def history(self, clear=False) -> np.ndarray:
        """Res at every check of iterate(): rows [iterations, Res entries 0..3]."""
        lib = load()
        n = ctypes.c_int64(0)
        _check(lib.pdhg_residual_history(self.h, None, 0, ctypes.byref(n), 0))
        out = np.zeros((max(n.value, 1), 5))
        _check(lib.pdhg_residual_history(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         max(n.value, 1), ctypes.byref(n), int(bool(clear))))
        return out[: n.value]

    def info(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        d, e = ctypes.c_int32(), ctypes.c_int32()
        _check(load().pdhg_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                ctypes.byref(d), ctypes.byref(e)))
        return {"ndof": a.value, "nt": b.value, "iterations": c.value, "precision": d.value,
                "path": {1: "plain", 2: "fused"}.get(e.value, e.value)}

    def launches(self, reset=False) -> int:
        n = ctypes.c_int64()
        _check(load().pdhg_launch_count(self.h, ctypes.byref(n), int(bool(reset))))
        return n.value

    def set_profiling(self, on=True):
        _check(load().pdhg_set_profiling(self.h, int(bool(on))))

    def set_graphs(self, on=True):
        _check(load().pdhg_set_graphs(self.h, int(bool(on))))

    def set_wait_budget(self, ns):
        """Budget (ns) of each bounded device wait; 0 forces the timeout path."""
        _check(load().pdhg_set_wait_budget(self.h, int(ns)))

    def stage_times(self):
        ms = (ctypes.c_double * len(STAGES))()
        n = (ctypes.c_int64 * len(STAGES))()
        _check(load().pdhg_stage_times(self.h, ms, n))
        return {STAGES[i]: (ms[i], n[i]) for i in range(len(STAGES)) if n[i] > 0}

    # ---- fields ----
    def _shape(self, field):
        sl = tuple(self.p.slice_shape)
        return {"u": (self.nt + 1,) + sl, "u_terminal": sl, "phi": (self.nt,) + sl,
                "phit": (self.nt,) + sl, "lambda": sl, "lambdat": sl}[field]

    def get(self, field):
        """Device copy of a field as a torch tensor of the handle's dtype."""
        t = self._torch.empty(self._shape(field), dtype=self.dtype, device=self.device)
        _check(load().pdhg_get_field(self.h, FIELD[field], ctypes.c_void_p(t.data_ptr()), 1))
        return t

    def get_host(self, field, out=None):
        """Copy a field into a host numpy array (pinned or pageable)."""
        np_dtype = np.float64 if self.precision == "fp64" else np.float32
        a = out if out is not None else np.empty(self._shape(field), dtype=np_dtype)
        _check(load().pdhg_get_field(self.h, FIELD[field], ctypes.c_void_p(a.ctypes.data), 0))
        return a

    def solution(self, which="u"):
        """pdhg_solution: u (all slices), u_terminal, phi or lambda as a device tensor."""
        t = self._torch.empty(self._shape(which), dtype=self.dtype, device=self.device)
        _check(load().pdhg_solution(self.h, ctypes.c_void_p(t.data_ptr()), 1, FIELD[which]))
        return t

    def set_stream(self, stream):
        """Later calls run on `stream` (a torch.cuda.Stream); the old stream's work finishes first."""
        _check(load().pdhg_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))
        self._stream = stream

    def set(self, field, value):
        t = self._torch.as_tensor(value, dtype=self.dtype, device=self.device).contiguous()
        assert tuple(t.shape) == self._shape(field)
        # the conversion above runs on torch's current stream; the copy runs on the
        # handle's stream, which must wait for it
        self._stream.wait_stream(self._torch.cuda.current_stream(self.device))
        _check(load().pdhg_set_field(self.h, FIELD[field], ctypes.c_void_p(t.data_ptr()), 1))


def solve(p, precision="fp32", max_iters=10000, tol=1e-6, check_every=50, relative=True, path="auto"):
    """Convenience: run Algorithm 1 to tolerance; returns (u as numpy, iterations, Res)."""
    with Solver(p, precision=precision, path=path) as s:
        it = s.iterate(max_iters, tol=tol, check_every=check_every, relative=relative)
        return s.get_host("u"), it, s.residual()


def solve_refine(p, levels, iters, tol=1e-3, check_every=1, relative=False, precision="fp64", path="auto",
                 device=None, stream=None):
    """Algorithm 2 (Sec. 3.4) on the final problem p: levels with p.nt >> (levels-1-k)
    slices, iters[k] iterations at most on level k.  Returns (Solver of the finest
    level, iterations per level)."""
    import torch
    lib = load()
    prob, grid, scheme, keep = structs(p, precision, path)
    nbytes = ctypes.c_size_t(0)
    _check(lib.pdhg_refine_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                          int(levels), ctypes.byref(nbytes)))
    dev = torch.device(device if device is not None else "cuda")
    ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    it_in = (ctypes.c_int64 * levels)(*[int(v) for v in iters])
    it_out = (ctypes.c_int64 * levels)()
    h = ctypes.c_void_p()
    _check(lib.pdhg_solve_refine(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme), int(levels), it_in,
                                 float(tol), int(check_every), int(bool(relative)), ctypes.c_void_p(ws.data_ptr()),
                                 nbytes.value, ctypes.c_void_p(s.cuda_stream), ctypes.byref(h), it_out))
    return Solver(p, precision=precision, device=dev, _adopt=(h, ws, s)), list(it_out)


def solve_one_step(p, tol=1e-3, max_iters_per_step=100000, check_every=1, precision="fp64", device=None,
                   stream=None, path="auto"):
    """Algorithm 3 (Sec. 3.5): returns (u* as a device tensor [nt+1][...], iterations per step).
    precision "mixed": each step in float32 to tol or float32's floor, then float64
    (PDHG_FLAG_MIXED_STEPS; u* in float64).  path: of the float32 step handles ("auto":
    the fused path for 2D finite differences where it applies; float64 steps run plain)."""
    import torch
    lib = load()
    prob, grid, scheme, keep = structs(p, "fp64" if precision == "mixed" else precision,
                                       "plain" if precision == "fp64" else path)
    if precision == "mixed":
        scheme.flags |= FLAG_MIXED_STEPS
    nbytes = ctypes.c_size_t(0)
    _check(lib.pdhg_one_step_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                            ctypes.byref(nbytes)))
    dev = torch.device(device if device is not None else "cuda")
    ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    dtype = torch.float32 if precision == "fp32" else torch.float64
    u = torch.empty((p.nt + 1,) + tuple(p.slice_shape), dtype=dtype, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))       # u was allocated on the current stream
    per = (ctypes.c_int64 * p.nt)()
    tot = ctypes.c_int64(0)
    _check(lib.pdhg_solve_one_step(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme), float(tol),
                                   int(max_iters_per_step), int(check_every), ctypes.c_void_p(ws.data_ptr()),
                                   nbytes.value, ctypes.c_void_p(s.cuda_stream), ctypes.c_void_p(u.data_ptr()),
                                   per, ctypes.byref(tot)))
    return u, list(per)


def solve_gradient(p, target, tol=1e-10, max_iters=100000, adj_tol=1e-10, adj_max_iters=100000, check_every=10,
                   precision="fp64", device=None, stream=None, u0_device=None):
    """Loss = w_x |u^nt - target|^2 of the scheme's solution and its gradient through
    the solve: returns (loss, dLoss/du0 as numpy, dLoss/dnu, [forward, adjoint] iterations).
    u0_device: u0 as a float64 CUDA tensor (used instead of p.u0, not copied to the host)."""
    import torch
    lib = load()
    prob, grid, scheme, keep = structs(p, precision, "plain", u0_device=u0_device)
    nbytes = ctypes.c_size_t(0)
    _check(lib.pdhg_gradient_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                            ctypes.byref(nbytes)))
    dev = torch.device(device if device is not None else "cuda")
    ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    tg = np.ascontiguousarray(target, dtype=np.float64).ravel()
    assert tg.size == p.ndof
    du0 = np.empty(p.ndof)
    loss, dnu = ctypes.c_double(0), ctypes.c_double(0)
    iters = (ctypes.c_int64 * 2)()
    _check(lib.pdhg_solve_gradient(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                   tg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(tol), int(max_iters),
                                   float(adj_tol), int(adj_max_iters), int(check_every),
                                   ctypes.c_void_p(ws.data_ptr()), nbytes.value, ctypes.c_void_p(s.cuda_stream),
                                   ctypes.byref(loss), du0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(dnu), iters))
    return loss.value, du0.reshape(p.slice_shape), dnu.value, list(iters)


def terminal_loss_fn():
    """A torch.autograd.Function: loss = TerminalLoss.apply(u0, nu, problem, target, opts)
    with u0 a float64 tensor of the slice shape (a CUDA tensor is passed to the library as
    a device pointer) and nu a 0-d float64 tensor; the backward pass returns dLoss/du0
    and dLoss/dnu computed by solve_gradient (opts may choose precision="fp32")."""
    import torch

    class TerminalLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u0, nu, problem, target, opts=None):
            # u0 stays in device memory (PDHG_FLAG_U0_ON_DEVICE) when it is a CUDA tensor
            q = problem.replace(nu=float(nu))
            if u0.is_cuda:
                dev_u0 = u0.detach().to(torch.float64).contiguous()
                loss, du0, dnu, _ = solve_gradient(q, target, device=u0.device, u0_device=dev_u0, **(opts or {}))
            else:
                q = q.replace(u0=u0.detach().numpy().astype(np.float64))
                loss, du0, dnu, _ = solve_gradient(q, target, **(opts or {}))
            ctx.save_for_backward(torch.as_tensor(du0, dtype=u0.dtype, device=u0.device),
                                  torch.as_tensor(dnu, dtype=nu.dtype, device=nu.device))
            return torch.as_tensor(loss, dtype=u0.dtype, device=u0.device)

        @staticmethod
        def backward(ctx, grad):
            du0, dnu = ctx.saved_tensors
            return grad * du0, grad * dnu, None, None, None

    return TerminalLoss


def solve_mixed(p, tol=1e-6, relative=True, check_every=50, max_iters=100000, path="auto", device=None,
                stream=None):
    """float32 until tol or float32's floor, then float64 to tol (pdhg_solve_mixed).
    Returns (float64 Solver holding the result, [float32, float64] iterations)."""
    import torch
    lib = load()
    prob, grid, scheme, keep = structs(p, "fp64", path)
    nbytes = ctypes.c_size_t(0)
    _check(lib.pdhg_mixed_workspace_size(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme),
                                         ctypes.byref(nbytes)))
    dev = torch.device(device if device is not None else "cuda")
    ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    h = ctypes.c_void_p()
    its = (ctypes.c_int64 * 2)()
    _check(lib.pdhg_solve_mixed(ctypes.byref(prob), ctypes.byref(grid), ctypes.byref(scheme), float(tol),
                                int(bool(relative)), int(check_every), int(max_iters), ctypes.c_void_p(ws.data_ptr()),
                                nbytes.value, ctypes.c_void_p(s.cuda_stream), ctypes.byref(h), its))
    return Solver(p, precision="fp64", device=dev, _adopt=(h, ws, s)), list(its)


class Batch:
    """Many independent 1D problems advanced by shared launches (pdhg_batch)."""

    def __init__(self, problems, precision="fp32", device=None, stream=None):
        import torch
        lib = load()
        self.problems = list(problems)
        n = len(self.problems)
        self.precision = precision
        self.device = torch.device(device if device is not None else "cuda")
        parts = [structs(p, precision, "plain") for p in self.problems]
        self._keep = [k for part in parts for k in part[3]]
        self._probs = (pdhg_problem * n)(*[part[0] for part in parts])
        self._grids = (pdhg_grid * n)(*[part[1] for part in parts])
        self._schemes = (pdhg_scheme * n)(*[part[2] for part in parts])
        nbytes = ctypes.c_size_t(0)
        _check(lib.pdhg_batch_workspace_size(n, self._probs, self._grids, self._schemes, ctypes.byref(nbytes)))
        self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=self.device)
        self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        b = ctypes.c_void_p()
        _check(lib.pdhg_batch_create(n, self._probs, self._grids, self._schemes,
                                     ctypes.c_void_p(self.workspace.data_ptr()), nbytes.value,
                                     ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(b)))
        self.b = b
        self.count = n
        # the autotuner's choice of tiles (batch_tiles.json, written by autotune.py), if any
        tf = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_tiles.json")
        if os.path.exists(tf) and os.environ.get("PDHG_BATCH_TILES") != "none":
            import json
            with open(tf) as f:
                cfg = json.load(f)
            self.set_launch(persistent=bool(cfg.get("persistent", False)),
                            blocks_per_sm=int(cfg.get("blocks_per_sm", 0)), order=int(cfg.get("order", 0)),
                            tiles=cfg.get("tiles", [1] * 8))

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            load().pdhg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def iterate(self, n, tol=0.0, check_every=0, relative=False):
        """Returns (iterations per instance in this call, state per instance:
        1 converged, 0 active, -1 non-finite or diverged)."""
        it = (ctypes.c_int64 * self.count)()
        st = (ctypes.c_int32 * self.count)()
        _check(load().pdhg_batch_iterate(self.b, int(n), float(tol), int(check_every), int(bool(relative)), it, st))
        return np.array(list(it)), np.array(list(st))

    def reset(self):
        _check(load().pdhg_batch_reset(self.b))

    def instance(self, i):
        """Borrowed view of instance i (a Solver that does not own its handle)."""
        h = ctypes.c_void_p()
        _check(load().pdhg_batch_instance(self.b, int(i), ctypes.byref(h)))
        return Solver(self.problems[i], precision=self.precision, device=self.device,
                      _adopt=(h, self.workspace, self._stream, False))

    def launches(self, reset=False) -> int:
        n = ctypes.c_int64()
        _check(load().pdhg_batch_launch_count(self.b, ctypes.byref(n), int(bool(reset))))
        return n.value

    def set_launch(self, persistent=True, blocks_per_sm=0, order=0, tiles=None):
        """One persistent launch per iteration or (persistent=False, the library's default)
        one launch per stage; resident blocks per multiprocessor (0: as many as fit); queue
        order (0 stage-major, 1 instance-major); tiles: row items per queue entry for the 8
        size classes (None: keep)."""
        t = (ctypes.c_int32 * 8)(*[int(v) for v in tiles]) if tiles is not None else None
        _check(load().pdhg_batch_set_launch(self.b, int(bool(persistent)), int(blocks_per_sm), int(order), t))

    def set_wait_budget(self, ns):
        """Budget (ns) of each bounded wait of the persistent iteration; 0 forces the timeout path."""
        _check(load().pdhg_batch_set_wait_budget(self.b, int(ns)))

    def set_graphs(self, enable):
        """CUDA-graph replay of check_every-iteration chunks (the default) or launches one by one."""
        _check(load().pdhg_batch_set_graphs(self.b, int(bool(enable))))

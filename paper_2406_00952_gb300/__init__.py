"""Block omega-circulant preconditioned all-at-once solver for theta-discretised parabolic optimal
control (Fung & Hon), on one GB300.  The compute path is libpcb.so (include/pcb.h); PyTorch only
supplies device memory and streams.

    prob = Problem(N=511, n=512, theta=1.0, gamma=1e-2, precision="mixed")
    b = prob.assemble_rhs(g, f)           # device tensors, (n+1)*m samples each
    x, info = prob.solve(b)
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib
from ._lib import PcbDesc, PcbSolveInfo, PcbSolveOpts, PcbTuneInfo, check

OPS = {"A": 0, "Ahat": 1}
PRECONDS = {None: 0, "none": 0, "abs_ps": 1, "ps": 2, "pms": 3}
METHODS = {"auto": 0, "minres": 1, "gmres": 2, "fgmres": 3}
PRECISIONS = {"fp64": 0, "mixed": 1}
BCS = {"dirichlet": 0, "neumann": 1}


def _ptr(t: torch.Tensor | None, numel: int | None = None) -> int | None:
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _opts(method="auto", precond=None, tol=1e-8, maxit=500, restart=30, max_refinements=10, fixed_iterations=0,
          profile=False, inner_floor=0.0, graphs=True):
    return PcbSolveOpts(METHODS[method], PRECONDS[precond], float(tol), int(maxit), int(restart),
                        int(max_refinements), int(fixed_iterations), int(bool(profile)), float(inner_floor),
                        int(not graphs))


class Problem:
    """One control problem on the current CUDA device and stream (C-ABI pcb_create).
    bc="neumann" selects Example 3's homogeneous Neumann grid (N nodes per side including the
    boundary); a is the constant coefficient when a_edges is None; fem=True selects bilinear finite
    elements (mass matrix M != I) in place of finite differences; multigrid=True solves the shifted
    systems with V-cycles also for a constant coefficient (the paper's route for Example 3)."""

    def __init__(self, N, n, theta, gamma, T=1.0, zeta=math.pi, a_edges=None, precision="fp64", mg_cycles=2,
                 stream: torch.cuda.Stream | None = None, bc="dirichlet", a=1.0, fem=False, multigrid=False):
        self.lib = _lib.load()
        self.N, self.n, self.theta, self.gamma, self.T = int(N), int(n), float(theta), float(gamma), float(T)
        self.m = self.N * self.N
        self.size = 2 * self.m * self.n
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._a = None
        ap = None
        if a_edges is not None:
            import numpy as np
            self._a = np.ascontiguousarray(a_edges, dtype=np.float64)
            ap = self._a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d = PcbDesc(self.N, self.n, self.theta, self.T, self.gamma, float(zeta), ap, PRECISIONS[precision],
                    int(mg_cycles), ctypes.c_void_p(self.stream.cuda_stream), BCS[bc], float(a), int(bool(fem)),
                    int(bool(multigrid)))
        h = ctypes.c_void_p()
        check("pcb_create", self.lib.pcb_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self.precision = precision

    def close(self):
        if getattr(self, "h", None):
            self.lib.pcb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self):
        return torch.empty(self.size, dtype=torch.float64, device="cuda")

    @property
    def workspace_bytes(self) -> int:
        return int(self.lib.pcb_workspace_bytes(self.h))

    def matvec(self, x, out=None, op="A"):
        out = self._empty() if out is None else out
        check("pcb_matvec", self.lib.pcb_matvec(self.h, OPS[op], _ptr(x, self.size), _ptr(out, self.size)))
        return out

    def lanczos_product(self, y, beta, r1=None, oldb=0.0, out=None, precision=None):
        """One Lanczos step of MINRES (C-ABI pcb_lanczos_product): out = A y/beta - (beta/oldb) r1 and
        y . out / beta, in FP64 or in the two-word FP32 arithmetic of mixed-precision inner iterations."""
        out = self._empty() if out is None else out
        dot = ctypes.c_double()
        r1p = _ptr(r1, self.size) if r1 is not None else None
        check("pcb_lanczos_product", self.lib.pcb_lanczos_product(
            self.h, PRECISIONS[precision or self.precision], _ptr(y, self.size), r1p, float(beta), float(oldb),
            _ptr(out, self.size), ctypes.byref(dot)))
        return out, dot.value

    def precond_apply(self, x, out=None, kind="abs_ps", precision=None):
        out = self._empty() if out is None else out
        prec = PRECISIONS[precision or self.precision]
        check("pcb_precond_apply", self.lib.pcb_precond_apply(self.h, PRECONDS[kind], prec, _ptr(x, self.size),
                                                             _ptr(out, self.size)))
        return out

    def autotune(self, kind=None, reps=3) -> dict:
        """Time the preconditioner apply under each kernel configuration that fits this problem and
        keep the fastest (C-ABI pcb_autotune); later problems of the same shape start with it."""
        info = PcbTuneInfo()
        check("pcb_autotune", self.lib.pcb_autotune(self.h, PRECONDS[kind], int(reps), ctypes.byref(info)))
        return info.as_dict()

    def tune_select(self, candidate) -> dict:
        """Run this problem in configuration `candidate` of the autotuner's list (C-ABI
        pcb_tune_select; candidate < 0: report the list's length and the current configuration)."""
        info = PcbTuneInfo()
        check("pcb_tune_select", self.lib.pcb_tune_select(self.h, int(candidate), ctypes.byref(info)))
        return info.as_dict()

    def assemble_rhs(self, g, f, y0=None, op="A", out=None):
        out = self._empty() if out is None else out
        ns = (self.n + 1) * self.m
        check("pcb_assemble_rhs", self.lib.pcb_assemble_rhs(self.h, OPS[op], _ptr(g, ns), _ptr(f, ns),
                                                           _ptr(y0, self.m), _ptr(out, self.size)))
        return out

    def recover(self, x):
        y = torch.empty(self.m * self.n, dtype=torch.float64, device="cuda")
        p = torch.empty_like(y)
        check("pcb_recover", self.lib.pcb_recover(self.h, _ptr(x, self.size), _ptr(y), _ptr(p)))
        return y, p

    def solve(self, b, x=None, allow_not_converged=False, **kw):
        x = self._empty() if x is None else x
        o = _opts(**kw)
        info = PcbSolveInfo()
        rc = self.lib.pcb_solve(self.h, ctypes.byref(o), _ptr(b, self.size), _ptr(x, self.size), ctypes.byref(info))
        check("pcb_solve", rc, allow_not_converged)
        return x, info.as_dict()

    def solve_host(self, b_host, x_host=None, allow_not_converged=False, **kw):
        """Host-buffer solve (copies in and out inside the call); b_host/x_host: float64 numpy arrays
        (pinned torch CPU tensors also accepted)."""
        import numpy as np
        if isinstance(b_host, torch.Tensor):
            bp = b_host.data_ptr()
            x_host = torch.empty_like(b_host) if x_host is None else x_host
            xp = x_host.data_ptr()
        else:
            b_host = np.ascontiguousarray(b_host, dtype=np.float64)
            x_host = np.empty_like(b_host) if x_host is None else x_host
            bp, xp = b_host.ctypes.data, x_host.ctypes.data
        o = _opts(**kw)
        info = PcbSolveInfo()
        rc = self.lib.pcb_solve_host(self.h, ctypes.byref(o), bp, xp, ctypes.byref(info))
        check("pcb_solve_host", rc, allow_not_converged)
        return x_host, info.as_dict()


def fp64_rates(stream: torch.cuda.Stream | None = None) -> dict:
    """Measured FP64 fused multiply-add and add instruction rates of the current device
    (C-ABI pcb_measure_fp64_rates), instructions per second."""
    lib = _lib.load()
    st = stream if stream is not None else torch.cuda.current_stream()
    f, a = ctypes.c_double(), ctypes.c_double()
    check("pcb_measure_fp64_rates", lib.pcb_measure_fp64_rates(ctypes.c_void_p(st.cuda_stream), ctypes.byref(f),
                                                               ctypes.byref(a)))
    return {"fma_per_s": f.value, "add_per_s": a.value}


def batch_solve(problems, bs, xs=None, allow_not_converged=False, **kw):
    """Solve independent problems with shared launches (C-ABI pcb_batch_solve)."""
    lib = _lib.load()
    k = len(problems)
    xs = [p._empty() for p in problems] if xs is None else xs
    H = (ctypes.c_void_p * k)(*[p.h.value for p in problems])
    Bp = (ctypes.c_void_p * k)(*[_ptr(b, p.size) for p, b in zip(problems, bs)])
    Xp = (ctypes.c_void_p * k)(*[_ptr(x, p.size) for p, x in zip(problems, xs)])
    infos = (PcbSolveInfo * k)()
    o = _opts(**kw)
    rc = lib.pcb_batch_solve(H, k, ctypes.byref(o), Bp, Xp, infos)
    check("pcb_batch_solve", rc, allow_not_converged)
    return xs, [i.as_dict() for i in infos]

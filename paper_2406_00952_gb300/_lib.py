"""ctypes binding of libpcb.so (include/pcb.h).  Argument marshalling only: every step of the
solver runs in the library's CUDA kernels.  Raises when the library is missing -- there is no
fallback path."""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, c_double, c_int, c_longlong, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpcb.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pcb.h")

PCB_OK = 0
PCB_NOT_CONVERGED = 1
STATUS = {0: "ok", 1: "not converged", -1: "invalid argument", -2: "unsupported", -3: "singular",
          -4: "out of memory", -5: "CUDA error", -6: "non-finite", -7: "breakdown", -8: "timeout",
          -9: "too large"}


class PcbDesc(ctypes.Structure):
    _fields_ = [("N", c_int), ("n", c_int), ("theta", c_double), ("T", c_double), ("gamma", c_double),
                ("zeta", c_double), ("a_edges", POINTER(c_double)), ("precision", c_int),
                ("mg_cycles", c_int), ("stream", c_void_p), ("bc", c_int), ("a_const", c_double),
                ("fem", c_int), ("multigrid", c_int)]


class PcbSolveOpts(ctypes.Structure):
    _fields_ = [("method", c_int), ("precond", c_int), ("tol", c_double), ("maxit", c_int),
                ("restart", c_int), ("max_refinements", c_int), ("fixed_iterations", c_int),
                ("profile", c_int), ("inner_floor", c_double), ("no_graphs", c_int)]


class PcbSolveInfo(ctypes.Structure):
    _fields_ = [("status", c_int), ("method", c_int), ("precond", c_int), ("iterations", c_int),
                ("refinements", c_int), ("relres", c_double), ("seconds", c_double),
                ("launches", c_longlong), ("precond_applies", c_int), ("precond_ms", c_double),
                ("matvecs", c_int), ("matvec_ms", c_double), ("matvecs_inner", c_int),
                ("matvec_inner_ms", c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PcbTuneInfo(ctypes.Structure):
    _fields_ = [("candidates", c_int), ("rejected", c_int), ("chosen", c_int), ("default_ms", c_double),
                ("best_ms", c_double),
                ("pipelined_dst", c_int), ("pipelined_time", c_int), ("time_major_handoff", c_int),
                ("dst_lanes", c_int), ("time_lanes", c_int), ("tile_scale", c_double), ("time512_blocks", c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PcbServerOpts(ctypes.Structure):
    _fields_ = [("budget_bytes", c_longlong), ("max_slots", c_int), ("precision", c_int), ("tol", c_double),
                ("maxit", c_int), ("restart", c_int), ("stream", c_void_p)]


class PcbServerDone(ctypes.Structure):
    _fields_ = [("tag", c_longlong), ("status", c_int), ("iterations", c_int), ("refinements", c_int),
                ("relres", c_double)]


_lib = None


def header_functions() -> list[str]:
    """Names of the functions include/pcb.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pcb_[a-z_0-9]+)\s*\(", txt)))


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2406_00952_gb300._build.build() "
                           "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "pcb_create": (c_int, [POINTER(PcbDesc), POINTER(c_void_p)]),
        "pcb_destroy": (None, [P]),
        "pcb_status_str": (ctypes.c_char_p, [c_int]),
        "pcb_unknowns": (c_longlong, [P]),
        "pcb_workspace_bytes": (c_longlong, [P]),
        "pcb_assemble_rhs": (c_int, [P, c_int, P, P, P, P]),
        "pcb_matvec": (c_int, [P, c_int, P, P]),
        "pcb_precond_apply": (c_int, [P, c_int, c_int, P, P]),
        "pcb_lanczos_product": (c_int, [P, c_int, P, P, c_double, c_double, P, POINTER(c_double)]),
        "pcb_recover": (c_int, [P, P, P, P]),
        "pcb_solve": (c_int, [P, POINTER(PcbSolveOpts), P, P, POINTER(PcbSolveInfo)]),
        "pcb_solve_host": (c_int, [P, POINTER(PcbSolveOpts), P, P, POINTER(PcbSolveInfo)]),
        "pcb_batch_solve": (c_int, [POINTER(c_void_p), c_int, POINTER(PcbSolveOpts), POINTER(c_void_p),
                                    POINTER(c_void_p), POINTER(PcbSolveInfo)]),
        "pcb_precond_apply_noalloc": (c_int, [POINTER(PcbDesc), c_int, c_int, P, P]),
        "pcb_autotune": (c_int, [P, c_int, c_int, POINTER(PcbTuneInfo)]),
        "pcb_tune_select": (c_int, [P, c_int, POINTER(PcbTuneInfo)]),
        "pcb_measure_fp64_rates": (c_int, [P, POINTER(c_double), POINTER(c_double)]),
        "pcb_server_create": (c_int, [POINTER(PcbServerOpts), POINTER(c_void_p)]),
        "pcb_server_destroy": (None, [P]),
        "pcb_server_submit": (c_int, [P, POINTER(PcbDesc), P, P, c_longlong]),
        "pcb_server_step": (c_int, [P, POINTER(PcbServerDone), c_int, POINTER(c_int), POINTER(c_int),
                                    POINTER(c_int)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PcbError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code})")
        self.code = code


def check(fn: str, code: int, allow_not_converged: bool = False) -> int:
    if code == PCB_OK or (allow_not_converged and code == PCB_NOT_CONVERGED):
        return code
    raise PcbError(fn, code)

"""Continuous-batching serving loop over the library's server (pcb_server_* in include/pcb.h).

Requests (independent control solves of different grid size, horizon, gamma and target) arrive on
a timeline; each is submitted when its arrival time has passed, admitted by the library when a slot
and HBM budget are free, advanced in launches shared with every other admitted request, and retired
when its true FP64 relative residual reaches the tolerance.  Latency = completion - arrival.

`one_at_a_time` runs the same timeline through single FP64 solves in arrival order (the baseline).
"""
from __future__ import annotations

import ctypes
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import BCS, PRECISIONS, Problem, _lib
from ._lib import PcbDesc, PcbServerDone, PcbServerOpts, check


@dataclass
class Completed:
    tag: int
    status: int
    iterations: int
    refinements: int
    relres: float
    done_s: float


class Server:
    def __init__(self, budget_bytes: int, max_slots: int = 32, precision: str = "mixed", tol: float = 1e-8,
                 maxit: int = 500, restart: int = 16, stream: torch.cuda.Stream | None = None):
        self.lib = _lib.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o = PcbServerOpts(int(budget_bytes), int(max_slots), PRECISIONS[precision], float(tol), int(maxit),
                          int(restart), ctypes.c_void_p(self.stream.cuda_stream))
        h = ctypes.c_void_p()
        check("pcb_server_create", self.lib.pcb_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        self._buf = (PcbServerDone * 256)()
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.pcb_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, N, n, theta, gamma, rhs_host: torch.Tensor, x_host: torch.Tensor, tag: int, T=1.0,
               bc="dirichlet", a=1.0):
        d = PcbDesc(int(N), int(n), float(theta), float(T), float(gamma), math.pi, None, 0, 2, None, BCS[bc],
                    float(a))
        self._keep[tag] = (rhs_host, x_host)
        check("pcb_server_submit", self.lib.pcb_server_submit(self.h, ctypes.byref(d), rhs_host.data_ptr(),
                                                              x_host.data_ptr(), int(tag)))

    def step(self):
        nd, na, nq = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check("pcb_server_step", self.lib.pcb_server_step(self.h, self._buf, len(self._buf), ctypes.byref(nd),
                                                          ctypes.byref(na), ctypes.byref(nq)))
        now = time.perf_counter()
        out = []
        for k in range(nd.value):
            r = self._buf[k]
            out.append(Completed(r.tag, r.status, r.iterations, r.refinements, r.relres, now))
            self._keep.pop(r.tag, None)
        return out, na.value, nq.value


@dataclass
class Request:
    tag: int
    arrival_s: float
    N: int
    n: int
    theta: float
    gamma: float
    rhs: torch.Tensor          # pinned host, the system's right-hand side
    x: torch.Tensor = None     # pinned host output
    bc: str = "dirichlet"      # "neumann": Example 3's grid, GMRES-P_S
    a: float = 1.0             # constant coefficient


def run(requests: list[Request], budget_bytes: int, max_slots: int = 32, precision: str = "mixed",
        tol: float = 1e-8, restart: int = 16) -> dict:
    """Serve the timeline; returns throughput and latency statistics."""
    srv = Server(budget_bytes, max_slots, precision, tol, restart=restart)
    pending = sorted(requests, key=lambda r: r.arrival_s)
    for r in pending:
        r.x = torch.empty_like(r.rhs).pin_memory() if r.x is None else r.x
    by_tag = {r.tag: r for r in pending}
    done: dict[int, Completed] = {}
    t0 = time.perf_counter()
    nxt = 0
    active = queued = 0
    while len(done) < len(pending):
        now = time.perf_counter() - t0
        while nxt < len(pending) and pending[nxt].arrival_s <= now:
            r = pending[nxt]
            srv.submit(r.N, r.n, r.theta, r.gamma, r.rhs, r.x, r.tag, bc=r.bc, a=r.a)
            nxt += 1
        if active == 0 and queued == 0 and nxt < len(pending) and pending[nxt].arrival_s > now:
            time.sleep(min(0.001, pending[nxt].arrival_s - now))
        comp, active, queued = srv.step()
        for c in comp:
            done[c.tag] = c
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array([done[t].done_s - t0 - by_tag[t].arrival_s for t in by_tag])
    unk = sum(2 * r.N * r.N * r.n for r in pending)
    return {"requests": len(pending), "wall_s": wall, "solves_per_s": len(pending) / wall,
            "unknowns_per_s": unk / wall, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "max_relres": max(done[t].relres for t in by_tag),
            "failed": sum(done[t].status < 0 for t in by_tag), "results": done}


def one_at_a_time(requests: list[Request], precision: str = "fp64", tol: float = 1e-8, restart: int = 16) -> dict:
    """Baseline: the same timeline solved one request at a time in arrival order."""
    pending = sorted(requests, key=lambda r: r.arrival_s)
    t0 = time.perf_counter()
    lat = []
    for r in pending:
        now = time.perf_counter() - t0
        if r.arrival_s > now:
            time.sleep(r.arrival_s - now)
        pr = Problem(r.N, r.n, r.theta, r.gamma, precision=precision)
        x = torch.empty_like(r.rhs).pin_memory()
        pr.solve_host(r.rhs, x, tol=tol, restart=restart, allow_not_converged=True)
        pr.close()
        lat.append(time.perf_counter() - t0 - r.arrival_s)
    wall = time.perf_counter() - t0
    lat = np.array(lat)
    unk = sum(2 * r.N * r.N * r.n for r in pending)
    return {"requests": len(pending), "wall_s": wall, "solves_per_s": len(pending) / wall,
            "unknowns_per_s": unk / wall, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99))}


def build_requests(trace, time_scale: float = 1.0) -> list[Request]:
    """Requests from a synth.serving_trace: the right-hand side of each instance is assembled on the
    device by the library (pcb_assemble_rhs) and kept in pinned host memory."""
    import synth
    out = []
    for q in trace:
        inst = q.inst
        g = synth.random_target(inst.N, inst.n, seed=inst._gseed)
        f = synth.manufactured_source(inst.N, inst.n)
        pr = Problem(inst.N, inst.n, inst.theta, inst.gamma)
        b = pr.assemble_rhs(torch.from_numpy(g.ravel()).cuda(), torch.from_numpy(f.ravel()).cuda(),
                            op="A" if inst.theta == 1.0 else "Ahat")
        rhs = b.cpu().pin_memory()
        pr.close()
        out.append(Request(q.rid, q.arrival_s * time_scale, inst.N, inst.n, inst.theta, inst.gamma, rhs))
    return out

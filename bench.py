#!/usr/bin/env python
"""Benchmark of the block omega-circulant preconditioned all-at-once solver on one GB300.

Workload (the paper's problem family at the large single-instance size): 2D heat tracking control
on the unit square, N = 511 (m = 261,121), n = 512 backward-Euler steps, T = 1, a(x) = 1,
gamma in {1e-2, 1e-6}, random smooth target g (seed 1) and analytic source f; 267,387,904 unknowns.
One step = one mixed-precision MINRES-|P_S| solve to true relative residual 1e-8 for each gamma
(two solves), inputs resident in HBM.  Metric: solves/s (higher is better).

Also reported: the same solves in plain FP64 on the GPU, an end-to-end figure through the host-buffer
C-ABI call (host->device copy of b and device->host copy of x inside the timed region), the
roofline of the preconditioner apply (the dominant kernel sequence) from CUDA events recorded on the
library's stream during the timed region, and the FP64 CPU oracle timed on the host cores.

Multi-GPU: every rank solves its own copy of the workload (independent problems, no data-path
collective: weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="heat-control N=511 n=512 backward-Euler a=1 (2.67e8 unknowns), gamma {1e-2,1e-6}",
                N=511, n=512, theta=1.0, T=1.0, gammas=(1e-2, 1e-6))
METRIC = "solves/s to relres 1e-8 (mixed-precision MINRES-|P_S|)"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "precond_apply_N511_n512.md")
# FP64 instructions per output value of the theta = 1 FP64 product with an epilogue (true
# residuals): the epilogue's scale folded into the operator's coefficients, ten operations
MV_FP64_OPS = 10.0
# bytes per unknown of the product with the MINRES epilogue: y and r1 read, the output written
MV_ALG_BYTES = 24.0


def args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the variable-a and uneven-batch figures")
    ap.add_argument("--serve-window", type=float, default=0.5,
                    help="seconds of the serving trace replayed for the serving figures (0: skip)")
    ap.add_argument("--small", action="store_true", help="N=255, n=256 instead (quick checks only)")
    ap.add_argument("--no-neumann", action="store_true", help="skip the Example 3 (Neumann) figures")
    ap.add_argument("--no-zeta-sweep", action="store_true", help="skip the omega = exp(i zeta) sweep")
    ap.add_argument("--no-omega-i", action="store_true", help="skip the omega = i run of the bench workload")
    ap.add_argument("--profile-apply", nargs=2, type=int, metavar=("N", "n"),
                    help="profiling mode: only run --prof-reps preconditioner applies (or products) on one "
                         "problem of this size, so that a profiler can capture single launches")
    ap.add_argument("--prof-prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--prof-kind", default="abs_ps", choices=["abs_ps", "ps", "pms", "matvec", "solve"])
    ap.add_argument("--prof-var-a", action="store_true", help="variable a(x) (config 2's): the multigrid route")
    ap.add_argument("--prof-fem", action="store_true", help="bilinear finite elements (M != I)")
    ap.add_argument("--prof-autotune", action="store_true", help="autotune the apply first (as the bench does)")
    ap.add_argument("--no-autotune", action="store_true", help="bench: keep the default kernel configuration")
    ap.add_argument("--prof-reps", type=int, default=3)
    ap.add_argument("--prof-theta", type=float, default=1.0, help="theta of the profiled problem (not --prof-neumann)")
    ap.add_argument("--prof-zeta", type=float, default=math.pi)
    ap.add_argument("--prof-neumann", action="store_true", help="Example 3's Neumann grid (DCT-I passes, kind ps)")
    return ap.parse_args()


class Nvtx:
    """An NVTX range around a region, so that an ncu launch list can select it (`--nvtx
    --nvtx-include <name>/`); a no-op where torch was built without NVTX."""

    def __init__(self, torch, name):
        self.torch, self.name = torch, name

    def __enter__(self):
        try:
            self.torch.cuda.nvtx.range_push(self.name)
            self.on = True
        except Exception:
            self.on = False
        return self

    def __exit__(self, *exc):
        if self.on:
            self.torch.cuda.nvtx.range_pop()
        return False


def profile_apply(a):
    """--profile-apply N n: a few applies of one kind (or products) on one problem, nothing else.
    With --prof-neumann the problem is Example 3's (N nodes per side with the boundary, a = 1e-3,
    Crank-Nicolson); --prof-zeta sets omega = exp(i zeta)."""
    import torch
    import paper_2406_00952_gb300 as P
    from paper_2406_00952_gb300 import _build
    _build.build()
    N, n = a.profile_apply
    if a.prof_neumann:
        gp = P.Problem(N, n, 0.5, 1e-2, precision=a.prof_prec, bc="neumann", a=1e-3)
    elif a.prof_var_a:
        import synth
        gp = P.Problem(N, n, a.prof_theta, 1e-2, a_edges=synth.variable_coefficient_edges(N), precision=a.prof_prec)
    else:
        gp = P.Problem(N, n, a.prof_theta, 1e-2, zeta=a.prof_zeta, precision=a.prof_prec, fem=a.prof_fem)
    if a.prof_autotune:
        print("autotune", gp.autotune(kind=None if a.prof_kind in ("solve", "matvec") else a.prof_kind))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(gp.size, dtype=torch.float64, device="cuda", generator=g)
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    with Nvtx(torch, "measured"):  # the launches below, without set-up and tuning
        if a.prof_kind == "solve":     # Krylov iterations (MINRES for theta = 1, else (F)GMRES), no graphs
            gp.solve(x, y, fixed_iterations=a.prof_reps, graphs=False)
        for _ in range(a.prof_reps if a.prof_kind != "solve" else 0):
            if a.prof_kind == "matvec":
                gp.matvec(x, out=y)
            else:
                gp.precond_apply(x, out=y, kind=a.prof_kind, precision=a.prof_prec)
        torch.cuda.synchronize()
    print("ok", N, n, a.prof_prec, a.prof_kind, a.prof_reps)


def replica_plan(world: int, rank: int, gammas) -> list:
    """Weak scaling: every rank solves its own full copy of the workload (independent problems, no
    data-path exchange); returns the (rank, gamma) solves this rank owns."""
    return [(rank, g) for g in gammas]


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """Timing reduction across ranks (the only collective: measurement, not data path)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush(); self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def profile_traffic():
    """DRAM bytes per preconditioner apply from the committed ncu summary, if it still matches the
    kernel source (its source hash); else None."""
    try:
        import hashlib
        txt = open(PROFILE_TRAFFIC).read()
        want = None; traffic = None
        for line in txt.splitlines():
            if line.startswith("source_sha256:"):
                want = line.split(":", 1)[1].strip()
            if line.startswith("traffic_bytes_per_apply:"):
                traffic = float(line.split(":", 1)[1].strip())
        h = hashlib.sha256()
        for f in ("fft_reg.cuh", "precond.cu", "precond_pipe.cu", "pcb_internal.cuh"):
            h.update(open(os.path.join(ROOT, "paper_2406_00952_gb300", "csrc", f), "rb").read())
        return traffic if (want == h.hexdigest() and traffic) else None
    except Exception:
        return None


SAMPLE_STEPS = 64     # time steps of the oracle's bounded sample (of the workload's 512)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_iterations(W):
    """FP64 oracle MINRES-|P_S| iteration counts on the full workload, per gamma, written by
    oracle/count_iterations.py (a full-size oracle run); {} if that file is absent."""
    p = os.path.join(ROOT, "tests", "golden", f"oracle_iterations_N{W['N']}_n{W['n']}.txt")
    out = {}
    try:
        for line in open(p):
            if line.strip() and not line.startswith("#"):
                g, secs, its = line.split()
                out[float(g)] = int(its)
    except Exception:
        return {}
    return out


def oracle_sample(W, workers):
    """The oracle as it stands, on a bounded sample of the workload: one MINRES-|P_S| iteration's
    operator work (one |P_S|^-1 apply and one product A x, the dominant cost of an iteration) on the
    workload's own grid (N = 511, gamma = 1e-2) with 64 of its 512 time steps, the library FFTs on
    `workers` host threads (scipy.fft.set_workers; the oracle's code is unchanged).  Returns the
    measured seconds of the sample and the seconds it scales to for one full-size iteration
    (x 512/64: the oracle's work per unknown is nearly independent of n; the full-size figure in
    tests/golden/oracle_iterations_N511_n512.txt, 84 s per iteration on one core, checks it)."""
    import numpy as np
    import scipy.fft
    from oracle import discretisation as ds
    from oracle import operators as op
    from oracle import precond as pc
    N, n = W["N"], SAMPLE_STEPS
    prob = ds.Problem(N, n, W["theta"], W["gammas"][0], W["T"])
    v = np.random.default_rng(0).standard_normal(2 * prob.m * n)
    with scipy.fft.set_workers(workers):
        t0 = time.perf_counter()
        pc.apply_abs_ps_inv(prob, v)
        op.matvec_A(prob, v)
        dt = time.perf_counter() - t0
    return dt, dt * W["n"] / n


def cpu_solves_per_s(W, t_iter):
    """Solves/s of the oracle on the workload (one solve per gamma) from the full-size time of one
    iteration and the oracle's own full-size iteration count for each gamma."""
    its = oracle_iterations(W)
    n_its = [its.get(g) for g in W["gammas"]]
    if not all(n_its):
        return None, n_its
    return len(W["gammas"]) / (t_iter * sum(n_its)), n_its


def cpu_baseline(W):
    """The oracle on all host cores, and beside it on one core (the same sample)."""
    workers = host_cores()
    dt, t_iter = oracle_sample(W, workers)
    val, n_its = cpu_solves_per_s(W, t_iter)
    dt1, t_iter1 = oracle_sample(W, 1)
    val1, _ = cpu_solves_per_s(W, t_iter1)
    return {"value": val, "unit": "solves/s", "cores": workers, "kind": "oracle",
            "sample": f"one oracle MINRES-|P_S| iteration's operator work (|P_S|^-1 apply + A x) at N=511 with "
                      f"{SAMPLE_STEPS} of the 512 time steps, {dt:.1f} s measured on {workers} host threads; scaled "
                      f"x{W['n'] // SAMPLE_STEPS} to {t_iter:.1f} s per full-size iteration, x the oracle's own "
                      f"full-size iteration counts {n_its} (gamma {list(W['gammas'])})",
            "single_core": {"value": val1, "unit": "solves/s", "cores": 1,
                            "sample": f"the same sample on one thread: {dt1:.1f} s, {t_iter1:.1f} s per full-size "
                                      f"iteration"}}


def reference_arm(a, W, rank, world):
    """--impl reference: the FP64 oracle (CPU) as it stands, on the host cores; each step is one
    bounded sample (oracle_sample) of the workload, and the line's value is the solves/s it scales
    to (cpu_solves_per_s).  Under torchrun only rank 0 runs."""
    if rank != 0:
        return
    workers = host_cores()
    times = []
    for s in range(a.warmup + a.steps):
        dt, t_iter = oracle_sample(W, workers)
        if s >= a.warmup:
            times.append((dt, t_iter))
    dt = statistics.median(t for t, _ in times)
    t_iter = statistics.median(t for _, t in times)
    val, n_its = cpu_solves_per_s(W, t_iter)
    sample = (f"per step: one oracle MINRES-|P_S| iteration's operator work (|P_S|^-1 apply + A x) at N=511 with "
              f"{SAMPLE_STEPS} of the 512 time steps on {workers} host threads ({dt:.1f} s median); value = solves/s "
              f"scaled x{W['n'] // SAMPLE_STEPS} to {t_iter:.1f} s per full-size iteration and x the oracle's own "
              f"full-size iteration counts {n_its}")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"], "sample": sample},
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


GOLDEN = os.path.join(ROOT, "tests", "golden")


def solution_sample(tag):
    """(size, positions, values) of an FP64 oracle solution sample stored in tests/golden (a data
    file the oracle's reference_solutions script writes), or None."""
    import numpy as np
    p = os.path.join(GOLDEN, f"solution_sample_{tag}.txt")
    if not os.path.exists(p):
        return None
    size, pos, val = None, [], []
    for line in open(p):
        if line.startswith("#") or not line.strip():
            continue
        a_, b_ = line.split()
        if a_ == "size":
            size = int(b_)
        elif a_ != "norm2":
            pos.append(int(a_)); val.append(float(b_))
    return size, np.array(pos), np.array(val)


def forward_error(tag, x):
    """||x[S] - x*[S]|| / ||x*[S]|| on the stored positions S of the oracle solution x* (tag), read
    from the device without copying the whole vector; None without a stored sample."""
    import numpy as np
    import torch
    s = solution_sample(tag)
    if s is None or x.numel() != s[0]:
        return None
    xs = x[torch.from_numpy(s[1]).to(x.device)].cpu().numpy()
    return float(np.linalg.norm(xs - s[2]) / np.linalg.norm(s[2]))


def timed(torch, stream, fn, reps=1):
    """Mean milliseconds of fn() over reps calls, CUDA events on `stream` (after the caller's warm-up)."""
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = [fn() for _ in range(reps)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def config2_figures(P, synth, torch, stream):
    """The variable-coefficient Crank-Nicolson workload (N = 255, n = 256, gamma = 1e-4,
    a = 1 + 0.5 sin sin): FGMRES(30) with two multigrid V-cycles per shifted solve, mixed (FP32
    multigrid) and FP64, to relres 1e-8; solve time from CUDA events after one warm-up solve."""
    inst = synth.config2()
    out = {"workload": f"N={inst.N} n={inst.n} Crank-Nicolson gamma={inst.gamma:g} a=1+0.5 sin(pi x1) sin(pi x2), "
                       "FGMRES(30) + 2 V-cycles", "unknowns": 2 * inst.N * inst.N * inst.n}
    g = torch.from_numpy(inst.g.ravel()).cuda(); f = torch.from_numpy(inst.f.ravel()).cuda()
    its = {}
    for prec in ("mixed", "fp64"):
        pr = P.Problem(inst.N, inst.n, inst.theta, inst.gamma, a_edges=inst.a_edges, mg_cycles=2, precision=prec,
                       stream=stream)
        b = pr.assemble_rhs(g, f, op="Ahat")
        x = pr._empty()
        pr.solve(b, x, tol=1e-8)
        ms, infos = timed(torch, stream, lambda: pr.solve(b, x, tol=1e-8)[1])
        its[prec] = infos[-1]["iterations"]
        out[prec] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": its[prec],
                     "relres": infos[-1]["relres"], "forward_error_vs_oracle": forward_error("cfg2", x)}
        pr.close(); del b, x
    out["within_plus2"] = its["mixed"] <= its["fp64"] + 2
    return out


def config3_figures(P, synth, torch, stream):
    """The uneven batch: 64 independent problems (N in {63..255}, n in {32..256}, theta in {1, 1/2},
    gamma log-uniform in [1e-6, 1e-1]) solved in mixed precision to relres 1e-8 with shared launches
    (pcb_batch_solve), against the same problems one at a time (mixed and FP64)."""
    insts = synth.config3()
    probs, bs = [], []
    for inst in insts:
        pr = P.Problem(inst.N, inst.n, inst.theta, inst.gamma, precision="mixed", stream=stream)
        probs.append(pr)
        bs.append(pr.assemble_rhs(torch.from_numpy(inst.g.ravel()).cuda(), torch.from_numpy(inst.f.ravel()).cuda(),
                                  op="A" if inst.theta == 1.0 else "Ahat"))
    unknowns = sum(p.size for p in probs)
    xs = [p._empty() for p in probs]
    P.batch_solve(probs, bs, xs, tol=1e-8, restart=16)
    ms_b, res = timed(torch, stream, lambda: P.batch_solve(probs, bs, xs, tol=1e-8, restart=16)[1])
    infos = res[-1]
    errs = {k: forward_error(f"cfg3_{k}", xs[k]) for k in (0, 2, 3, 4)}
    ms_1, _ = timed(torch, stream, lambda: [p.solve(b, x, tol=1e-8, restart=16) for p, b, x in zip(probs, bs, xs)])
    fp = [P.Problem(i.N, i.n, i.theta, i.gamma, precision="fp64", stream=stream) for i in insts]
    its64 = [p.solve(b, x, tol=1e-8, restart=16)[1]["iterations"] for p, b, x in zip(fp, bs, xs)]
    ms_64, _ = timed(torch, stream, lambda: [p.solve(b, x, tol=1e-8, restart=16) for p, b, x in zip(fp, bs, xs)])
    itsm = [i["iterations"] for i in infos]
    for p in fp:
        p.close()
    # autotuned kernel shapes: each problem tunes its apply (shapes seen before reuse the choice)
    tuned = [p.autotune(reps=2) for p in probs]
    P.batch_solve(probs, bs, xs, tol=1e-8, restart=16)
    ms_t, _ = timed(torch, stream, lambda: P.batch_solve(probs, bs, xs, tol=1e-8, restart=16)[1])
    for p in probs:
        p.close()
    return {"workload": f"{len(insts)} uneven instances (synth.config3), {unknowns:.3g} unknowns in all, mixed",
            "batched": {"solves_per_s": len(insts) / (ms_b / 1e3), "unknowns_per_s": unknowns / (ms_b / 1e3),
                        "ms": ms_b, "max_relres": max(i["relres"] for i in infos)},
            "batched_autotuned": {"solves_per_s": len(insts) / (ms_t / 1e3), "ms": ms_t,
                                  "non_default_choices": sum(t["chosen"] != 0 for t in tuned),
                                  "rejected": sum(t["rejected"] for t in tuned),
                                  "apply_ms_default_sum": sum(t["default_ms"] for t in tuned),
                                  "apply_ms_tuned_sum": sum(t["best_ms"] for t in tuned)},
            "one_at_a_time_mixed": {"solves_per_s": len(insts) / (ms_1 / 1e3), "ms": ms_1},
            "one_at_a_time_fp64": {"solves_per_s": len(insts) / (ms_64 / 1e3), "ms": ms_64},
            "iterations_mixed_minus_fp64_max": max(m - f for m, f in zip(itsm, its64)),
            "within_plus2_count": sum(m <= f + 2 for m, f in zip(itsm, its64)),
            "forward_error_vs_oracle_sample": errs}


def serving_figures(synth, torch, window):
    """A window of the serving trace (Poisson arrivals at 200/s; 95% of requests sized like the
    uneven batch, 5% at N = 511, n = 512; random g and gamma), served by the continuous-batching
    server in mixed precision under a 150 GB budget, against single FP64 solves in arrival order.
    The offered 200/s exceeds what one GPU sustains, so the same requests are also replayed at
    the sustained rate (arrivals slowed to 90% of the measured throughput) for steady-state
    latencies."""
    from paper_2406_00952_gb300 import serve
    trace = synth.serving_trace(duration_s=window)
    reqs = serve.build_requests(trace)
    torch.cuda.synchronize()
    srv = serve.run(reqs, budget_bytes=150 << 30, max_slots=32, precision="mixed")
    rate = srv["solves_per_s"]
    scale = 200.0 / (0.9 * rate)
    for r in reqs:
        r.x = None
    for r, q in zip(reqs, trace):
        r.arrival_s = q.arrival_s * scale
    steady = serve.run(reqs, budget_bytes=150 << 30, max_slots=32, precision="mixed")
    for r, q in zip(reqs, trace):
        r.arrival_s = q.arrival_s
    base = serve.one_at_a_time(reqs, precision="fp64")
    keys = ("solves_per_s", "p50_latency_s", "p99_latency_s")
    return {"trace": f"Poisson 200/s, first {window:g} s ({len(reqs)} requests, {sum(r.N == 511 for r in reqs)} at "
                     f"N=511 n=512), HBM budget 150 GB", "offered_rate_hz": 200.0,
            "solves_per_s": srv["solves_per_s"], "p50_latency_s": srv["p50_latency_s"],
            "p99_latency_s": srv["p99_latency_s"], "max_relres": srv["max_relres"], "failed": srv["failed"],
            "sustained": {"arrival_rate_hz": 200.0 / scale, **{k: steady[k] for k in keys},
                          "failed": steady["failed"]},
            "fp64_one_at_a_time": {k: base[k] for k in keys}}


def neumann_figures(P, synth, np, torch, stream, steps):
    """Mixed and FP64 GMRES-P_S on Example 3 (N = 257 nodes, n = 256), timed with CUDA events after
    one warm-up solve; e_h against the exact solution; the FP32 P_S apply against the HBM roofline."""
    N = 257; n = 256; gam = 1e-2
    g, f, ye, pe = synth.example3_data(N, n)
    out = {"workload": f"Example 3 Neumann N={N} nodes (h=1/256) n={n} CN a=1e-3 gamma={gam:g}",
           "unknowns": 2 * N * N * n}
    gd = torch.from_numpy(g.ravel()).cuda(); fd = torch.from_numpy(f.ravel()).cuda()
    y0 = torch.from_numpy(np.ascontiguousarray(ye[0])).cuda()
    hbm, _ = peaks()
    for prec in ("mixed", "fp64"):
        pr = P.Problem(N, n, 0.5, gam, precision=prec, stream=stream, bc="neumann", a=1e-3)
        b = pr.assemble_rhs(gd, fd, y0, op="Ahat")
        x = pr._empty()
        pr.solve(b, x, tol=1e-8)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [pr.solve(b, x, tol=1e-8, profile=True)[1] for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        y, p = pr.recover(x)
        ey = y.cpu().numpy().reshape(n, -1) - ye[1:]
        ep = p.cpu().numpy().reshape(n, -1) - pe[:-1]
        eh = float((np.sqrt((ey ** 2).sum(1) + (ep ** 2).sum(1)) / (N - 1)).max())
        applies = sum(i["precond_applies"] for i in infos); pms = sum(i["precond_ms"] for i in infos)
        out[prec] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": infos[-1]["iterations"],
                     "relres": infos[-1]["relres"], "e_h": eh, "precond_avg_ms": pms / applies}
        if prec == "mixed":
            ach = 16.0 * out["unknowns"] / (pms / applies / 1e3) / 1e9
            out["precond_roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                                       "frac": ach / hbm, "kernel": "P_S^-1 apply, DCT-I passes (FP32)"}
        pr.close(); del b, x, y, p
    return out


def zeta_sweep(P, synth, torch, stream):
    """Mixed MINRES-|P_S| on the bench family at N = 255, n = 256 (gamma = 1e-2) for several
    omega = exp(i zeta): the choice the paper settled on (zeta = pi) against the circulant
    (zeta = 0) and intermediate values; iterations and solve time (CUDA events)."""
    N, n, gam = 255, 256, 1e-2
    g = torch.from_numpy(synth.random_target(N, n, seed=1).ravel()).cuda()
    f = torch.from_numpy(synth.manufactured_source(N, n).ravel()).cuda()
    rows = []
    for zeta in (0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4, math.pi):
        pr = P.Problem(N, n, 1.0, gam, zeta=zeta, precision="mixed", stream=stream)
        b = pr.assemble_rhs(g, f)
        x = pr._empty()
        pr.solve(b, x, tol=1e-8)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = pr.solve(b, x, tol=1e-8)
        e1.record(stream)
        torch.cuda.synchronize()
        rows.append({"zeta": round(zeta, 6), "iterations": info["iterations"], "ms_per_solve": e0.elapsed_time(e1),
                     "relres": info["relres"]})
        pr.close(); del b, x
    return {"workload": f"heat-control N={N} n={n} backward-Euler a=1 gamma={gam:g}, mixed MINRES-|P_S|",
            "rows": rows}


def omega_i_figures(P, torch, stream, W, g, f, steps):
    """The bench workload with omega = i (zeta = pi/2) instead of the paper's -1: under the
    real-part reading the preconditioner is the mean of the omega = i and omega = -i ones.  Mixed
    step (both gamma) timed with CUDA events like the headline, and one FP64 solve per gamma."""
    N, n = W["N"], W["n"]
    probs, bs = [], []
    for gam in W["gammas"]:
        pr = P.Problem(N, n, W["theta"], gam, W["T"], zeta=math.pi / 2, precision="mixed", stream=stream)
        probs.append(pr)
        bs.append(pr.assemble_rhs(g, f))
    xs = [pr._empty() for pr in probs]
    for pr, b, x in zip(probs, bs, xs):
        pr.solve(b, x, tol=1e-8, maxit=400)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    its = []
    for _ in range(steps):
        for pr, b, x in zip(probs, bs, xs):
            its.append(pr.solve(b, x, tol=1e-8, maxit=400)[1]["iterations"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    fp = []
    for gam, b in zip(W["gammas"], bs):
        pr = P.Problem(N, n, W["theta"], gam, W["T"], zeta=math.pi / 2, precision="fp64", stream=stream)
        x = pr._empty()
        torch.cuda.synchronize(); t0 = time.perf_counter()
        _, inf = pr.solve(b, x, tol=1e-8, maxit=400)
        torch.cuda.synchronize()
        fp.append({"iterations": inf["iterations"], "s": time.perf_counter() - t0})
        pr.close(); del x
    for pr in probs:
        pr.close()
    return {"zeta": math.pi / 2, "workload": W["name"], "mixed": {"solves_per_s": len(W["gammas"]) / (ms / 1e3),
            "ms_per_step": ms, "iterations": its[:len(W["gammas"])]},
            "fp64_gpu": {"solves_per_s": len(fp) / sum(r["s"] for r in fp), "iterations": [r["iterations"] for r in fp]}}


def main():
    a = args()
    rank = int(os.environ.get("RANK", 0)); world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    W = dict(WORKLOAD)
    if a.small:
        W.update(N=255, n=256, name="heat-control N=255 n=256 backward-Euler a=1, gamma {1e-2,1e-6}")
    if a.impl == "reference":
        return reference_arm(a, W, rank, world)
    if a.profile_apply:
        return profile_apply(a)

    import numpy as np
    import torch

    import synth
    import paper_2406_00952_gb300 as P
    from paper_2406_00952_gb300 import _build
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    N, n = W["N"], W["n"]
    stream = torch.cuda.current_stream()
    probs, bs = [], []
    g = torch.from_numpy(synth.random_target(N, n, seed=1).ravel()).cuda()
    f = torch.from_numpy(synth.manufactured_source(N, n).ravel()).cuda()
    for gam in W["gammas"]:
        pr = P.Problem(N, n, W["theta"], gam, W["T"], precision="mixed", stream=stream)
        probs.append(pr)
        bs.append(pr.assemble_rhs(g, f))
    gf = (g, f)
    del g, f
    # autotuned kernel shapes: the first problem times the candidate configurations
    # of its preconditioner apply and keeps the fastest; the second, of the same shape, inherits it
    tune = None if a.no_autotune else probs[0].autotune(reps=3)
    if tune is not None:
        probs[1:] = [P.Problem(N, n, W["theta"], gam, W["T"], precision="mixed", stream=stream)
                     for gam in W["gammas"][1:]]
    xs = [pr._empty() for pr in probs]
    unknowns = probs[0].size
    opts = dict(tol=1e-8, maxit=400)

    def step(profile=False):
        infos = []
        for pr, b, x in zip(probs, bs, xs):
            _, info = pr.solve(b, x, profile=profile, **opts)
            infos.append(info)
        return infos

    for _ in range(a.warmup):
        step()
    barrier()
    clk = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    with Nvtx(torch, "timed"):
        e0.record(stream)
        infos = []
        for _ in range(a.steps):
            infos += step()
        e1.record(stream)
        torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, device="cuda")
    barrier()
    solves = len(replica_plan(world, rank, W["gammas"])) * a.steps * world
    value = solves / (ms / 1e3)
    hbm, peak_kind = peaks()
    # kernel figures: one more step, untimed, with CUDA events around every preconditioner apply
    # and product (profiling launches each MINRES iteration directly instead of from its graph)
    p0 = torch.cuda.Event(enable_timing=True); p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    pinfos = step(profile=True)
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms = p0.elapsed_time(p1)
    applies = sum(i["precond_applies"] for i in pinfos)
    pms = sum(i["precond_ms"] for i in pinfos)
    mvs = sum(i["matvecs"] for i in pinfos)
    mvms = sum(i["matvec_ms"] for i in pinfos)
    # the inner iterations' products (two-word FP32 arithmetic) and the FP64 true-residual products
    mvi = sum(i["matvecs_inner"] for i in pinfos)
    mvims = sum(i["matvec_inner_ms"] for i in pinfos)
    mvr, mvrms = mvs - mvi, mvms - mvims
    alg_bytes = 16.0 * unknowns            # precond apply: read 2mn + write 2mn FP64 values
    achieved = alg_bytes / (pms / applies / 1e3) / 1e9
    iters = [i["iterations"] for i in infos]
    fp64r = P.fp64_rates(stream)
    fp64_peak = fp64r["fma_per_s"]
    # forward error of the mixed solutions against the oracle's (sampled positions, relres 1e-12 truth)
    fe_mixed = [forward_error(f"cfg1_g{gam:g}", x) for gam, x in zip(W["gammas"], xs)] if not a.small else None

    # plain FP64 GPU solver on the same inputs (one solve per gamma)
    fp64 = None
    if not a.no_fp64:
        t_fp = 0.0; it_fp = []; fe_fp = []
        for gam, b in zip(W["gammas"], bs):
            pr = P.Problem(N, n, W["theta"], gam, W["T"], precision="fp64", stream=stream)
            x = pr._empty()
            pr.solve(b, x, **opts)            # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, inf = pr.solve(b, x, **opts)
            torch.cuda.synchronize()
            t_fp += time.perf_counter() - t0
            it_fp.append(inf["iterations"])
            fe_fp.append(forward_error(f"cfg1_g{gam:g}", x))
            pr.close(); del x
        fp64 = {"value": len(W["gammas"]) / t_fp, "unit": "solves/s", "iterations": it_fp,
                "forward_error_vs_oracle": fe_fp}

    # end to end through the host-buffer C-ABI call: b from pinned host memory, x back to host
    e2e = None
    if a.e2e_steps > 0:
        bh = [b.cpu().pin_memory() for b in bs]
        xh = [torch.empty_like(h).pin_memory() for h in bh]
        for pr, b_, x_ in zip(probs, bh, xh):
            pr.solve_host(b_, x_, **opts)
        barrier()
        t0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            for pr, b_, x_ in zip(probs, bh, xh):
                pr.solve_host(b_, x_, **opts)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        nb = 8 * unknowns
        e2e = {"value": len(W["gammas"]) * a.e2e_steps * world / dt, "unit": "solves/s",
               "h2d_bytes_per_step": nb * len(W["gammas"]), "d2h_bytes_per_step": nb * len(W["gammas"])}

    # serving: a window of the Poisson request trace, served by the continuous-batching server
    serving = None
    if rank == 0 and a.serve_window > 0:
        serving = serving_figures(synth, torch, a.serve_window)
    cfg2 = config2_figures(P, synth, torch, stream) if rank == 0 and not a.no_configs else None
    cfg3 = config3_figures(P, synth, torch, stream) if rank == 0 and not a.no_configs else None

    # Example 3 (homogeneous Neumann, a = 1e-3, Crank-Nicolson, gamma = 1e-2) at the size of
    # Table 4's finest row: 257 nodes per side (h = 1/256), n = 256, GMRES-P_S with the DCT-I passes
    neumann = None
    if rank == 0 and not a.no_neumann:
        neumann = neumann_figures(P, synth, np, torch, stream, a.steps)
    zsweep = None
    if rank == 0 and not a.no_zeta_sweep:
        zsweep = zeta_sweep(P, synth, torch, stream)
    omega_i = None
    if rank == 0 and not a.no_omega_i:
        omega_i = omega_i_figures(P, torch, stream, W, gf[0], gf[1], a.steps)
    del gf

    cpu = None
    if rank == 0 and not a.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(W)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": W["name"], "unknowns": unknowns, "solver": "MINRES-|P_S| mixed",
                       "tol": 1e-8, "l2": "inputs larger than L2 (2.1 GB vectors)", "parallelism": f"replicas x{world}",
                       "iterations": iters},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": profile_traffic(), "kernel": "precond apply |P_S|^-1 (FP32)",
                         "alg_bytes_per_launch": alg_bytes, "avg_ms": pms / applies, "peak_kind": peak_kind},
            "kernels": {"precond_ms_share": pms / prof_ms, "matvec_ms_share": mvms / prof_ms,
                        # the inner iterations' product (k_matvec_tw, two-word FP32 arithmetic with the
                        # MINRES epilogue): MV_ALG_BYTES per unknown against the copy bandwidth
                        "matvec_roofline": {"bound": "hbm", "kernel": "MINRES product, two-word FP32 (inner iterations)",
                                            "launches": mvi, "avg_ms": mvims / mvi if mvi else None,
                                            "alg_bytes_per_unknown": MV_ALG_BYTES,
                                            "achieved": MV_ALG_BYTES * unknowns / (mvims / mvi / 1e3) / 1e9 if mvi else None,
                                            "peak": hbm, "unit": "GB/s", "peak_kind": peak_kind,
                                            "frac": MV_ALG_BYTES * unknowns / (mvims / mvi / 1e3) / 1e9 / hbm if mvi else None},
                        # the true-residual products stay FP64 and are bound by FP64 issue: MV_FP64_OPS
                        # FP64 instructions per unknown against this device's FP64 FMA instruction
                        # rate, measured here (pcb_measure_fp64_rates)
                        "residual_product_roofline": {"bound": "alu", "unit": "G FP64 instr/s", "launches": mvr,
                                                      "avg_ms": mvrms / mvr if mvr else None,
                                                      "fp64_instr_per_unknown": MV_FP64_OPS,
                                                      "achieved": MV_FP64_OPS * unknowns / (mvrms / mvr / 1e3) / 1e9 if mvr else None,
                                                      "peak": fp64_peak / 1e9, "peak_kind": "measured (FP64 FMA rate)",
                                                      "frac": MV_FP64_OPS * unknowns / (mvrms / mvr / 1e3) / fp64_peak if mvr else None,
                                                      "fp64_add_instr_per_s": fp64r["add_per_s"]}},
            "fp64_gpu": fp64,
            "mixed_vs_fp64": [{"gamma": gam, "mixed_iterations": im, "fp64_iterations": i64,
                               "within_plus2": im <= i64 + 2, "mixed_forward_error_vs_oracle": fe}
                              for gam, im, i64, fe in zip(W["gammas"], iters[:len(W["gammas"])],
                                                          fp64["iterations"] if fp64 else [None] * len(W["gammas"]),
                                                          fe_mixed or [None] * len(W["gammas"]))] if fp64 else None,
            "autotune": tune,
            "config2_variable_a": cfg2,
            "config3_uneven_batch": cfg3,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": sum(i["launches"] for i in infos),
            "serving": serving,
            "neumann": neumann,
            "zeta_sweep": zsweep,
            "omega_i": omega_i,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

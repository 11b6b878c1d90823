"""Write sampled FP64 oracle solutions of the benchmark workloads to tests/golden/, so that the GPU
results can be given a forward error against the oracle at sizes the oracle cannot re-solve
inside a test or a benchmark run.  Calls only the oracle (and the seeded input generators).

For each case the oracle solves its system to true relative residual 1e-12, or to the attainable
accuracy of float64 where that lies above it (no worse than 1e-10; the "truth" x*), with
the method the paper uses for it (Sec. 4): MINRES-|P_S| for backward Euler with a = 1,
FGMRES(30) with the multigrid P_S (two V-cycles, Lemma 3.14 decoupling) for the variable-a
Crank-Nicolson case, GMRES-P_S for Crank-Nicolson with a = 1.  The file keeps ||x*||_2, the count,
and x* at 1024 positions drawn from a fixed seed; a GPU solution x then has the sampled forward
error ||x[S] - x*[S]|| / ||x*[S]||.

    python -m oracle.reference_solutions [cfg1|cfg2|cfg3] [workers]

cfg1 (N = 511, n = 512, both gamma) takes about an hour and 30 GB of host memory; cfg2 (N = 255,
n = 256, multigrid) some minutes; cfg3 (four instances of the uneven batch) a minute.
"""
from __future__ import annotations

import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import discretisation as ds  # noqa: E402
from oracle import krylov as kr  # noqa: E402
from oracle import operators as op  # noqa: E402
from oracle import precond as pc  # noqa: E402

SAMPLES = 1024
GOLDEN = os.path.join(ROOT, "tests", "golden")
CFG3_SAMPLE = (0, 2, 3, 4)          # four instances of synth.config3() (three MINRES, one GMRES)


def sample_positions(size: int, seed: int = 2406) -> np.ndarray:
    return np.sort(np.random.default_rng(seed).choice(size, size=min(SAMPLES, size), replace=False))


def path_for(tag: str) -> str:
    return os.path.join(GOLDEN, f"solution_sample_{tag}.txt")


def solve(inst, tol=1e-12, accept=1e-10):
    """The oracle's solve of one instance; returns (x*, method, iterations, seconds)."""
    prob = ds.Problem.from_instance(inst)
    t0 = time.time()
    if inst.theta == 1.0 and inst.a_edges is None:
        b = ds.rhs_minres(prob, inst.g, inst.f)
        x, info = kr.minres(lambda z: op.matvec_A(prob, z), b, lambda r: pc.apply_abs_ps_inv(prob, r),
                            tol=tol, maxit=1000, stall=1e-3)
        method = "MINRES-|P_S|"
    elif inst.a_edges is None:
        b = ds.rhs_gmres(prob, inst.g, inst.f)
        x, info = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), b, lambda r: pc.apply_ps_inv(prob, r),
                            tol=tol, maxit=1000, restart=30, stall=1e-3)
        method = "GMRES(30)-P_S"
    else:
        b = ds.rhs_gmres(prob, inst.g, inst.f)
        x, info = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), b, lambda r: pc.apply_mg_ps_inv(prob, r, cycles=2),
                            tol=tol, maxit=1000, restart=30, stall=1e-3)
        method = "FGMRES(30)-P_S, 2 V-cycles"
    if not info.relres <= accept:
        raise RuntimeError(f"oracle did not converge on {inst.tag}: {info}")
    return x, method, info.iterations, time.time() - t0, info.relres


def write(tag: str, desc: str, inst, x, method, its, secs, relres):
    pos = sample_positions(x.size)
    lines = [f"# FP64 oracle solution sample: {desc}",
             f"# method {method}, true relative residual {relres:.3e} (target 1e-12), {its} iterations, {secs:.0f} s",
             "# written by oracle/reference_solutions.py; the positions come from numpy default_rng(2406)",
             f"size {x.size}", f"norm2 {float(np.linalg.norm(x)):.17g}", "# position value"]
    lines += [f"{int(p)} {x[p]:.17g}" for p in pos]
    with open(path_for(tag), "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(tag, method, its, f"{secs:.0f} s", flush=True)


def read(tag: str):
    """(size, ||x*||_2, positions, values) of a stored sample, or None."""
    p = path_for(tag)
    if not os.path.exists(p):
        return None
    size = norm = None
    pos, val = [], []
    for line in open(p):
        if line.startswith("#") or not line.strip():
            continue
        a, b = line.split()
        if a == "size":
            size = int(b)
        elif a == "norm2":
            norm = float(b)
        else:
            pos.append(int(a)); val.append(float(b))
    return size, norm, np.array(pos), np.array(val)


def sampled_forward_error(tag: str, x: np.ndarray):
    """||x[S] - x*[S]|| / ||x*[S]|| on the stored positions S (None without a stored sample)."""
    s = read(tag)
    if s is None:
        return None
    size, _, pos, val = s
    if x.size != size:
        raise ValueError(f"{tag}: size {x.size} != {size}")
    return float(np.linalg.norm(x[pos] - val) / np.linalg.norm(val))


def main(which="cfg2", workers=1):
    import scipy.fft
    with scipy.fft.set_workers(workers):
        if which == "cfg1":
            for gamma in (1e-2, 1e-6):
                inst = synth.config1(gamma)
                x, *rest = solve(inst)
                write(f"cfg1_g{gamma:g}", f"N=511 n=512 backward Euler a=1 gamma={gamma:g} (synth.config1)",
                      inst, x, *rest)
        elif which == "cfg2":
            inst = synth.config2()
            x, *rest = solve(inst)
            write("cfg2", "N=255 n=256 Crank-Nicolson gamma=1e-4 a=1+0.5 sin sin (synth.config2)", inst, x, *rest)
        elif which == "cfg3":
            insts = synth.config3()
            for k in CFG3_SAMPLE:
                inst = insts[k]
                x, *rest = solve(inst)
                write(f"cfg3_{k}", f"uneven batch instance {k}: N={inst.N} n={inst.n} theta={inst.theta:g} "
                      f"gamma={inst.gamma:.6g} (synth.config3)", inst, x, *rest)
        else:
            raise SystemExit(f"unknown case {which}")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "cfg2", int(sys.argv[2]) if len(sys.argv) > 2 else 1)

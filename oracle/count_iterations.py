"""Write the FP64 oracle's MINRES-|P_S| iteration count for the large backward-Euler workload
(N = 511, n = 512, gamma = 1e-2 and 1e-6, target g from seed 1, analytic source) to
tests/golden/oracle_iterations_N511_n512.txt.  Calls only the oracle; takes about an hour on one
core and ~40 GB of host memory.

    python -m oracle.count_iterations [N n]
"""
from __future__ import annotations

import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import discretisation as ds  # noqa: E402
from oracle import krylov as kr  # noqa: E402
from oracle import operators as op  # noqa: E402
from oracle import precond as pc  # noqa: E402


def main(N=511, n=512):
    out = os.path.join(ROOT, "tests", "golden", f"oracle_iterations_N{N}_n{n}.txt")
    lines = [f"# FP64 oracle MINRES-|P_S| iteration counts to true relative residual 1e-8, N={N}, n={n},",
             "# backward Euler, T=1, a=1, g = synth.random_target(seed=1), f = synth.manufactured_source.",
             "# written by oracle/count_iterations.py; columns: gamma seconds iterations"]
    for gamma in (1e-2, 1e-6):
        prob = ds.Problem(N, n, 1.0, gamma)
        b = ds.rhs_minres(prob, synth.random_target(N, n, seed=1), synth.manufactured_source(N, n))
        t0 = time.time()
        _, info = kr.minres(lambda z: op.matvec_A(prob, z), b, lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-8)
        lines.append(f"{gamma:g} {time.time() - t0:.0f} {info.iterations}")
        print(lines[-1], flush=True)
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    a = [int(v) for v in sys.argv[1:3]]
    main(*a)

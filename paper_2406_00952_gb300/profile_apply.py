"""Profiling driver: runs a few preconditioner applies (or operator products) on one problem so a
profiler can capture individual launches.

    python -m paper_2406_00952_gb300.profile_apply N n [mixed|fp64] [abs_ps|ps|pms|matvec] [repeats] [neumann|zeta=Z]

Each apply is five launches (x1-line DST, x2-line DST, time pass, x2-line DST, x1-line DST).
With `neumann` the problem is Example 3's (N nodes per side with the boundary, a = 1e-3,
Crank-Nicolson), whose applies run the DCT-I passes (kind ps); `zeta=Z` sets omega = exp(i Z).
"""
from __future__ import annotations

import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv):
    import paper_2406_00952_gb300 as P
    N, n = int(argv[0]), int(argv[1])
    prec = argv[2] if len(argv) > 2 else "mixed"
    kind = argv[3] if len(argv) > 3 else "abs_ps"
    reps = int(argv[4]) if len(argv) > 4 else 3
    if len(argv) > 5 and argv[5] == "neumann":
        gp = P.Problem(N, n, 0.5, 1e-2, precision=prec, bc="neumann", a=1e-3)
    elif len(argv) > 5 and argv[5].startswith("zeta="):
        gp = P.Problem(N, n, 1.0, 1e-2, zeta=float(argv[5][5:]), precision=prec)
    else:
        gp = P.Problem(N, n, 1.0, 1e-2, precision=prec)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(gp.size, dtype=torch.float64, device="cuda", generator=g)
    y = torch.empty_like(x)
    for _ in range(reps):
        if kind == "matvec":
            gp.matvec(x, out=y)
        else:
            gp.precond_apply(x, out=y, kind=kind, precision=prec)
    torch.cuda.synchronize()
    print("ok", N, n, prec, kind, reps)


if __name__ == "__main__":
    main(sys.argv[1:])

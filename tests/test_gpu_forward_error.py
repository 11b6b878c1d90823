"""Forward error of GPU solutions against the FP64 oracle's solutions of the benchmark workloads
(stored samples in tests/golden/solution_sample_*.txt, written by oracle/reference_solutions.py,
each x* solved to true relative residual 1e-12 or float64's attainable accuracy).  The error is
||x[S] - x*[S]|| / ||x*[S]|| over the 1024 stored positions S.

Bounds: a mixed-precision solve to relres 1e-8 within 1e-7 of x*; an FP64 GPU solve to relres
1e-10 within 1e-10 of x*.  The uneven batch is checked both batched and alone."""
import numpy as np
import pytest
import torch

import synth
from oracle import reference_solutions as rs

pytestmark = pytest.mark.gpu
CFG3 = rs.CFG3_SAMPLE


@pytest.fixture(scope="module")
def P():
    from paper_2406_00952_gb300 import _build
    _build.build()
    import paper_2406_00952_gb300 as P
    return P


def need(tag):
    if rs.read(tag) is None:
        pytest.skip(f"no stored oracle solution {tag}")


def fe(tag, x):
    return rs.sampled_forward_error(tag, x.cpu().numpy())


def rhs(pr, inst):
    g = torch.from_numpy(inst.g.ravel()).cuda(); f = torch.from_numpy(inst.f.ravel()).cuda()
    return pr.assemble_rhs(g, f, op="A" if inst.theta == 1.0 and inst.a_edges is None else "Ahat")


def test_uneven_batch_sample(P):
    insts = synth.config3()
    for k in CFG3:
        need(f"cfg3_{k}")
    probs = [P.Problem(i.N, i.n, i.theta, i.gamma, precision="mixed") for i in insts]
    bs = [rhs(p, i) for p, i in zip(probs, insts)]
    xs = [p._empty() for p in probs]
    P.batch_solve(probs, bs, xs, tol=1e-8, restart=16)
    for k in CFG3:
        e = fe(f"cfg3_{k}", xs[k])
        assert e <= 1e-7, ("batched", k, e)
    for k in CFG3:
        inst = insts[k]
        x, info = probs[k].solve(bs[k], tol=1e-8, restart=16)
        assert fe(f"cfg3_{k}", x) <= 1e-7, ("alone", k)
        g64 = P.Problem(inst.N, inst.n, inst.theta, inst.gamma, precision="fp64")
        x64, i64 = g64.solve(rhs(g64, inst), tol=1e-10, restart=30)
        e = fe(f"cfg3_{k}", x64)
        assert i64["relres"] <= 1e-10 and e <= 1e-10, ("fp64", k, e)
        g64.close()
    for p in probs:
        p.close()


def test_variable_coefficient_multigrid_workload(P):
    need("cfg2")
    inst = synth.config2()
    for prec, tol, bound in (("mixed", 1e-8, 1e-7), ("fp64", 1e-10, 1e-10)):
        pr = P.Problem(inst.N, inst.n, inst.theta, inst.gamma, a_edges=inst.a_edges, mg_cycles=2, precision=prec)
        x, info = pr.solve(rhs(pr, inst), tol=tol)
        e = fe("cfg2", x)
        assert info["relres"] <= tol and e <= bound, (prec, info, e)
        pr.close()


@pytest.mark.parametrize("gamma", [1e-2, 1e-6])
def test_large_single_instance(P, gamma):
    tag = f"cfg1_g{gamma:g}"
    need(tag)
    inst = synth.config1(gamma)
    for prec, tol, bound in (("mixed", 1e-8, 1e-7), ("fp64", 1e-10, 1e-10)):
        pr = P.Problem(inst.N, inst.n, inst.theta, inst.gamma, precision=prec)
        x, info = pr.solve(rhs(pr, inst), tol=tol)
        e = fe(tag, x)
        assert info["relres"] <= tol and e <= bound, (prec, info, e)
        pr.close()
        del x
        torch.cuda.empty_cache()

"""The autotuner (pcb_autotune): it times the preconditioner apply under every kernel configuration
that fits a problem (pipelined or tile kernels per pass, the n = 512 time-major hand-off, the
tile kernels' radix and tile size), rejects any configuration whose result differs from the
default's, keeps the fastest, and hands it to later problems of the same shape.  The tuned apply
is compared with the FP64 oracle element by element, and tuned instances in a shared-launch
batch give the same results as alone."""
import math

import numpy as np
import pytest
import torch

import synth
from closeness import assert_close
from oracle import discretisation as ds
from oracle import operators as op
from oracle import precond as pc

pytestmark = pytest.mark.gpu
ORACLE = {"abs_ps": pc.apply_abs_ps_inv, "ps": pc.apply_ps_inv, "pms": pc.apply_pms_inv}
TOL = {"mixed": 2e-6, "fp64": 1e-12}


@pytest.fixture(scope="module")
def P():
    from paper_2406_00952_gb300 import _build
    _build.build()
    import paper_2406_00952_gb300 as P
    return P


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# (N, n, theta, gamma, kind, precision, zeta, bc): pipelined-eligible shapes (with the n = 512
# hand-off), shapes only the tile kernels take (N + 1 = 192), FP64, general zeta and Neumann
CASES = [(63, 64, 1.0, 1e-2, "abs_ps", "mixed", math.pi, "dirichlet"),
         (127, 128, 0.5, 1e-3, "ps", "mixed", math.pi, "dirichlet"),
         (191, 64, 1.0, 1e-4, "pms", "mixed", math.pi, "dirichlet"),
         (255, 512, 1.0, 1e-2, "abs_ps", "mixed", math.pi, "dirichlet"),
         (63, 32, 0.5, 1e-2, "ps", "fp64", math.pi, "dirichlet"),
         (127, 64, 1.0, 1e-3, "abs_ps", "mixed", math.pi / 2, "dirichlet"),
         (129, 128, 0.5, 1e-2, "ps", "mixed", math.pi, "neumann")]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "N%d-n%d-%s-%s-z%.2f-%s" % (c[0], c[1], c[4], c[5], c[6], c[7]))
def test_autotuned_apply_matches_oracle(P, case):
    N, n, theta, gamma, kind, prec, zeta, bc = case
    a = 1e-3 if bc == "neumann" else 1.0
    prob = ds.Problem(N, n, theta, gamma, zeta=zeta, bc=bc, a0=a)
    v = synth.random_vector(2 * prob.m * n, seed=800 + N + n)
    ref = ORACLE[kind](prob, v)
    gp = P.Problem(N, n, theta, gamma, zeta=zeta, precision=prec, bc=bc, a=a)
    info = gp.autotune(kind=kind, reps=2)
    print(case[:2], prec, info)
    assert info["candidates"] >= 1 and info["rejected"] == 0, info
    assert info["best_ms"] <= info["default_ms"] * 1.0001, info
    out = gp.precond_apply(dev(v), kind=kind, precision=prec).cpu().numpy()
    assert_close(out, ref, TOL[prec], what=info)
    # a problem of the same shape created afterwards starts with the tuned configuration
    gp2 = P.Problem(N, n, theta, gamma, zeta=zeta, precision=prec, bc=bc, a=a)
    out2 = gp2.precond_apply(dev(v), kind=kind, precision=prec).cpu().numpy()
    assert np.array_equal(out, out2)


def test_autotuned_batch_equals_alone(P):
    """Tuned instances of the uneven-batch family in one shared-launch batch: each result equals the
    instance solved alone and meets the oracle's FP64 residual."""
    insts = synth.config3(count=6, seed=11, Ns=(63, 127, 191), ns=(32, 64, 128))
    probs, bs, oracles = [], [], []
    for inst in insts:
        prob = ds.Problem.from_instance(inst)
        b = ds.rhs_minres(prob, inst.g, inst.f) if inst.theta == 1.0 else ds.rhs_gmres(prob, inst.g, inst.f)
        gp = P.Problem(inst.N, inst.n, inst.theta, inst.gamma, precision="mixed")
        gp.autotune(reps=1)
        probs.append(gp); bs.append(b); oracles.append(prob)
    xs, infos = P.batch_solve(probs, [dev(b) for b in bs], tol=1e-8, restart=16)
    for gp, b, prob, x, info in zip(probs, bs, oracles, xs, infos):
        xo = x.cpu().numpy()
        assert info["relres"] <= 1e-8
        A = (lambda z: op.matvec_A(prob, z)) if prob.theta == 1.0 else (lambda z: op.matvec_A_hat(prob, z))
        assert np.linalg.norm(b - A(xo)) / np.linalg.norm(b) <= 1.5e-8
        x1, i1 = P.batch_solve([gp], [dev(b)], tol=1e-8, restart=16)
        assert_close(xo, x1[0].cpu().numpy(), 1e-12)
        assert i1[0]["iterations"] == info["iterations"]


# every configuration of the autotuner's list, installed directly, against the oracle: shapes with
# the n = 512 time pass (its three resident-block variants, with and without the time-major
# hand-off), the pipelined and tile kernels with their radices and tile sizes, FP64 and Neumann
SELECT_CASES = [(255, 512, 1.0, 1e-2, "abs_ps", "mixed", math.pi, "dirichlet"),
                (63, 512, 0.5, 1e-3, "ps", "mixed", math.pi, "dirichlet"),
                (127, 64, 1.0, 1e-4, "pms", "mixed", math.pi, "dirichlet"),
                (63, 32, 0.5, 1e-2, "ps", "fp64", math.pi, "dirichlet"),
                (127, 512, 1.0, 1e-3, "ps", "mixed", math.pi / 2, "dirichlet"),
                (129, 128, 0.5, 1e-2, "ps", "mixed", math.pi, "neumann")]


@pytest.mark.parametrize("case", SELECT_CASES, ids=lambda c: "N%d-n%d-%s-%s-z%.2f-%s" % (c[0], c[1], c[4], c[5], c[6], c[7]))
def test_every_configuration_matches_oracle(P, case):
    N, n, theta, gamma, kind, prec, zeta, bc = case
    a = 1e-3 if bc == "neumann" else 1.0
    prob = ds.Problem(N, n, theta, gamma, zeta=zeta, bc=bc, a0=a)
    v = synth.random_vector(2 * prob.m * n, seed=700 + N + n)
    ref = ORACLE[kind](prob, v)
    gp = P.Problem(N, n, theta, gamma, zeta=zeta, precision=prec, bc=bc, a=a)
    count = gp.tune_select(-1)["candidates"]
    assert count >= 1
    seen = set()
    for k in range(count):
        info = gp.tune_select(k)
        seen.add((info["pipelined_dst"], info["pipelined_time"], info["time_major_handoff"], info["time512_blocks"]))
        out = gp.precond_apply(dev(v), kind=kind, precision=prec).cpu().numpy()
        assert_close(out, ref, TOL[prec], what=info)
    if n == 512 and prec == "mixed" and zeta == math.pi:
        assert {b for *_, b in seen} == {2, 3, 4}, seen
    if n == 512 and prec == "mixed":       # with and without the time-major hand-off
        assert {h for _, _, h, _ in seen} == {0, 1}, seen
    with pytest.raises(Exception):
        gp.tune_select(count)

"""GPU parity of the finite-element route (bilinear elements, M != I: the system of Eq. main_system
with K~ = M^{-1/2} K M^{-1/2}) against the FP64 oracle, through the C-ABI.  The products and the
mass factors run through the FP64 2D DST-I (K~ and M are diagonal in the sine basis); the
preconditioners are the finite-difference kernels with the element eigenvalues in their tables.
Tolerances as in the other parity tests (relative 2-norm and max-norm): products through two FP64
transforms <= 1e-12, FP64 preconditioner <= 1e-12, FP32 preconditioner <= 2e-6, same-algorithm
iterates <= 1e-10, mixed solutions <= 1e-7 of the oracle's."""
import numpy as np
import pytest
import torch

import synth
from closeness import assert_close
from oracle import discretisation as ds
from oracle import krylov as kr
from oracle import operators as op
from oracle import precond as pc

pytestmark = pytest.mark.gpu
ORACLE = {"abs_ps": pc.apply_abs_ps_inv, "ps": pc.apply_ps_inv, "pms": pc.apply_pms_inv}


@pytest.fixture(scope="module")
def P():
    from paper_2406_00952_gb300 import _build
    _build.build()
    import paper_2406_00952_gb300 as P
    return P


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SHAPES = [(7, 8, 1.0, 1e-2), (15, 16, 0.5, 1e-4), (31, 64, 0.75, 1e-3), (63, 32, 1.0, 1e-6), (127, 128, 0.5, 1e-2),
          (255, 16, 1.0, 1e-2)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "N%d-n%d-th%g-g%g" % s)
def test_fem_products_and_preconditioners(P, shape):
    N, n, theta, gamma = shape
    prob = ds.Problem(N, n, theta, gamma, fem=True)
    v = synth.random_vector(2 * prob.m * n, seed=900 + N + n)
    gp = P.Problem(N, n, theta, gamma, precision="fp64", fem=True)
    for opname, ref in (("A", op.matvec_A(prob, v)), ("Ahat", op.matvec_A_hat(prob, v))):
        assert_close(gp.matvec(dev(v), op=opname).cpu().numpy(), ref, 1e-12, what=opname)
    for kind in ("abs_ps", "ps", "pms"):
        ref = ORACLE[kind](prob, v)
        assert_close(gp.precond_apply(dev(v), kind=kind, precision="fp64").cpu().numpy(), ref, 1e-12, what=kind)
        assert_close(gp.precond_apply(dev(v), kind=kind, precision="mixed").cpu().numpy(), ref, 2e-6, what=kind)


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_fem_rhs_and_recover(P, theta):
    N, n, gamma = 31, 16, 3e-3
    prob = ds.Problem(N, n, theta, gamma, fem=True)
    g = synth.random_target(N, n, seed=31); f = synth.manufactured_source(N, n)
    gp = P.Problem(N, n, theta, gamma, fem=True)
    for opname, ref in (("A", ds.rhs_minres(prob, g, f)), ("Ahat", ds.rhs_gmres(prob, g, f))):
        assert_close(gp.assemble_rhs(dev(g.ravel()), dev(f.ravel()), op=opname).cpu().numpy(), ref, 1e-12)
    x = synth.random_vector(2 * prob.m * n, seed=32)
    y, p = gp.recover(dev(x))
    yr, pr = ds.recover(prob, x)
    assert_close(y.cpu().numpy(), yr.ravel(), 1e-12)
    assert_close(p.cpu().numpy(), pr.ravel(), 1e-12)
    with pytest.raises(Exception) as e:         # y0 != 0 is not taken by the element route
        gp.assemble_rhs(dev(g.ravel()), dev(f.ravel()), dev(np.ones(N * N)))
    assert "unsupported" in str(e.value)


@pytest.mark.parametrize("case", [("minres", "abs_ps", 1.0), ("minres", "pms", 1.0), ("gmres", "ps", 0.5)])
def test_fem_same_algorithm_iterates_and_solves(P, case):
    method, kind, theta = case
    N, n, gamma = 31, 32, 1e-3
    prob = ds.Problem(N, n, theta, gamma, fem=True)
    g = synth.random_target(N, n, seed=33); f = synth.manufactured_source(N, n)
    b = ds.rhs_minres(prob, g, f) if method == "minres" else ds.rhs_gmres(prob, g, f)
    M = lambda r: ORACLE[kind](prob, r)
    A = (lambda z: op.matvec_A(prob, z)) if method == "minres" else (lambda z: op.matvec_A_hat(prob, z))
    solver = kr.minres if method == "minres" else kr.fgmres
    gp = P.Problem(N, n, theta, gamma, precision="fp64", fem=True)
    for k in (3, 8):
        xo, _ = solver(A, b, M, fixed_iterations=k)
        x, info = gp.solve(dev(b), method=method, precond=kind, fixed_iterations=k, restart=30)
        assert info["iterations"] == k
        assert_close(x.cpu().numpy(), xo, 1e-10, what=k)
    xs, _ = solver(A, b, M, tol=1e-12)
    x, i64 = gp.solve(dev(b), method=method, precond=kind, tol=1e-8)
    assert i64["relres"] <= 1e-8 and rel(x.cpu().numpy(), xs) <= 1e-7
    gm = P.Problem(N, n, theta, gamma, precision="mixed", fem=True)
    xm, im = gm.solve(dev(b), method=method, precond=kind, tol=1e-8)
    assert im["relres"] <= 1e-8 and rel(xm.cpu().numpy(), xs) <= 1e-7
    assert np.linalg.norm(b - A(xm.cpu().numpy())) / np.linalg.norm(b) <= 1.5e-8
    assert im["iterations"] <= i64["iterations"] + 2, (im, i64)


def test_fem_example1_counts(P):
    """Example 1 with bilinear elements at h = 2^-5 (gamma = 1e-2, Crank-Nicolson): the GPU takes
    Table 1's counts (GMRES-P_S 3, MINRES-|P_S| 6), as the oracle does, and the same e_h."""
    N, n, gamma = 31, 32, 1e-2
    prob = ds.Problem(N, n, 0.5, gamma, fem=True)
    g, f, ye, pe = synth.example1_data(N, n)
    gp = P.Problem(N, n, 0.5, gamma, precision="fp64", fem=True)
    for method, kind, b, want in (("gmres", "ps", ds.rhs_gmres(prob, g, f, ye[0]), 3),
                                  ("minres", "abs_ps", ds.rhs_minres(prob, g, f, ye[0]), 6)):
        x, info = gp.solve(dev(b), method=method, precond=kind, tol=1e-8)
        assert info["iterations"] == want, (method, info)
        y, p = gp.recover(x)
        e = ds.error_eh(prob, y.cpu().numpy().reshape(n, -1), p.cpu().numpy().reshape(n, -1), ye, pe)
        yo, po = ds.recover(prob, x.cpu().numpy())
        assert abs(e - ds.error_eh(prob, yo, po, ye, pe)) <= 1e-6 * e

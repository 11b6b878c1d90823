"""GPU parity of the Neumann route (Example 3: mirrored stencil, DCT-I in place of the DST-I,
GMRES-P_S) against the FP64 oracle, through the C-ABI.

Tolerances are those of the Dirichlet parity tests, each on the relative 2-norm and the relative
max-norm error (tests/closeness.py): FP64 transforms and operators <= 1e-12 (products <= 1e-13),
the FP32 preconditioner <= 2e-6, same-algorithm FP64 iterates <= 1e-10.
"""
import math

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
PI = math.pi


@pytest.fixture(scope="module")
def P():
    from paper_2406_00952_gb300 import _build
    _build.build()
    import paper_2406_00952_gb300 as P
    return P


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# (N, n, theta, gamma, a, zeta): N - 1 = 2^a 3^b covers the register-FFT variants Q = 1 .. 32,
# radix-3 lines (N = 25, 49, 97), the smallest grid and the largest (N = 513, a length-1024 line);
# FP32 applies with 2(N-1) = 32 P (P = 8, 16, 32) and n = 64 ... 512 run the pipelined kernels
SHAPES = [(3, 2, 1.0, 1.0, 1.0, PI), (5, 4, 0.5, 1e-2, 1e-3, PI), (17, 16, 0.5, 1e-2, 1e-3, PI),
          (33, 32, 1.0, 1e-4, 0.3, PI), (49, 8, 0.5, 1e-6, 1.0, PI), (65, 64, 0.5, 1e-3, 1e-3, 0.4),
          (97, 128, 1.0, 1e-2, 2.0, PI), (129, 512, 0.5, 1e-2, 1e-3, PI), (257, 32, 0.5, 1e-2, 1e-3, PI),
          (513, 4, 0.5, 1e-2, 1e-3, PI), (25, 1024, 0.5, 1e-2, 1e-3, 0.0), (7, 256, 1.0, 1e-5, 1.0, PI),
          # the pipelined DCT-I passes (2(N-1) = 32 P, P = 8, 16, 32; n = 512 with the time-major hand-off)
          (257, 256, 0.5, 1e-2, 1e-3, PI), (513, 64, 1.0, 1e-4, 0.5, PI), (257, 512, 0.5, 1e-3, 1e-3, PI),
          (129, 128, 1.0, 1e-6, 2.0, PI)]


def _prob(s):
    N, n, theta, gamma, a, zeta = s
    return ds.Problem(N, n, theta, gamma, zeta=zeta, bc="neumann", a0=a)


def _gpu(P, s, precision="fp64"):
    N, n, theta, gamma, a, zeta = s
    return P.Problem(N, n, theta, gamma, zeta=zeta, precision=precision, bc="neumann", a=a)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "N%d-n%d-th%g-g%g-a%g-z%.2f" % s)
def test_neumann_precond_parity(P, shape):
    prob = _prob(shape)
    v = synth.random_vector(2 * prob.m * prob.n, seed=700 + shape[0] + shape[1])
    ref = pc.apply_ps_inv(prob, v)
    gp = _gpu(P, shape)
    out64 = gp.precond_apply(dev(v), kind="ps", precision="fp64").cpu().numpy()
    out32 = gp.precond_apply(dev(v), kind="ps", precision="mixed").cpu().numpy()
    assert_close(out64, ref, 1e-12, what="fp64")
    assert_close(out32, ref, 2e-6, what="fp32")
    t = dev(v)
    gp.precond_apply(t, out=t, kind="ps", precision="fp64")
    assert_close(t.cpu().numpy(), ref, 1e-12, what="fp64 in place")


def test_neumann_refuses_minres_preconditioners(P):
    gp = _gpu(P, SHAPES[2])
    v = dev(np.ones(2 * 17 * 17 * 16))
    for kind in ("abs_ps", "pms"):
        with pytest.raises(RuntimeError):
            gp.precond_apply(v, kind=kind)
    with pytest.raises(RuntimeError):
        gp.solve(v, method="minres", precond="abs_ps")


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[2], SHAPES[3], SHAPES[6], SHAPES[9]],
                         ids=lambda s: "N%d-n%d-th%g" % s[:3])
@pytest.mark.parametrize("opname", ["A", "Ahat"])
def test_neumann_matvec_parity(P, shape, opname):
    prob = _prob(shape)
    v = synth.random_vector(2 * prob.m * prob.n, seed=800 + shape[0])
    ref = op.matvec_A(prob, v) if opname == "A" else op.matvec_A_hat(prob, v)
    out = _gpu(P, shape).matvec(dev(v), op=opname).cpu().numpy()
    assert_close(out, ref, 1e-13)


@pytest.mark.parametrize("theta", [1.0, 0.5, 0.8])
def test_neumann_rhs_parity(P, theta):
    N, n, a = 17, 8, 0.05
    prob = ds.Problem(N, n, theta, 3e-3, bc="neumann", a0=a)
    g, f, ye, _ = synth.example3_data(N, n, a0=a)
    y0 = synth.random_vector(N * N, seed=14)
    gp = P.Problem(N, n, theta, 3e-3, bc="neumann", a=a)
    for opname, ref in (("A", ds.rhs_minres(prob, g, f, y0)), ("Ahat", ds.rhs_gmres(prob, g, f, y0))):
        b = gp.assemble_rhs(dev(g.ravel()), dev(f.ravel()), dev(y0), op=opname).cpu().numpy()
        assert_close(b, ref, 1e-14)


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_neumann_same_algorithm_iterates(P, theta):
    """GMRES-P_S, oracle and GPU, after 3 and 8 iterations (FP64): the product's residual epilogue
    (theta = 1 folded path) and the DCT-I passes inside one algorithm."""
    N, n, gamma, a = 33, 32, 1e-4, 1e-2
    prob = ds.Problem(N, n, theta, gamma, bc="neumann", a0=a)
    g = synth.random_target(N, n, seed=21)      # values on the N x N node array (layout only)
    f = synth.manufactured_source(N, n)
    b = ds.rhs_gmres(prob, g, f)
    for k in (3, 8):
        xo, _ = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), b, lambda r: pc.apply_ps_inv(prob, r),
                          tol=1e-14, fixed_iterations=k)
        gp = P.Problem(N, n, theta, gamma, precision="fp64", bc="neumann", a=a)
        x, info = gp.solve(dev(b), method="gmres", precond="ps", fixed_iterations=k, restart=30)
        assert info["iterations"] == k
        assert_close(x.cpu().numpy(), xo, 1e-10)


@pytest.mark.parametrize("gamma", [1e-10, 1e-8, 1e-6, 1e-4, 1e-2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_neumann_example3_solve(P, gamma, precision):
    """Example 3 (Table 4's problem, Crank-Nicolson, a = 1e-3) on the 33-node grid (h = 1/32, a
    line length the DCT-I radices cover): GMRES-P_S to 1e-8 on the GPU; the discrete error e_h
    matches the oracle's solve of the same system, and the iteration count the oracle's."""
    N, n = 33, 32
    prob = ds.Problem(N, n, 0.5, gamma, bc="neumann", a0=1e-3)
    g, f, ye, pe = synth.example3_data(N, n)
    bo = ds.rhs_gmres(prob, g, f, ye[0])
    xo, io = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), bo, lambda r: pc.apply_ps_inv(prob, r), tol=1e-8)
    eo = ds.error_eh(prob, *ds.recover(prob, xo), ye, pe)
    gp = P.Problem(N, n, 0.5, gamma, precision=precision, bc="neumann", a=1e-3)
    b = gp.assemble_rhs(dev(g.ravel()), dev(f.ravel()), dev(ye[0]), op="Ahat")
    assert_close(b.cpu().numpy(), bo, 1e-14)
    # mixed: the refinement stops as soon as the FP64 residual allows, and a relative residual r
    # leaves an error of about r |y| in the state, which at gamma = 1e-10 (e_h ~ 1e-11) is above the
    # discretisation error unless r ~ 1e-12; the error comparison asks the mixed solve for that
    tol = 1e-8 if precision == "fp64" else 1e-12
    x, info = gp.solve(b, tol=tol)
    assert info["method"] == 2 and info["precond"] == 2          # AUTO picks GMRES-P_S
    assert info["relres"] <= tol
    if precision == "fp64":
        assert info["iterations"] == io.iterations
    y, p = gp.recover(x)
    e = ds.error_eh(prob, y.cpu().numpy().reshape(n, -1), p.cpu().numpy().reshape(n, -1), ye, pe)
    assert abs(e - eo) / eo < 0.02, (e, eo)


def test_neumann_example3_refinement(P):
    """Second-order convergence on the GPU: e_h at h = 1/64 and 1/128 (n = 1/h) drops by ~4."""
    es = []
    for N in (65, 129):
        n = N - 1
        g, f, ye, pe = synth.example3_data(N, n)
        gp = P.Problem(N, n, 0.5, 1e-2, precision="fp64", bc="neumann", a=1e-3)
        b = gp.assemble_rhs(dev(g.ravel()), dev(f.ravel()), dev(ye[0]), op="Ahat")
        x, info = gp.solve(b, tol=1e-8)
        assert info["relres"] <= 1e-8 and info["iterations"] <= 4
        prob = ds.Problem(N, n, 0.5, 1e-2, bc="neumann", a0=1e-3)
        y, p = gp.recover(x)
        es.append(ds.error_eh(prob, y.cpu().numpy().reshape(n, -1), p.cpu().numpy().reshape(n, -1), ye, pe))
    assert 3.6 < es[0] / es[1] < 4.4, es


def test_neumann_batch_with_dirichlet(P):
    """A batch mixing Neumann and Dirichlet GMRES instances: shared launches, per-instance
    transforms; each result equals the instance solved alone."""
    specs = [dict(N=33, n=32, bc="neumann", a=1e-3), dict(N=31, n=32, bc="dirichlet", a=1.0),
             dict(N=17, n=64, bc="neumann", a=0.1)]
    probs, bs = [], []
    for k, sp_ in enumerate(specs):
        prob = ds.Problem(sp_["N"], sp_["n"], 0.5, 1e-3, bc=sp_["bc"], a0=sp_["a"])
        g = synth.random_target(sp_["N"], sp_["n"], seed=40 + k); f = synth.manufactured_source(sp_["N"], sp_["n"])
        bs.append(ds.rhs_gmres(prob, g, f))
        probs.append((prob, P.Problem(sp_["N"], sp_["n"], 0.5, 1e-3, precision="mixed", bc=sp_["bc"], a=sp_["a"])))
    xs, infos = P.batch_solve([gp for _, gp in probs], [dev(b) for b in bs], tol=1e-8, restart=16)
    for (prob, gp), b, x, info in zip(probs, bs, xs, infos):
        assert info["relres"] <= 1e-8
        xo = x.cpu().numpy()
        assert np.linalg.norm(b - op.matvec_A_hat(prob, xo)) / np.linalg.norm(b) <= 1.5e-8
        x1, i1 = P.batch_solve([gp], [dev(b)], tol=1e-8, restart=16)
        assert_close(xo, x1[0].cpu().numpy(), 1e-12)
        assert i1[0]["iterations"] == info["iterations"]


# ---------------------------------------------------------------- multigrid route (Sec. 4, Example 3)
MG_SHAPES = [(5, 4, 0.5, 1e-2, 1e-3), (17, 16, 1.0, 1e-4, 0.3), (33, 32, 0.5, 1e-2, 1e-3), (65, 64, 0.5, 1e-6, 1e-3),
             (129, 8, 1.0, 1e-2, 1.0), (257, 32, 0.5, 1e-3, 1e-3)]


@pytest.mark.parametrize("shape", MG_SHAPES, ids=lambda s: "N%d-n%d-th%g-g%g-a%g" % s)
def test_neumann_multigrid_precond_parity(P, shape):
    """P_S^{-1} with two V-cycles per shifted solve on the Neumann grid (N = 2^k + 1 nodes), against
    the oracle's multigrid route element by element (FP64 <= 1e-12, FP32 <= 5e-6)."""
    N, n, theta, gamma, a = shape
    prob = ds.Problem(N, n, theta, gamma, bc="neumann", a0=a)
    v = synth.random_vector(2 * prob.m * n, seed=950 + N + n)
    ref = pc.apply_mg_ps_inv(prob, v, cycles=2)
    gp = P.Problem(N, n, theta, gamma, bc="neumann", a=a, multigrid=True, mg_cycles=2)
    assert_close(gp.precond_apply(dev(v), kind="ps", precision="fp64").cpu().numpy(), ref, 1e-12, what="fp64")
    assert_close(gp.precond_apply(dev(v), kind="ps", precision="mixed").cpu().numpy(), ref, 5e-6, what="fp32")


@pytest.mark.parametrize("gamma", [1e-10, 1e-6, 1e-2])
def test_neumann_example3_multigrid_solve(P, gamma):
    """Example 3 with the multigrid shifted solves on the GPU: FP64 GMRES-P_S iterates equal the
    oracle's (8 iterations, same algorithm), the solve to 1e-8 takes the oracle's count and its e_h;
    the mixed solve converges to the same tolerance."""
    N, n = 33, 32
    prob = ds.Problem(N, n, 0.5, gamma, bc="neumann", a0=1e-3)
    g, f, ye, pe = synth.example3_data(N, n)
    b = ds.rhs_gmres(prob, g, f, ye[0])
    M = lambda r: pc.apply_mg_ps_inv(prob, r, cycles=2)
    A = lambda z: op.matvec_A_hat(prob, z)
    gp = P.Problem(N, n, 0.5, gamma, bc="neumann", a=1e-3, multigrid=True, mg_cycles=2, precision="fp64")
    xo, _ = kr.fgmres(A, b, M, fixed_iterations=4)
    x, info = gp.solve(dev(b), method="fgmres", precond="ps", fixed_iterations=4, restart=30)
    assert_close(x.cpu().numpy(), xo, 1e-10)
    xo, io = kr.fgmres(A, b, M, tol=1e-8)
    x, info = gp.solve(dev(b), tol=1e-8)
    assert info["method"] in (2, 3) and info["iterations"] == io.iterations and info["relres"] <= 1e-8
    y, p = gp.recover(x)
    e = ds.error_eh(prob, y.cpu().numpy().reshape(n, -1), p.cpu().numpy().reshape(n, -1), ye, pe)
    assert abs(e - ds.error_eh(prob, *ds.recover(prob, xo), ye, pe)) <= 0.02 * e
    gm = P.Problem(N, n, 0.5, gamma, bc="neumann", a=1e-3, multigrid=True, mg_cycles=2, precision="mixed")
    xm, im = gm.solve(dev(b), tol=1e-8)
    assert im["relres"] <= 1e-8
    assert np.linalg.norm(b - A(xm.cpu().numpy())) / np.linalg.norm(b) <= 1.5e-8


def test_dirichlet_constant_coefficient_multigrid_route(P):
    """multigrid=True with a constant coefficient on a Dirichlet grid runs the variable-coefficient
    route with every edge value equal to a: the same result as the oracle's multigrid route."""
    N, n, a = 63, 32, 0.7
    edges = np.full(2 * N * (N + 1), a)
    prob = ds.Problem(N, n, 0.5, 1e-3, a_edges=edges)
    v = synth.random_vector(2 * prob.m * n, seed=977)
    ref = pc.apply_mg_ps_inv(prob, v, cycles=2)
    gp = P.Problem(N, n, 0.5, 1e-3, a=a, multigrid=True, mg_cycles=2)
    assert_close(gp.precond_apply(dev(v), kind="ps", precision="fp64").cpu().numpy(), ref, 1e-12)
    assert_close(gp.matvec(dev(v), op="Ahat").cpu().numpy(), op.matvec_A_hat(prob, v), 1e-13)

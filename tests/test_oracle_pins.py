"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: dense matrices built straight
from the paper's definitions, closed forms (Lemma 3.4, B_n entries), spectral statements
(Props. 3.1, 3.2, Thm 3.3, Thm 3.11), a sparse direct solve of the paper's block system, brute-force
transforms, and the iteration counts / errors printed in Table 1.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import discretisation as ds
from oracle import krylov as kr
from oracle import multigrid as mg
from oracle import operators as op
from oracle import precond as pc
from oracle import spectra as spc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(12345)

CASES = [(1.0, math.pi), (0.5, math.pi), (0.75, math.pi), (1.0, 0.0), (0.75, 0.0), (1.0, 1.1), (0.5, 2.3)]


# ---------------------------------------------------------------- P1: omega-circulant spectra
@pytest.mark.parametrize("n", [4, 7, 16])
@pytest.mark.parametrize("theta,zeta", CASES)
def test_omega_circulant_factorisation(n, theta, zeta):
    """S^(j) = D^{-1} F^{-1} diag(lambda^(j)) F D against the dense matrices of Sec. 1 (corner
    entries -omega and omega(1-theta)); eigenvalue sets against the paper's printed index set."""
    F = np.fft.fft(np.eye(n), axis=0)
    D = np.diag(spc.D_omega(n, zeta))
    Finv = np.linalg.inv(F)
    k = np.arange(n)
    ph = (zeta + 2 * math.pi * k) / n                   # the paper's printed index set
    cases = ((spc.S1_dense(n, zeta), spc.lam_S1(n, zeta), 1 - np.exp(1j * ph)),
             (spc.S2_dense(n, theta, zeta), spc.lam_S2(n, theta, zeta, remedy=False),
              theta + (1 - theta) * np.exp(1j * ph)))
    for S, lam, printed in cases:
        rebuilt = np.linalg.inv(D) @ Finv @ np.diag(lam) @ F @ D
        assert np.abs(rebuilt - S).max() < 1e-13
        for a in (np.linalg.eigvals(S), printed):
            d = np.abs(np.sort_complex(np.round(a, 10)) - np.sort_complex(np.round(lam, 10)))
            assert d.max() < 1e-8


@pytest.mark.parametrize("n,theta,zeta", [(8, 1.0, math.pi), (10, 0.5, math.pi), (6, 0.7, 0.4)])
def test_Sn_spectrum_dense(n, theta, zeta):
    Sn = spc.S1_dense(n, zeta) @ np.linalg.inv(spc.S2_dense(n, theta, zeta))
    ev = np.sort_complex(np.round(np.linalg.eigvals(Sn), 9))
    lam = np.sort_complex(np.round(spc.lam_Sn(n, theta, zeta), 9))
    assert np.abs(ev - lam).max() < 1e-7


def test_singular_S2_remedy():
    """Remark 1: S^(2) is singular for theta = 1/2 with zeta = 0, n even (and zeta = pi, n odd);
    the replacement value is 1."""
    lam = spc.lam_S2(8, 0.5, 0.0, remedy=False)
    assert np.min(np.abs(lam)) < 1e-15
    assert np.min(np.abs(spc.lam_S2(8, 0.5, 0.0))) > 0.1
    assert np.min(np.abs(spc.lam_S2(7, 0.5, math.pi, remedy=False))) < 1e-15
    assert np.min(np.abs(spc.lam_S2(8, 0.5, math.pi, remedy=False))) > 1e-3


# ---------------------------------------------------------------- P4: Lemma 3.4
@pytest.mark.parametrize("theta", [0.5, 0.6, 0.8, 1.0])
@pytest.mark.parametrize("zeta", [0.2, math.pi])
def test_lemma_3_4_closed_form(theta, zeta):
    n = 12
    lam = spc.lam_Sn(n, theta, zeta)
    ph = spc.phi(n, zeta)
    closed = 2 * (2 * theta - 1) * (1 - np.cos(ph)) / (theta ** 2 + (1 - theta) ** 2 + 2 * theta * (1 - theta) * np.cos(ph))
    assert np.all(np.abs(2 * lam.real - closed) <= 1e-13 * np.maximum(1.0, np.abs(lam) ** 2))
    assert np.all(closed >= -1e-15)
    if theta == 0.5:
        assert np.all(np.abs(lam.real) <= 1e-14 * np.maximum(1.0, np.abs(lam) ** 2))   # Remark 3
    Sn = spc.S1_dense(n, zeta) @ np.linalg.inv(spc.S2_dense(n, theta, zeta))
    assert np.linalg.eigvalsh(Sn + Sn.conj().T).min() > -1e-12


# ---------------------------------------------------------------- P8: B_n
@pytest.mark.parametrize("theta", [0.5, 0.6, 1.0])
def test_Bn_entries_and_application(theta):
    n = 9
    Bn = ds.B1_dense(n) @ np.linalg.inv(ds.B2_dense(n, theta))
    assert np.abs(Bn - ds.Bn_closed_form(n, theta)).max() < 1e-12
    assert np.abs(Bn - np.linalg.inv(ds.B2_dense(n, theta)) @ ds.B1_dense(n)).max() < 1e-12
    x = rng.standard_normal((n, 5))
    assert np.abs(ds.apply_Bn(theta, x) - Bn @ x).max() < 1e-12
    assert np.abs(ds.apply_Bn(theta, x, transpose=True) - Bn.T @ x).max() < 1e-12


# ---------------------------------------------------------------- P12: transforms
@pytest.mark.parametrize("N", [1, 3, 7, 15])
def test_dst_and_laplacian_eigenbasis(N):
    S = spc.dst_matrix(N)
    assert np.abs(S @ S - np.eye(N)).max() < 1e-13            # orthogonal and involutory
    assert np.abs(S - S.T).max() < 1e-15
    prob = ds.Problem(N, 2, 1.0, 1.0)
    K = pc.dense_K(prob)
    S2 = np.kron(S, S)
    assert np.abs(K @ S2 - S2 @ np.diag(spc.kappa2d(N).ravel())).max() < 1e-9 * (N + 1) ** 2
    u = rng.standard_normal((3, N * N))
    assert np.abs(spc.dst2(u, N) - u @ S2.T).max() < 1e-13


@pytest.mark.parametrize("n,zeta", [(5, math.pi), (8, math.pi), (6, 0.0), (7, 1.3)])
def test_time_transform_brute_force(n, zeta):
    v = rng.standard_normal((n, 3))
    brute = np.array([[sum(v[t, c] * np.exp(1j * t * p) for t in range(n)) for c in range(3)]
                      for p in spc.phi(n, zeta)])
    assert np.abs(spc.time_forward(v, zeta) - brute).max() < 1e-12
    assert np.abs(spc.time_inverse(brute, zeta) - v).max() < 1e-12


def test_K_variable_coefficient():
    N = 7
    prob = ds.Problem(N, 2, 1.0, 1.0, a_edges=synth.variable_coefficient_edges(N))
    K = pc.dense_K(prob)
    assert np.abs(K - K.T).max() < 1e-10
    assert np.linalg.eigvalsh(K).min() > 0
    u = rng.standard_normal((2, N * N))
    assert np.abs(ds.apply_K(prob, u) - u @ K.T).max() < 1e-9
    # second-order consistency with -div(a grad u) on a smooth u
    for Nc in (15, 31):
        pr = ds.Problem(Nc, 2, 1.0, 1.0, a_edges=synth.variable_coefficient_edges(Nc))
        x1, x2 = synth.grid(Nc)
        uu = np.sin(math.pi * x1) * np.sin(2 * math.pi * x2)
        a = 1 + 0.5 * np.sin(math.pi * x1) * np.sin(math.pi * x2)
        ax_ = 0.5 * math.pi * np.cos(math.pi * x1) * np.sin(math.pi * x2)
        ay_ = 0.5 * math.pi * np.sin(math.pi * x1) * np.cos(math.pi * x2)
        ux = math.pi * np.cos(math.pi * x1) * np.sin(2 * math.pi * x2)
        uy = 2 * math.pi * np.sin(math.pi * x1) * np.cos(2 * math.pi * x2)
        lap = -(math.pi ** 2 + 4 * math.pi ** 2) * uu
        exact = -(a * lap + ax_ * ux + ay_ * uy)
        err = np.abs(ds.apply_K(pr, uu.ravel()) - exact.ravel()).max()
        if Nc == 15:
            e15 = err
    assert err < e15 / 3.0


# ---------------------------------------------------------------- P3 / P2: preconditioners
SMALL = [(3, 4), (5, 6), (4, 8)]


@pytest.mark.parametrize("N,n", SMALL)
@pytest.mark.parametrize("theta,zeta", [(1.0, math.pi), (0.5, math.pi), (0.75, math.pi), (1.0, 0.0), (0.5, 1.1)])
@pytest.mark.parametrize("gamma", [1e-2, 1e-6])
def test_preconditioners_vs_dense(N, n, theta, zeta, gamma):
    prob = ds.Problem(N, n, theta, gamma, zeta=zeta)
    v = rng.standard_normal(2 * prob.m * prob.n)
    P = pc.dense_P_S(prob)
    w = pc.apply_ps_inv(prob, v, real=False)
    assert np.abs(P @ w - v).max() < 1e-12 * np.abs(v).max()
    assert np.abs(w - np.linalg.solve(P, v)).max() < 1e-11 * np.abs(w).max()
    aP = pc.dense_abs_P_S(prob)
    exact = np.linalg.solve(aP, v)
    w = pc.apply_abs_ps_inv(prob, v)
    assert np.abs(w - exact.real).max() < 1e-11 * np.abs(exact).max()
    if zeta in (0.0, math.pi):
        assert np.abs(exact.imag).max() < 1e-12 * np.abs(exact).max()   # real operator
        assert np.abs(aP - aP.conj().T).max() < 1e-9
        assert np.linalg.eigvalsh(0.5 * (aP + aP.conj().T)).min() > 0
    Pm = pc.dense_P_MS(prob)
    exact = np.linalg.solve(Pm, v)
    assert np.abs(pc.apply_pms_inv(prob, v) - exact.real).max() < 1e-11 * np.abs(exact).max()


def test_remedied_S2_rank_one_and_fast_apply():
    """Remark 1: replacing the zero eigenvalue of S^(2) gives a rank-1 modification; the fast
    P_S^{-1} then equals the dense inverse built from the remedied S_n."""
    N, n, theta, zeta = 3, 5, 0.5, math.pi
    prob = ds.Problem(N, n, theta, 1e-2, zeta=zeta)
    F = np.fft.fft(np.eye(n), axis=0); D = np.diag(spc.D_omega(n, zeta))
    S2t = np.linalg.inv(D) @ np.linalg.inv(F) @ np.diag(spc.lam_S2(n, theta, zeta)) @ F @ D
    assert np.linalg.matrix_rank(S2t - spc.S2_dense(n, theta, zeta), tol=1e-10) == 1
    Sn = spc.S1_dense(n, zeta) @ np.linalg.inv(S2t)
    calS = np.kron(Sn, np.eye(prob.m)) + prob.tau * np.kron(np.eye(n), pc.dense_K(prob))
    I = np.eye(calS.shape[0]); a = prob.alpha
    P = np.block([[calS, -a * I], [a * I, calS.conj().T]])
    v = rng.standard_normal(2 * prob.m * n)
    assert np.abs(P @ pc.apply_ps_inv(prob, v, real=False) - v).max() < 1e-11


def test_preconditioner_variable_a_dense():
    """P_S^{-1} with many V-cycles converges to the dense inverse built with variable-a K."""
    N, n = 7, 4
    prob = ds.Problem(N, n, 0.5, 1e-4, a_edges=synth.variable_coefficient_edges(N))
    v = rng.standard_normal(2 * prob.m * n)
    exact = np.linalg.solve(pc.dense_P_S(prob), v).real
    prev = None
    for cyc in (2, 8, 30):
        err = np.abs(pc.apply_mg_ps_inv(prob, v, cycles=cyc) - exact).max() / np.abs(exact).max()
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 1e-10


# ---------------------------------------------------------------- P5, P6, P7: spectral statements
@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_prop_3_1_rank(theta):
    prob = ds.Problem(3, 8, theta, 1e-3)
    n, m = prob.n, prob.m
    Bn = ds.B1_dense(n) @ np.linalg.inv(ds.B2_dense(n, theta))
    assert np.linalg.matrix_rank(pc.dense_Sn(prob) - Bn, tol=1e-10) <= 2
    R = pc.dense_P_S(prob) - pc.dense_A_hat(prob)
    assert np.linalg.matrix_rank(R, tol=1e-9) <= 4 * m


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_prop_3_2_ideal(theta):
    prob = ds.Problem(3, 6, theta, 1e-2)
    A = pc.dense_A(prob)
    Q = np.linalg.solve(pc.dense_abs_A(prob), A)
    assert np.abs(Q - Q.T).max() < 1e-9
    assert np.abs(Q @ Q - np.eye(A.shape[0])).max() < 1e-9
    assert np.abs(np.abs(np.linalg.eigvals(Q)) - 1).max() < 1e-8


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_thm_3_3_clustering(theta):
    outliers = []
    for n in (8, 16):
        prob = ds.Problem(3, n, theta, 1e-2)
        ev = np.linalg.eigvals(np.linalg.solve(pc.dense_abs_P_S(prob), pc.dense_A(prob)))
        assert np.abs(ev.imag).max() < 1e-8
        k = int(np.sum(np.abs(np.abs(ev.real) - 1) > 1e-6))
        assert k <= 8 * prob.m                    # Hermitian-unitary + rank <= 4m perturbation
        outliers.append(k)
    assert outliers[1] <= outliers[0] + 2         # number of outliers does not grow with n


@pytest.mark.parametrize("theta,bound", [(1.0, math.sqrt(2)), (0.75, math.sqrt(2)), (0.5, 1.0)])
@pytest.mark.parametrize("gamma", [1e-10, 1e-2])
def test_thm_3_11_spectral_equivalence(theta, bound, gamma):
    prob = ds.Problem(3, 8, theta, gamma)
    ev = np.linalg.eigvals(np.linalg.solve(pc.dense_P_MS(prob), pc.dense_abs_P_S(prob)))
    assert np.abs(ev.imag).max() < 1e-9
    assert ev.real.min() >= 1 / math.sqrt(2) - 1e-9
    assert ev.real.max() <= bound + 1e-9


def test_lemma_3_14_decoupling():
    for _ in range(20):
        lam = complex(rng.uniform(-1, 2), rng.uniform(-3, 3)); alpha = rng.uniform(0.01, 5)
        M1, M2, D1, D2 = pc.lemma314(np.array([lam]), alpha)
        G = np.array([[lam, -alpha], [alpha, np.conj(lam)]])
        W = np.array([[1, M2[0]], [M1[0], 1]])
        assert np.abs(W @ np.diag([D1[0], D2[0]]) @ np.linalg.inv(W) - G).max() < 1e-12
        s = math.sqrt(lam.imag ** 2 + alpha ** 2)
        assert abs(D1[0] - complex(lam.real, s)) < 1e-12 and abs(D2[0] - complex(lam.real, -s)) < 1e-12
        assert abs(M1[0] - M2[0]) < 1e-14


# ---------------------------------------------------------------- matvec and symmetrisation
@pytest.mark.parametrize("theta", [1.0, 0.5, 0.8])
def test_matvec_vs_dense(theta):
    prob = ds.Problem(4, 7, theta, 1e-3, a_edges=synth.variable_coefficient_edges(4))
    v = rng.standard_normal(2 * prob.m * prob.n)
    A = pc.dense_A(prob)
    assert np.abs(A - A.T).max() < 1e-10
    assert np.abs(op.matvec_A(prob, v) - A @ v).max() < 1e-10
    assert np.abs(op.matvec_A_hat(prob, v) - pc.dense_A_hat(prob) @ v).max() < 1e-10


@pytest.mark.parametrize("theta", [1.0, 0.5, 0.8])
def test_symmetrised_system_equals_paper_system(theta):
    """A [sqrt(g) B2 y; B2^T p] = [g_tilde; sqrt(g) f_tilde] for the solution of A_tilde (Eq. main_system)."""
    N, n = 5, 6
    prob = ds.Problem(N, n, theta, 3e-3)
    g = rng.standard_normal((n + 1, N * N)); f = rng.standard_normal((n + 1, N * N)); y0 = rng.standard_normal(N * N)
    y, p = ds.solve_direct(prob, g, f, y0)
    x = ds.to_symmetric_unknowns(prob, y, p)
    b = ds.rhs_minres(prob, g, f, y0)
    assert np.abs(op.matvec_A(prob, x) - b).max() < 1e-10 * np.abs(b).max()
    bh = ds.rhs_gmres(prob, g, f, y0)
    assert np.abs(op.matvec_A_hat(prob, x) - bh).max() < 1e-10 * np.abs(bh).max()
    yr, pr = ds.recover(prob, x)
    assert np.abs(yr - y).max() < 1e-12 * np.abs(y).max() and np.abs(pr - p).max() < 1e-12 * np.abs(p).max()


# ---------------------------------------------------------------- P9: Krylov vs sparse direct
@pytest.mark.parametrize("theta,zeta", [(1.0, math.pi), (0.5, math.pi), (1.0, 0.0)])
def test_krylov_vs_direct(theta, zeta):
    N, n = 7, 8
    prob = ds.Problem(N, n, theta, 1e-3, zeta=zeta)
    g = synth.random_target(N, n, seed=5); f = synth.manufactured_source(N, n)
    yd, pd = ds.solve_direct(prob, g, f)
    x, info = kr.minres(lambda z: op.matvec_A(prob, z), ds.rhs_minres(prob, g, f),
                        lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-12)
    assert info.converged
    y, p = ds.recover(prob, x)
    assert np.abs(y - yd).max() < 1e-9 * np.abs(yd).max() and np.abs(p - pd).max() < 1e-9 * np.abs(pd).max()
    x, info = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), ds.rhs_gmres(prob, g, f),
                        lambda r: pc.apply_ps_inv(prob, r), tol=1e-12)
    assert info.converged
    y, p = ds.recover(prob, x)
    assert np.abs(y - yd).max() < 1e-9 * np.abs(yd).max() and np.abs(p - pd).max() < 1e-9 * np.abs(pd).max()


def test_krylov_variable_a_fgmres_vs_direct():
    N, n = 7, 8
    prob = ds.Problem(N, n, 0.5, 1e-4, a_edges=synth.variable_coefficient_edges(N))
    g = synth.random_target(N, n, seed=6); f = synth.manufactured_source(N, n)
    yd, pd = ds.solve_direct(prob, g, f)
    x, info = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), ds.rhs_gmres(prob, g, f),
                        lambda r: pc.apply_mg_ps_inv(prob, r), tol=1e-11)
    assert info.converged and info.iterations <= 25
    y, p = ds.recover(prob, x)
    assert np.abs(y - yd).max() < 1e-8 * np.abs(yd).max()


# ---------------------------------------------------------------- P10: manufactured solution
def test_config0_manufactured_solution():
    inst = synth.config0()
    prob = ds.Problem.from_instance(inst)
    x1, x2 = synth.grid(prob.N)
    ylev = synth.times(prob.n)[:, None] * (np.sin(math.pi * x1) * np.sin(math.pi * x2)).reshape(1, -1)
    gt, ft, y_ex, p_ex = ds.manufactured_rhs(prob, ylev, inst.g)
    b = np.concatenate([gt.ravel(), math.sqrt(prob.gamma) * ft.ravel()])
    x, info = kr.minres(lambda z: op.matvec_A(prob, z), b, lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-10)
    assert info.converged and info.relres <= 1e-10
    y, p = ds.recover(prob, x)
    cond = 100.0
    assert np.abs(y - y_ex).max() / np.abs(y_ex).max() < cond * 1e-10
    assert np.abs(p - p_ex).max() / np.abs(p_ex).max() < cond * 1e-10


# ---------------------------------------------------------------- P11: flat iteration counts
def test_iteration_counts_flat_example1():
    """Example 1 (the paper's data), Crank-Nicolson: counts do not grow as h and tau halve."""
    its = []
    for k in (4, 5, 6):
        N, n = 2 ** k - 1, 2 ** k
        prob = ds.Problem(N, n, 0.5, 1e-2)
        g, f, ye, _ = synth.example1_data(N, n)
        _, im = kr.minres(lambda z: op.matvec_A(prob, z), ds.rhs_minres(prob, g, f, ye[0]),
                          lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-8)
        _, ig = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), ds.rhs_gmres(prob, g, f, ye[0]),
                          lambda r: pc.apply_ps_inv(prob, r), tol=1e-8)
        its.append((im.iterations, ig.iterations))
    assert max(i for i, _ in its) - min(i for i, _ in its) <= 1, its
    assert max(j for _, j in its) - min(j for _, j in its) <= 1, its


def test_iteration_counts_random_target_backward_euler():
    """Random multi-mode target, backward Euler: GMRES-P_S stays flat; MINRES-|P_S| grows slowly
    (Thm 3.3 bounds the outliers by 4m, which grows with N)."""
    gm, mr = [], []
    for N, n in ((7, 8), (15, 16), (31, 32)):
        prob = ds.Problem(N, n, 1.0, 1e-2)
        g = synth.random_target(N, n, seed=7); f = synth.manufactured_source(N, n)
        _, im = kr.minres(lambda z: op.matvec_A(prob, z), ds.rhs_minres(prob, g, f),
                          lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-8)
        _, ig = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), ds.rhs_gmres(prob, g, f),
                          lambda r: pc.apply_ps_inv(prob, r), tol=1e-8)
        mr.append(im.iterations); gm.append(ig.iterations)
    assert max(gm) - min(gm) <= 1, gm
    assert all(0 <= b - a <= 3 for a, b in zip(mr, mr[1:])), mr


# ---------------------------------------------------------------- P13: Table 1
def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_example1_cn.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                g, k, dof, gi, ge, mi, me = line.split()
                rows.append((float(g), int(k), int(dof), int(gi), float(ge), int(mi), float(me)))
    return rows


def _check_table1_row(row):
    gamma, k, dof, git, geh, mit, meh = row
    N, n = 2 ** k - 1, 2 ** k
    assert 2 * N * N * n == dof
    prob = ds.Problem(N, n, 0.5, gamma)
    g, f, ye, pe = synth.example1_data(N, n)
    x, info = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), ds.rhs_gmres(prob, g, f, ye[0]),
                        lambda r: pc.apply_ps_inv(prob, r), tol=1e-8)
    assert info.converged and info.iterations == git
    y, p = ds.recover(prob, x)
    eh = ds.error_eh(prob, y, p, ye, pe)
    assert abs(eh - geh) / geh < 0.01, (eh, geh)          # printed to 3 digits
    x, info = kr.minres(lambda z: op.matvec_A(prob, z), ds.rhs_minres(prob, g, f, ye[0]),
                        lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-8)
    assert info.converged and info.iterations == mit
    y, p = ds.recover(prob, x)
    eh = ds.error_eh(prob, y, p, ye, pe)
    # the MINRES error includes solver error, which depends on the stopping rule's norm
    assert abs(eh - meh) / meh < 0.15, (eh, meh)


@pytest.mark.parametrize("row", [r for r in _table1() if r[1] == 5], ids=lambda r: f"g{r[0]:g}-h2^-{r[1]}")
def test_table1_example1(row):
    _check_table1_row(row)


@pytest.mark.slow
@pytest.mark.parametrize("row", [r for r in _table1() if r[1] == 6], ids=lambda r: f"g{r[0]:g}-h2^-{r[1]}")
def test_table1_example1_h64(row):
    _check_table1_row(row)


# ---------------------------------------------------------------- multigrid
def test_multigrid_transfer_and_convergence():
    N = 15
    R = rng.standard_normal((N, N))
    E = rng.standard_normal(((N - 1) // 2,) * 2)
    # full weighting = (1/4) x bilinear prolongation transposed
    assert abs(np.sum(mg.restrict(R) * E) - 0.25 * np.sum(R * mg.prolong(E, N))) < 1e-12
    prob = ds.Problem(N, 4, 0.5, 1e-4)
    ax, ay = prob.edges()
    levels = mg.hierarchy(N, ax, ay, prob.tau)
    assert [L.N for L in levels] == [15, 7, 3, 1]
    mu = np.array([0.3 + 2.0j, 1e-3j, 5.0 + 0j, 0.7j])[:, None, None]
    Rr = rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))
    lam = prob.tau * spc.kappa2d(N)
    exact = spc.dst2((spc.dst2(Rr.reshape(4, -1), N) / (mu.reshape(4, 1) + lam.reshape(1, -1))), N).reshape(4, N, N)
    errs = [np.abs(mg.solve(levels, mu, Rr, c) - exact).max() / np.abs(exact).max() for c in (1, 2, 6)]
    assert errs[0] < 0.5 and errs[1] < errs[0] and errs[2] < 1e-4
    # linearity of the fixed-count V-cycle
    R2 = rng.standard_normal((4, N, N)) + 0j
    assert np.abs(mg.solve(levels, mu, Rr + 2 * R2, 2) - mg.solve(levels, mu, Rr, 2) - 2 * mg.solve(levels, mu, R2, 2)).max() < 1e-10


def test_backward_euler_convergence_order():
    """Backward Euler on Example 1: e_h = O(tau + h^2) with h ~ tau, so halving both halves e_h
    (consistency of the theta = 1 right-hand side and recovery; the paper prints no theta = 1 data)."""
    errs = []
    for k in (3, 4, 5):
        N, n = 2 ** k - 1, 2 ** k
        prob = ds.Problem(N, n, 1.0, 1e-2)
        g, f, ye, pe = synth.example1_data(N, n)
        x, info = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), ds.rhs_gmres(prob, g, f, ye[0]),
                            lambda r: pc.apply_ps_inv(prob, r), tol=1e-12)
        y, p = ds.recover(prob, x)
        errs.append(ds.error_eh(prob, y, p, ye, pe))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.7 < r1 < 2.5 and 1.7 < r2 < 2.3, errs


def test_multigrid_contraction_variable_a():
    """The V-cycle for (mu I + tau K) with variable a contracts the error by a grid-independent factor."""
    rates = []
    for N in (15, 31, 63):
        prob = ds.Problem(N, 4, 0.5, 1e-4, a_edges=synth.variable_coefficient_edges(N))
        ax, ay = prob.edges()
        levels = mg.hierarchy(N, ax, ay, prob.tau)
        mu = np.array([1e-3j, 0.05j, 1.0 + 0.5j])[:, None, None]
        Z = rng.standard_normal((3, N, N)) + 0j
        L = levels[0]
        R = mu * Z + L.tau * L.K(Z)
        e1 = np.abs(mg.solve(levels, mu, R, 1) - Z).max() / np.abs(Z).max()
        e3 = np.abs(mg.solve(levels, mu, R, 3) - Z).max() / np.abs(Z).max()
        rates.append((e3 / e1) ** 0.5)
    assert max(rates) < 0.2, rates
    assert rates[-1] < 1.5 * rates[0] + 0.02, rates


# ---------------------------------------------------------------- omega sweep (real-part reading)
def test_real_part_preconditioner_is_the_mean_of_omega_and_conjugate():
    """For real v, Re(|P_S(omega)|^{-1}) v equals the mean of the applies at omega and conj(omega)
    (zeta and 2 pi - zeta), each taken complex; and it is symmetric positive definite."""
    N, n, theta, gamma, zeta = 3, 4, 1.0, 1e-2, 1.1
    p1 = ds.Problem(N, n, theta, gamma, zeta=zeta)
    p2 = ds.Problem(N, n, theta, gamma, zeta=2 * math.pi - zeta)
    m = 2 * p1.m * n
    E = np.eye(m)
    R = np.stack([pc.apply_abs_ps_inv(p1, E[:, k]) for k in range(m)], axis=1)
    C1 = np.linalg.inv(pc.dense_abs_P_S(p1))
    C2 = np.linalg.inv(pc.dense_abs_P_S(p2))
    assert np.abs(R - 0.5 * (C1 + C2)).max() < 1e-10 * np.abs(R).max()
    assert np.abs(R - R.T).max() < 1e-10 * np.abs(R).max()
    assert np.linalg.eigvalsh(0.5 * (R + R.T)).min() > 0


def test_zeta_sweep_half_pi_beats_zero_and_pi():
    """MINRES-|P_S| iterations on the bench family (N = 31, n = 32, gamma = 1e-2): under the
    real-part reading, zeta = pi/2 needs fewer iterations than zeta = 0 and zeta = pi (a measured
    property of that reading, kept as a regression check, not a statement of the paper)."""
    N, n, gamma = 31, 32, 1e-2
    g = synth.random_target(N, n, seed=1); f = synth.manufactured_source(N, n)
    its = {}
    for zeta in (0.0, math.pi / 2, math.pi):
        prob = ds.Problem(N, n, 1.0, gamma, zeta=zeta)
        b = ds.rhs_minres(prob, g, f)
        _, info = kr.minres(lambda z: op.matvec_A(prob, z), b, lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-8)
        assert info.converged
        its[zeta] = info.iterations
    assert its[math.pi / 2] < its[math.pi] and its[math.pi / 2] < its[0.0], its


@pytest.mark.parametrize("method", ["minres", "fgmres"])
def test_krylov_stall_exit_below_attainable_accuracy(method):
    """Asked for a residual float64 cannot reach, the stall exit returns within a few iterations of
    the attainable accuracy, unconverged, with its true residual -- and without stall the same
    solve, to a reachable tolerance, is unchanged by the keyword."""
    N, n = 7, 8
    prob = ds.Problem(N, n, 1.0, 1e-2)
    g = synth.random_target(N, n, seed=3); f = synth.manufactured_source(N, n)
    b = ds.rhs_minres(prob, g, f)
    A = lambda z: op.matvec_A(prob, z)
    M = lambda r: pc.apply_abs_ps_inv(prob, r)
    solver = kr.minres if method == "minres" else kr.fgmres
    x, info = solver(A, b, M, tol=1e-30, maxit=400, stall=1e-3)
    assert not info.converged and info.relres < 1e-13 and info.iterations < 100, info.iterations
    x1, i1 = solver(A, b, M, tol=1e-8)
    x2, i2 = solver(A, b, M, tol=1e-8, stall=1e-3)
    assert i1.iterations == i2.iterations and np.array_equal(x1, x2)


def test_stored_oracle_solution_sample_reproduces():
    """The stored oracle solution of the smallest sampled uneven-batch instance (N = 63, n = 32)
    is what the oracle computes now: a fresh MINRES-|P_S| solve to 1e-10 lies within 1e-9 of it
    on the stored positions, and the stored norm is that of the fresh solve."""
    from oracle import reference_solutions as rs
    s = rs.read("cfg3_3")
    if s is None:
        pytest.skip("no stored sample")
    inst = synth.config3()[3]
    prob = ds.Problem.from_instance(inst)
    b = ds.rhs_minres(prob, inst.g, inst.f)
    x, info = kr.minres(lambda z: op.matvec_A(prob, z), b, lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-10)
    assert info.converged and x.size == s[0]
    assert rs.sampled_forward_error("cfg3_3", x) <= 1e-9
    assert abs(np.linalg.norm(x) - s[1]) <= 1e-9 * s[1]

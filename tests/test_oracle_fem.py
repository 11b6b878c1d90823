"""Pins of the oracle's finite-element route (M != I, the general M_m, K_m of Sec. 1 with bilinear
elements on the Dirichlet grid) against facts independent of its own formulas:
  * the 1D and 2D matrices against element-by-element assembly of the linear and bilinear element
    matrices (a route that shares nothing with the tensor-product formulas);
  * the sine basis diagonalises M1 and K1 with the textbook eigenvalues;
  * the symmetrised system of Eq. (main_system), solved and mapped back through the change of
    variables, equals a sparse direct solve of the unsymmetrised system of Eq. (matrix_A_before);
  * the fast preconditioner applies equal their dense constructions with K~ = M^{-1/2} K M^{-1/2};
  * Example 1 solved with elements converges at second order, and GMRES-P_S / MINRES-|P_S| take
    Table 1's iteration counts (the paper states that its preconditioners apply to finite elements
    with minimal modification; it prints no finite-element numbers).
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import discretisation as ds
from oracle import krylov as kr
from oracle import operators as op
from oracle import precond as pc
from oracle import spectra as spc


def _elements_1d(N):
    """Linear elements on N + 2 nodes (boundary included), element matrices (h/6)[2 1; 1 2] and
    (1/h)[1 -1; -1 1], boundary rows and columns dropped."""
    h = 1.0 / (N + 1)
    M = np.zeros((N + 2, N + 2)); K = np.zeros((N + 2, N + 2))
    for e in range(N + 1):
        idx = [e, e + 1]
        M[np.ix_(idx, idx)] += h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
        K[np.ix_(idx, idx)] += 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    return M[1:-1, 1:-1], K[1:-1, 1:-1]


def _elements_2d(N):
    """Bilinear elements on the (N+2)^2 node grid: for the element with corners (i, j), (i+1, j),
    (i+1, j+1), (i, j+1), mass (h^2/36)[[4,2,1,2],[2,4,2,1],[1,2,4,2],[2,1,2,4]] and Laplacian
    stiffness (1/6)[[4,-1,-2,-1],[-1,4,-1,-2],[-2,-1,4,-1],[-1,-2,-1,4]]; boundary nodes dropped;
    node (i, j) (1-based interior) at index (i-1) + (j-1) N."""
    h = 1.0 / (N + 1)
    n1 = N + 2
    Me = h * h / 36.0 * np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]], dtype=float)
    Ke = 1.0 / 6.0 * np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]], dtype=float)
    M = np.zeros((n1 * n1, n1 * n1)); K = np.zeros_like(M)
    for j in range(n1 - 1):
        for i in range(n1 - 1):
            idx = [i + j * n1, (i + 1) + j * n1, (i + 1) + (j + 1) * n1, i + (j + 1) * n1]
            M[np.ix_(idx, idx)] += Me
            K[np.ix_(idx, idx)] += Ke
    inner = [i + j * n1 for j in range(1, n1 - 1) for i in range(1, n1 - 1)]
    return M[np.ix_(inner, inner)], K[np.ix_(inner, inner)]


@pytest.mark.parametrize("N", [1, 4, 9])
def test_1d_matrices_from_element_assembly(N):
    M, K = _elements_1d(N)
    assert np.abs(ds.mass_1d(N).toarray() - M).max() < 1e-15
    assert np.abs(ds.stiffness_1d(N).toarray() - K).max() < 1e-12


@pytest.mark.parametrize("N", [2, 5])
def test_2d_matrices_from_bilinear_element_assembly(N):
    M, K = _elements_2d(N)
    prob = ds.Problem(N, 4, 1.0, 1e-2, fem=True, a0=0.7)
    assert np.abs(ds.M_sparse(prob).toarray() - M).max() < 1e-15
    assert np.abs(ds.K_sparse(prob).toarray() - 0.7 * K).max() < 1e-12
    u = np.random.default_rng(1).standard_normal((3, N * N))
    assert np.abs(ds.apply_K(prob, u) - (0.7 * K @ u.T).T).max() < 1e-12
    assert np.abs(ds.apply_M(prob, u) - (M @ u.T).T).max() < 1e-15


def test_sine_basis_diagonalises_the_element_matrices():
    N = 11
    S = spc.dst_matrix(N)
    M1, K1 = ds.mass_1d(N).toarray(), ds.stiffness_1d(N).toarray()
    assert np.abs(S @ M1 @ S - np.diag(spc.mass_eigenvalues(N))).max() < 1e-14
    assert np.abs(S @ K1 @ S - np.diag(spc.stiffness_eigenvalues(N))).max() < 1e-12
    prob = ds.Problem(N, 4, 1.0, 1e-2, fem=True)
    u = np.random.default_rng(2).standard_normal(N * N)
    Md = ds.M_sparse(prob).toarray()
    w, V = np.linalg.eigh(Md)
    Mh = (V * np.sqrt(w)) @ V.T
    assert np.abs(ds.apply_M_power(prob, u, 0.5) - Mh @ u).max() < 1e-14
    assert np.abs(ds.apply_M_power(prob, ds.apply_M_power(prob, u, 0.5), -0.5) - u).max() < 1e-12


@pytest.mark.parametrize("theta", [1.0, 0.5, 0.75])
@pytest.mark.parametrize("with_y0", [False, True])
def test_symmetrised_solve_equals_direct_solve_of_the_element_system(theta, with_y0):
    N, n, gamma = 7, 8, 3e-2
    prob = ds.Problem(N, n, theta, gamma, fem=True)
    g = synth.random_target(N, n, seed=21); f = synth.manufactured_source(N, n)
    y0 = synth.random_vector(N * N, seed=22) if with_y0 else None
    yd, pd = ds.solve_direct(prob, g, f, y0)
    b = ds.rhs_minres(prob, g, f, y0)
    x, info = kr.minres(lambda z: op.matvec_A(prob, z), b, lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-13)
    y, p = ds.recover(prob, x)
    assert np.abs(y - yd).max() <= 1e-10 * np.abs(yd).max()
    assert np.abs(p - pd).max() <= 1e-10 * np.abs(pd).max()
    # the change of variables and its inverse
    assert np.abs(ds.to_symmetric_unknowns(prob, y, p) - x).max() <= 1e-12 * np.abs(x).max()


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_element_preconditioners_equal_dense_constructions(theta):
    N, n = 3, 4
    prob = ds.Problem(N, n, theta, 1e-2, fem=True)
    v = synth.random_vector(2 * prob.m * n, seed=23)
    dense = {"abs_ps": pc.dense_abs_P_S(prob), "ps": pc.dense_P_S(prob), "pms": pc.dense_P_MS(prob)}
    fast = {"abs_ps": pc.apply_abs_ps_inv, "ps": pc.apply_ps_inv, "pms": pc.apply_pms_inv}
    for kind in dense:
        ref = np.real(np.linalg.solve(dense[kind], v))
        out = fast[kind](prob, v)
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max(), kind
    A = pc.dense_A(prob)
    assert np.abs(A @ v - op.matvec_A(prob, v)).max() <= 1e-12 * np.abs(A @ v).max()


def test_example1_with_elements_converges_and_keeps_table1_counts():
    """Example 1 (Crank-Nicolson) discretised with bilinear elements: e_h drops by about 4 per
    refinement, and the iteration counts are Table 1's at h = 2^-5 (gamma = 1e-2: GMRES-P_S 3,
    MINRES-|P_S| 6)."""
    es = []
    for k in (4, 5):
        N, n = 2 ** k - 1, 2 ** k
        prob = ds.Problem(N, n, 0.5, 1e-2, fem=True)
        g, f, ye, pe = synth.example1_data(N, n)
        xg, ig = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), ds.rhs_gmres(prob, g, f, ye[0]),
                           lambda r: pc.apply_ps_inv(prob, r), tol=1e-10)
        es.append(ds.error_eh(prob, *ds.recover(prob, xg), ye, pe))
        if k == 5:
            x8, i8 = kr.fgmres(lambda z: op.matvec_A_hat(prob, z), ds.rhs_gmres(prob, g, f, ye[0]),
                               lambda r: pc.apply_ps_inv(prob, r), tol=1e-8)
            xm, im = kr.minres(lambda z: op.matvec_A(prob, z), ds.rhs_minres(prob, g, f, ye[0]),
                               lambda r: pc.apply_abs_ps_inv(prob, r), tol=1e-8)
            assert i8.iterations == 3 and im.iterations == 6, (i8.iterations, im.iterations)
    assert 3.5 < es[0] / es[1] < 4.5, es

"""Discretisation of the optimality system (paper Sec. 1): theta-scheme in time, 5-point
finite differences in space (M = I, K = -L), the all-at-once system of Eq. (main_system_before)
/ (matrix_A_before), its right-hand side, the symmetrising change of variables of
Eq. (main_system), and the error measure of Eq. (error_measure).

Two boundary conditions:
  dirichlet (Examples 1-2): N interior nodes per side, h = 1/(N+1), zero boundary values,
            conservative edge-weighted stencil (a(x) at cell-edge midpoints, or the constant a0).
            With fem=True the space discretisation is bilinear (Q1) finite elements on the same
            grid instead (Sec. 1: M_m the mass and K_m the stiffness matrix, both symmetric, M_m
            positive definite): M = M1 (x) M1, K = a0 (K1 (x) M1 + M1 (x) K1) with the 1D linear-
            element matrices M1 = (h/6) tridiag(1, 4, 1) and K1 = (1/h) tridiag(-1, 2, -1).  The
            symmetrised system then carries K~ = M^{-1/2} K M^{-1/2} (Eq. matrix_A), and the
            right-hand side and unknowns the M^{-1/2}, M^{1/2} factors of Eq. (main_system).
  neumann   (Example 3, homogeneous Neumann): N nodes per side *including* the boundary,
            x_i = i h, h = 1/(N-1), the constant coefficient a0, second differences with the
            ghost values mirrored across the boundary (u_{-1} = u_1, u_N = u_{N-2}).  This K is
            not symmetric; the paper's block matrices are formed with it as printed (K in both
            the state and the adjoint rows), which is why the Neumann A is not symmetric and the
            paper uses GMRES-P_S there.  Reading pinned by Table 4's e_h.

Vector layout: a time block holds the N*N spatial values with x1 fastest, index i + j*N.
The unknown y = [y^(1) .. y^(n)], p = [p^(0) .. p^(n-1)].
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.linalg import solve_banded


class Problem:
    """Parameters of one instance: N, n, theta, T, gamma, zeta, optional a(x) edge values,
    boundary condition bc ("dirichlet" or "neumann") and constant coefficient a0 (used when
    a_edges is None)."""

    def __init__(self, N, n, theta, gamma, T=1.0, zeta=math.pi, a_edges=None, bc="dirichlet", a0=1.0, fem=False):
        self.N, self.n = int(N), int(n)
        self.theta, self.gamma, self.T, self.zeta = float(theta), float(gamma), float(T), float(zeta)
        self.a_edges = None if a_edges is None else np.asarray(a_edges, dtype=np.float64)
        if bc not in ("dirichlet", "neumann"):
            raise ValueError("bc must be 'dirichlet' or 'neumann'")
        if bc == "neumann" and (a_edges is not None or self.N < 3):
            raise ValueError("neumann takes a constant coefficient and N >= 3")
        if fem and (bc != "dirichlet" or a_edges is not None):
            raise ValueError("the finite-element discretisation is built for Dirichlet data and a constant a")
        self.bc, self.a0, self.fem = bc, float(a0), bool(fem)

    @classmethod
    def from_instance(cls, inst):
        return cls(inst.N, inst.n, inst.theta, inst.gamma, inst.T, inst.zeta, inst.a_edges,
                   getattr(inst, "bc", "dirichlet"), getattr(inst, "a0", 1.0), getattr(inst, "fem", False))

    @property
    def m(self):
        return self.N * self.N

    @property
    def h(self):
        return 1.0 / (self.N - 1) if self.bc == "neumann" else 1.0 / (self.N + 1)

    @property
    def tau(self):
        return self.T / self.n

    @property
    def alpha(self):
        # alpha = tau / sqrt(gamma)   (Sec. 1, after Eq. matrix_A)
        return self.tau / math.sqrt(self.gamma)

    def edges(self):
        """(ax, ay): ax[j, e] couples nodes (e, j+1)-(e+1, j+1), shape (N, N+1);
        ay[e, i] couples nodes (i+1, e)-(i+1, e+1), shape (N+1, N).  a = 1 when not given."""
        N = self.N
        if self.a_edges is None:
            return self.a0 * np.ones((N, N + 1)), self.a0 * np.ones((N + 1, N))
        ax = self.a_edges[: N * (N + 1)].reshape(N, N + 1)
        ay = self.a_edges[N * (N + 1):].reshape(N + 1, N)
        return ax, ay


# ----------------------------------------------------------------------------------------
# Spatial operator K = -L_m (Sec. 1: M = I, K = -L for finite differences)
# ----------------------------------------------------------------------------------------

# ----------------------------------------------------------------------------------------
# Bilinear (Q1) finite elements on the Dirichlet grid (the M_m != I case of Sec. 1)
# ----------------------------------------------------------------------------------------

def mass_1d(N):
    """1D linear-element mass matrix on N interior nodes, h = 1/(N+1): (h/6) tridiag(1, 4, 1)."""
    h = 1.0 / (N + 1)
    return sp.diags([np.full(N - 1, h / 6), np.full(N, 4 * h / 6), np.full(N - 1, h / 6)], [-1, 0, 1], format="csr")


def stiffness_1d(N):
    """1D linear-element stiffness matrix on N interior nodes: (1/h) tridiag(-1, 2, -1)."""
    h = 1.0 / (N + 1)
    return sp.diags([np.full(N - 1, -1 / h), np.full(N, 2 / h), np.full(N - 1, -1 / h)], [-1, 0, 1], format="csr")


def _along(A1, U, axis):
    """Apply the 1D matrix A1 along one grid axis of U[..., j, i] (axis -1: x1, -2: x2)."""
    V = np.moveaxis(U, axis, -1)
    sh = V.shape
    W = (A1 @ V.reshape(-1, sh[-1]).T).T.reshape(sh)
    return np.moveaxis(W, -1, axis)


def apply_M(prob: Problem, u: np.ndarray) -> np.ndarray:
    """M u: the identity for finite differences, M1 (x) M1 for finite elements."""
    if not prob.fem:
        return np.array(u, dtype=np.float64, copy=True)
    N = prob.N
    M1 = mass_1d(N)
    U = u.reshape(u.shape[:-1] + (N, N))
    return _along(M1, _along(M1, U, -1), -2).reshape(u.shape)


def M_sparse(prob: Problem) -> sp.csr_matrix:
    if not prob.fem:
        return sp.identity(prob.m, format="csr")
    M1 = mass_1d(prob.N)
    return sp.kron(M1, M1, format="csr")


def apply_M_power(prob: Problem, u: np.ndarray, power: float) -> np.ndarray:
    """M^power u (power = 1/2 or -1/2 in Eq. main_system).  M is symmetric positive definite and
    its square roots are taken through its eigendecomposition, for which the orthonormal DST-I
    S_N (x) S_N serves (it diagonalises M1: the textbook eigenvectors of a symmetric tridiagonal
    Toeplitz matrix)."""
    if not prob.fem:
        return np.array(u, dtype=np.float64, copy=True)
    from . import spectra as spc
    lam = spc.mass_eigenvalues_2d(prob.N).ravel()
    return spc.dst2(lam ** power * spc.dst2(u, prob.N), prob.N)


def apply_K(prob: Problem, u: np.ndarray) -> np.ndarray:
    """K u for u of shape (..., N*N).  Dirichlet: conservative 5-point stencil with zero boundary
    data, (K u)_ij = sum over the four edges of a_edge (u_ij - u_neighbour) / h^2.  Neumann:
    a0 (4 u_ij - sum of the four neighbours) / h^2 with mirrored ghost values.  Finite elements:
    a0 (K1 (x) M1 + M1 (x) K1) u."""
    N = prob.N
    if prob.fem:
        U = u.reshape(u.shape[:-1] + (N, N))
        M1, K1 = mass_1d(N), stiffness_1d(N)
        out = _along(M1, _along(K1, U, -1), -2) + _along(K1, _along(M1, U, -1), -2)
        return (prob.a0 * out).reshape(u.shape)
    if prob.bc == "neumann":
        U = u.reshape(u.shape[:-1] + (N, N))
        # mirror: padded index 0 holds u_1, padded index N+1 holds u_{N-2}
        P = np.pad(U, [(0, 0)] * (U.ndim - 2) + [(1, 1), (1, 1)], mode="reflect")
        c = P[..., 1:-1, 1:-1]
        nb = P[..., 1:-1, :-2] + P[..., 1:-1, 2:] + P[..., :-2, 1:-1] + P[..., 2:, 1:-1]
        return (prob.a0 * (4.0 * c - nb) / prob.h ** 2).reshape(u.shape)
    ax, ay = prob.edges()
    U = u.reshape(u.shape[:-1] + (N, N))             # [..., j, i]
    P = np.zeros(u.shape[:-1] + (N + 2, N + 2), dtype=u.dtype)
    P[..., 1:-1, 1:-1] = U
    c = P[..., 1:-1, 1:-1]
    left, right = P[..., 1:-1, :-2], P[..., 1:-1, 2:]
    down, up = P[..., :-2, 1:-1], P[..., 2:, 1:-1]
    out = (ax[:, :-1] * (c - left) + ax[:, 1:] * (c - right)
           + ay[:-1, :] * (c - down) + ay[1:, :] * (c - up)) / prob.h ** 2
    return out.reshape(u.shape)


def apply_K_tilde(prob: Problem, u: np.ndarray) -> np.ndarray:
    """K~ u = M^{-1/2} K M^{-1/2} u, the spatial operator of Eq. (matrix_A) (K itself when M = I)."""
    if not prob.fem:
        return apply_K(prob, u)
    return apply_M_power(prob, apply_K(prob, apply_M_power(prob, u, -0.5)), -0.5)


def K_sparse(prob: Problem) -> sp.csr_matrix:
    """K as a sparse m x m matrix, assembled entry by entry from the same stencil definition."""
    N = prob.N
    if prob.fem:
        M1, K1 = mass_1d(N), stiffness_1d(N)
        return (prob.a0 * (sp.kron(M1, K1) + sp.kron(K1, M1))).tocsr()
    if prob.bc == "neumann":
        c = prob.a0 / prob.h ** 2
        rows, cols, vals = [], [], []
        for j in range(N):
            for i in range(N):
                r = i + j * N
                rows.append(r); cols.append(r); vals.append(4.0 * c)
                # a missing neighbour is the mirror image of the one across the node
                for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                    ii, jj = i + di, j + dj
                    if ii < 0 or ii > N - 1:
                        ii = i - di
                    if jj < 0 or jj > N - 1:
                        jj = j - dj
                    rows.append(r); cols.append(ii + jj * N); vals.append(-c)
        return sp.csr_matrix((vals, (rows, cols)), shape=(N * N, N * N))
    ax, ay = prob.edges()
    h2 = prob.h ** 2
    rows, cols, vals = [], [], []
    for j in range(N):
        for i in range(N):
            r = i + j * N
            aL, aR, aD, aU = ax[j, i], ax[j, i + 1], ay[j, i], ay[j + 1, i]
            rows.append(r); cols.append(r); vals.append((aL + aR + aD + aU) / h2)
            if i > 0:
                rows.append(r); cols.append(r - 1); vals.append(-aL / h2)
            if i < N - 1:
                rows.append(r); cols.append(r + 1); vals.append(-aR / h2)
            if j > 0:
                rows.append(r); cols.append(r - N); vals.append(-aD / h2)
            if j < N - 1:
                rows.append(r); cols.append(r + N); vals.append(-aU / h2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N * N, N * N))


# ----------------------------------------------------------------------------------------
# Time factors B_n^(1), B_n^(2), B_n = B^(1) (B^(2))^{-1}   (Sec. 1)
# ----------------------------------------------------------------------------------------

def B1_dense(n):
    return np.eye(n) - np.eye(n, k=-1)


def B2_dense(n, theta):
    return theta * np.eye(n) + (1.0 - theta) * np.eye(n, k=-1)


def Bn_closed_form(n, theta):
    """Lower-triangular Toeplitz B_n with the explicit entries printed in Sec. 1:
    diagonal 1/theta, first subdiagonal -1/theta^2, k-th subdiagonal -(theta-1)^(k-1)/theta^(k+1)."""
    col = np.zeros(n)
    col[0] = 1.0 / theta
    for k in range(1, n):
        col[k] = -((theta - 1.0) ** (k - 1)) / theta ** (k + 1)
    B = np.zeros((n, n))
    for k in range(n):
        B += np.diag(np.full(n - k, col[k]), -k)
    return B


def _solve_B2(theta, x, transpose=False):
    """(B2^{-1} (x) I) x (lower bidiagonal solve along time) or (B2^{-T} (x) I) x (upper)."""
    n = x.shape[0]
    ab = np.zeros((2, n))
    if not transpose:
        ab[0, :] = theta
        ab[1, :-1] = 1.0 - theta
        return solve_banded((1, 0), ab, x)
    ab[0, 1:] = 1.0 - theta
    ab[1, :] = theta
    return solve_banded((0, 1), ab, x)


def apply_B1(x, transpose=False):
    """(B1 (x) I) x: x_t - x_{t-1};  transpose: x_t - x_{t+1}.  x has shape (n, m)."""
    out = x.copy()
    if not transpose:
        out[1:] -= x[:-1]
    else:
        out[:-1] -= x[1:]
    return out


def apply_Bn(theta, x, transpose=False):
    """(B_n (x) I) x with B_n applied as B^(1) then (B^(2))^{-1} (B_n = B1 B2^{-1} = B2^{-1} B1)."""
    return _solve_B2(theta, apply_B1(x, transpose), transpose)


# ----------------------------------------------------------------------------------------
# All-at-once system (Eqs. main_system_before, matrix_A_before) and right-hand side
# ----------------------------------------------------------------------------------------

def tilde_rhs(prob: Problem, g, f, y0=None):
    """(g_tilde, f_tilde), each (n, m), from samples g, f of shape (n+1, m) at t_k = k tau (Sec. 1):
      f_tilde^(r) = M tau (theta f^(r) + (1-theta) f^(r-1)) [+ (M - (1-theta) tau K) y0 for r = 1]
      g_tilde^(r) = tau M (theta g^(r-1) + (1-theta) g^(r)) [- tau (1-theta) M y0 for r = 1]."""
    th, tau = prob.theta, prob.tau
    g = np.asarray(g, dtype=np.float64); f = np.asarray(f, dtype=np.float64)
    ft = apply_M(prob, tau * (th * f[1:] + (1.0 - th) * f[:-1]))
    gt = apply_M(prob, tau * (th * g[:-1] + (1.0 - th) * g[1:]))
    if y0 is not None:
        y0 = np.asarray(y0, dtype=np.float64)
        ft[0] += apply_M(prob, y0) - (1.0 - th) * tau * apply_K(prob, y0)
        gt[0] -= tau * (1.0 - th) * apply_M(prob, y0)
    return gt, ft


def rhs_minres(prob, g, f, y0=None):
    """b = [g; sqrt(gamma) f] of Eq. (main_system), g = (I (x) M^{-1/2}) g_tilde and
    f = (I (x) M^{-1/2}) f_tilde, flattened to 2mn."""
    gt, ft = tilde_rhs(prob, g, f, y0)
    gs, fs = apply_M_power(prob, gt, -0.5), apply_M_power(prob, ft, -0.5)
    return np.concatenate([gs.ravel(), math.sqrt(prob.gamma) * fs.ravel()])


def rhs_gmres(prob, g, f, y0=None):
    """b_hat = [sqrt(gamma) f; g] of Eq. (main_system_nonsym)."""
    gt, ft = tilde_rhs(prob, g, f, y0)
    gs, fs = apply_M_power(prob, gt, -0.5), apply_M_power(prob, ft, -0.5)
    return np.concatenate([math.sqrt(prob.gamma) * fs.ravel(), gs.ravel()])


def A_tilde_sparse(prob: Problem) -> sp.csr_matrix:
    """The unsymmetrised block matrix of Eq. (matrix_A_before):
      [[tau B2 (x) M,          B1^T (x) M + tau B2^T (x) K],
       [B1 (x) M + tau B2 (x) K,  -(tau/gamma) B2^T (x) M ]]  acting on [y; p]."""
    n, th, tau, gam = prob.n, prob.theta, prob.tau, prob.gamma
    I = M_sparse(prob)
    K = K_sparse(prob)
    B1 = sp.csr_matrix(B1_dense(n)); B2 = sp.csr_matrix(B2_dense(n, th))
    top = sp.hstack([tau * sp.kron(B2, I), sp.kron(B1.T, I) + tau * sp.kron(B2.T, K)])
    bot = sp.hstack([sp.kron(B1, I) + tau * sp.kron(B2, K), -(tau / gam) * sp.kron(B2.T, I)])
    return sp.vstack([top, bot]).tocsr()


def solve_direct(prob, g, f, y0=None):
    """Sparse direct solve of A_tilde [y; p] = [g_tilde; f_tilde]; returns (y, p), each (n, m)."""
    gt, ft = tilde_rhs(prob, g, f, y0)
    sol = spla.spsolve(A_tilde_sparse(prob).tocsc(), np.concatenate([gt.ravel(), ft.ravel()]))
    mn = prob.m * prob.n
    return sol[:mn].reshape(prob.n, prob.m), sol[mn:].reshape(prob.n, prob.m)


# ----------------------------------------------------------------------------------------
# Symmetrising change of variables (Eq. main_system) and its inverse
# ----------------------------------------------------------------------------------------

def to_symmetric_unknowns(prob, y, p):
    """x = [sqrt(gamma) (B2 (x) M^{1/2}) y ; (B2^T (x) M^{1/2}) p]."""
    th = prob.theta
    yt = th * y.copy(); yt[1:] += (1.0 - th) * y[:-1]
    pt = th * p.copy(); pt[:-1] += (1.0 - th) * p[1:]
    yt, pt = apply_M_power(prob, yt, 0.5), apply_M_power(prob, pt, 0.5)
    return np.concatenate([math.sqrt(prob.gamma) * yt.ravel(), pt.ravel()])


def recover(prob, x):
    """Inverse of the change of variables: y = (B2^{-1} (x) M^{-1/2}) x1 / sqrt(gamma),
    p = (B2^{-T} (x) M^{-1/2}) x2; returns (y, p), each (n, m)."""
    mn = prob.m * prob.n
    x1 = x[:mn].reshape(prob.n, prob.m); x2 = x[mn:].reshape(prob.n, prob.m)
    y = apply_M_power(prob, _solve_B2(prob.theta, x1), -0.5) / math.sqrt(prob.gamma)
    p = apply_M_power(prob, _solve_B2(prob.theta, x2, transpose=True), -0.5)
    return y, p


# ----------------------------------------------------------------------------------------
# Discrete manufactured solution and error measure
# ----------------------------------------------------------------------------------------

def manufactured_rhs(prob, y_levels, g):
    """RHS (g_tilde, f_tilde) whose exact discrete solution has the state y^(k) = y_levels[k]
    (k = 1..n, y0 = y_levels[0]) for a given target g: the adjoint block rows of A_tilde are
    marched backward for p (p^(n) = 0), then f_tilde is read off the state block rows."""
    n, th, tau = prob.n, prob.theta, prob.tau
    gt, _ = tilde_rhs(prob, g, np.zeros_like(g), y_levels[0])
    Ks = K_sparse(prob)
    I = sp.identity(prob.m, format="csc")
    lhs = (I + tau * th * Ks).tocsc()
    P = np.zeros((n + 1, prob.m))     # p^(0..n), p^(n) = 0
    for k in range(n - 1, -1, -1):
        # adjoint row k: (I + tau th K) p^k - (I - tau (1-th) K) p^{k+1}
        #                + tau (th y^{k+1} + (1-th) y^k) = g_tilde^(k+1)   (y^0 term moved for k=0)
        rhs = gt[k] + (P[k + 1] - tau * (1.0 - th) * (Ks @ P[k + 1])) - tau * th * y_levels[k + 1]
        if k > 0:
            rhs -= tau * (1.0 - th) * y_levels[k]
        P[k] = spla.spsolve(lhs, rhs)
    y = y_levels[1:]
    p = P[:-1]
    ft = np.empty((n, prob.m))
    for r in range(n):
        # state row r: (I + tau th K) y^(r+1) - (I - tau (1-th) K) y^(r) - (tau/gamma)(th p^r + (1-th) p^{r+1})
        ft[r] = (y_levels[r + 1] + tau * th * (Ks @ y_levels[r + 1])
                 - (tau / prob.gamma) * (th * P[r] + (1.0 - th) * P[r + 1]))
        if r > 0:
            ft[r] -= y_levels[r] - tau * (1.0 - th) * (Ks @ y_levels[r])
    return gt, ft, y, p


def error_eh(prob, y, p, y_exact, p_exact):
    """e_h of Eq. (error_measure): max over time blocks r of h * || [y^(r) - y(t_r); p^(r-1) - p(t_{r-1})] ||_2
    with y at t_1..t_n and p at t_0..t_{n-1} (discrete L2(Omega) norm on interior nodes)."""
    ey = y - y_exact[1:]
    ep = p - p_exact[:-1]
    per = np.sqrt(np.sum(ey ** 2, axis=1) + np.sum(ep ** 2, axis=1)) * prob.h
    return float(per.max())

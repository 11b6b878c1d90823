"""Preconditioner applications (paper Sec. 1, Sec. 3.5) and their dense constructions.

Fast routes (any size):
  apply_abs_ps_inv : |P_S|^{-1} v   three steps of Sec. 3.5 (MINRES route): U* v, scale by
                     1/sqrt(|lambda_k + tau kappa_pq|^2 + alpha^2), U w.
  apply_ps_inv     : P_S^{-1} v     (GMRES route): per mode the 2x2 system
                     [[lam, -alpha], [alpha, conj(lam)]] with lam = lambda_k(S_n) + tau kappa_pq.
  apply_pms_inv    : P_MS^{-1} v    per mode 1/(sqrt(|lambda_k|^2 + alpha^2) + tau kappa_pq);
                     with a(x) variable, the shifted solves use the multigrid V-cycle.
  apply_mg_ps_inv  : P_S^{-1} v for variable a(x): time transform, Lemma 3.14 decoupling of the
                     per-frequency 2x2 block, multigrid on (mu_k I + tau K) for both components.
Both halves use the same unitary Q = (F D / sqrt(n)) (x) (S_N (x) S_N)  [reading of the second
diagonal block of U, U~ in Sec. 3.5: S is normal, so S*S = SS* and the two blocks of |P_S| agree].
For zeta in {0, pi} the operators are real on real vectors; for other zeta the applied operator
is the real part of the complex one.

Neumann (Example 3): K is not symmetric, and P_S is formed as printed with K in both diagonal
blocks, [[calS, -alpha I], [alpha I, S_n^* (x) I + tau I (x) K]] (the paper's Sec. 1 formulas with
K_m in place, as for A).  Both blocks are diagonalised by (F D) (x) V^{-1} (x) V^{-1} with V the
scaled DCT-I basis (spectra.py), so apply_ps_inv runs the same per-mode 2x2 solve.  |P_S| and P_MS
belong to MINRES, which the nonsymmetric A excludes; they are not defined for Neumann here.

Dense routes (tiny sizes): the matrices exactly as Eqs. (matrix_S), (matrix_P_GMRES), (matrix_P),
(matrix_P_MS), (abs_ideal_matrix_H) define them.
"""
from __future__ import annotations

import math

import numpy as np

from . import spectra as spc
from . import multigrid as mg
from .discretisation import K_sparse, M_sparse, B1_dense, B2_dense


def _halves(prob, v):
    mn = prob.m * prob.n
    return v[:mn].reshape(prob.n, prob.m), v[mn:].reshape(prob.n, prob.m)


def _forward(prob, x):
    """Q-transform up to scaling: time (F D) then the 2D spatial transform (DST-I, or the scaled
    DCT-I basis for Neumann); x (n, m) real -> complex (n, m)."""
    return spc.space_forward(spc.time_forward(x, prob.zeta), prob.N, prob.bc)


def _inverse(prob, w):
    return spc.time_inverse(spc.space_inverse(w, prob.N, prob.bc), prob.zeta)


def _kappa2d(prob):
    """a0 (kappa_p + kappa_q): eigenvalues of K (constant coefficient); with finite elements, of
    K~ = M^{-1/2} K M^{-1/2}."""
    return prob.a0 * spc.kappa2d(prob.N, prob.bc, getattr(prob, "fem", False))


def _modes(prob):
    """lambda_k(S_n) + tau (kappa_p + kappa_q), shape (n, m)."""
    lam = spc.lam_Sn(prob.n, prob.theta, prob.zeta)
    return lam[:, None] + prob.tau * _kappa2d(prob).reshape(1, -1)


def _no_neumann(prob):
    if prob.bc == "neumann":
        raise ValueError("|P_S| and P_MS are MINRES preconditioners; the Neumann A is not symmetric")


def apply_abs_ps_inv(prob, v):
    """|P_S|^{-1} v (a = 1)."""
    _no_neumann(prob)
    W = 1.0 / np.sqrt(np.abs(_modes(prob)) ** 2 + prob.alpha ** 2)
    out = []
    for x in _halves(prob, v):
        out.append(np.real(_inverse(prob, W * _forward(prob, x))).ravel())
    return np.concatenate(out)


def apply_ps_inv(prob, v, real=True):
    """P_S^{-1} v (a = 1)."""
    lam = _modes(prob)
    a = prob.alpha
    x1, x2 = _halves(prob, v)
    r1, r2 = _forward(prob, x1), _forward(prob, x2)
    det = np.abs(lam) ** 2 + a * a
    u1 = (np.conj(lam) * r1 + a * r2) / det
    u2 = (lam * r2 - a * r1) / det
    o1, o2 = _inverse(prob, u1), _inverse(prob, u2)
    if real:
        o1, o2 = np.real(o1), np.real(o2)
    return np.concatenate([o1.ravel(), o2.ravel()])


def sigma_ms(prob):
    """sqrt(|lambda_k(S_n)|^2 + alpha^2): the time factor of P_MS (Eq. matrix_P_MS)."""
    return np.sqrt(np.abs(spc.lam_Sn(prob.n, prob.theta, prob.zeta)) ** 2 + prob.alpha ** 2)


def apply_pms_inv(prob, v, cycles=None):
    """P_MS^{-1} v: time transform, per frequency (sigma_k I + tau K)^{-1}, inverse transform
    (three steps in Sec. 3.5).  a = 1 and cycles None: exact DST solve; otherwise `cycles`
    multigrid V-cycles."""
    _no_neumann(prob)
    sig = sigma_ms(prob)
    out = []
    for x in _halves(prob, v):
        X = spc.time_forward(x, prob.zeta)
        if cycles is None:
            if prob.a_edges is not None:
                raise ValueError("exact P_MS solve needs a = 1; pass cycles for variable a")
            W = 1.0 / (sig[:, None] + prob.tau * _kappa2d(prob).reshape(1, -1))
            Z = spc.space_inverse(W * spc.space_forward(X, prob.N, prob.bc), prob.N, prob.bc)
        else:
            ax, ay = prob.edges()
            levels = mg.hierarchy(prob.N, ax, ay, prob.tau)
            R = X.reshape(prob.n, prob.N, prob.N)
            Z = mg.solve(levels, sig[:, None, None].astype(complex), R, cycles).reshape(prob.n, prob.m)
        out.append(np.real(spc.time_inverse(Z, prob.zeta)).ravel())
    return np.concatenate(out)


def lemma314(lam, alpha):
    """Lemma 3.14 applied to G = [[lam, -alpha], [alpha, conj(lam)]] (principal square root):
    returns (M, D1, D2) with G = W diag(D1, D2) W^{-1}, W = [[1, M], [M, 1]]."""
    lam = np.asarray(lam, dtype=complex)
    G1, G2, G3, G4 = lam, -alpha, alpha, np.conj(lam)
    root = np.sqrt((G4 - G1) ** 2 + 4.0 * G2 * G3 + 0j)
    M1 = 0.5 / G2 * (G4 - G1 + root)
    M2 = -0.5 / G3 * (G4 - G1 + root)
    D1 = G1 + G2 * M1
    D2 = G4 + G3 * M2
    return M1, M2, D1, D2


def apply_mg_ps_inv(prob, v, cycles=2, nu1=2, nu2=2, real=True):
    """P_S^{-1} v with the spatial solves done by multigrid (variable a(x), or Example 3's Neumann
    grid as the paper solves it), following the three steps after Lemma 3.14: v~ = V* v,
    w~ = blockdiag(D1 + tau K, D2 + tau K)^{-1} v~, w = V w~."""
    if prob.bc == "neumann":
        levels = mg.hierarchy_neumann(prob.N, prob.a0, prob.tau)
    else:
        ax, ay = prob.edges()
        levels = mg.hierarchy(prob.N, ax, ay, prob.tau)
    lam = spc.lam_Sn(prob.n, prob.theta, prob.zeta)
    M1, M2, D1, D2 = lemma314(lam, prob.alpha)
    x1, x2 = _halves(prob, v)
    V1 = spc.time_forward(x1, prob.zeta)
    V2 = spc.time_forward(x2, prob.zeta)
    det = 1.0 - M1 * M2
    T1 = (V1 - M2[:, None] * V2) / det[:, None]        # W^{-1} [V1; V2], W = [[1, M2], [M1, 1]]
    T2 = (V2 - M1[:, None] * V1) / det[:, None]
    shp = (prob.n, prob.N, prob.N)
    Z1 = mg.solve(levels, D1[:, None, None], T1.reshape(shp), cycles, nu1, nu2).reshape(prob.n, prob.m)
    Z2 = mg.solve(levels, D2[:, None, None], T2.reshape(shp), cycles, nu1, nu2).reshape(prob.n, prob.m)
    U1 = Z1 + M2[:, None] * Z2
    U2 = M1[:, None] * Z1 + Z2
    o1, o2 = spc.time_inverse(U1, prob.zeta), spc.time_inverse(U2, prob.zeta)
    if real:
        o1, o2 = np.real(o1), np.real(o2)
    return np.concatenate([o1.ravel(), o2.ravel()])


# ---------------------------------------------------------------------------------------
# Dense constructions (tiny sizes only)
# ---------------------------------------------------------------------------------------

def dense_K(prob):
    """The spatial operator of Eq. (matrix_A): K, or M^{-1/2} K M^{-1/2} with finite elements
    (the square root from a dense symmetric eigendecomposition of M)."""
    K = K_sparse(prob).toarray()
    if getattr(prob, "fem", False):
        Mi = _sqrtm_herm(np.linalg.inv(M_sparse(prob).toarray()))
        K = Mi @ K @ Mi
    return K


def dense_Sn(prob):
    S1 = spc.S1_dense(prob.n, prob.zeta)
    S2 = spc.S2_dense(prob.n, prob.theta, prob.zeta)
    return S1 @ np.linalg.inv(S2)


def dense_calS(prob):
    """calS = S_n (x) I_m + tau I_n (x) (-L_m)   (Eq. matrix_S)."""
    return np.kron(dense_Sn(prob), np.eye(prob.m)) + prob.tau * np.kron(np.eye(prob.n), dense_K(prob))


def dense_calS_second(prob):
    """Second diagonal block of P_S: calS^* = S_n^* (x) I + tau I (x) K^T; with the Neumann K the
    printed formula keeps K itself, S_n^* (x) I + tau I (x) K (equal for symmetric K)."""
    K = dense_K(prob)
    return (np.kron(dense_Sn(prob).conj().T, np.eye(prob.m))
            + prob.tau * np.kron(np.eye(prob.n), K if prob.bc == "neumann" else K.T))


def dense_T(prob):
    Bn = B1_dense(prob.n) @ np.linalg.inv(B2_dense(prob.n, prob.theta))
    return np.kron(Bn, np.eye(prob.m)) + prob.tau * np.kron(np.eye(prob.n), dense_K(prob))


def dense_T_second(prob):
    """The adjoint-row block T^T = B_n^T (x) I + tau I (x) K^T; the Neumann K enters as printed,
    B_n^T (x) I + tau I (x) K (equal for symmetric K)."""
    Bn = B1_dense(prob.n) @ np.linalg.inv(B2_dense(prob.n, prob.theta))
    K = dense_K(prob)
    return np.kron(Bn.T, np.eye(prob.m)) + prob.tau * np.kron(np.eye(prob.n), K if prob.bc == "neumann" else K.T)


def dense_A(prob):
    T = dense_T(prob); a = prob.alpha; I = np.eye(T.shape[0])
    return np.block([[a * I, dense_T_second(prob)], [T, -a * I]])


def dense_A_hat(prob):
    T = dense_T(prob); a = prob.alpha; I = np.eye(T.shape[0])
    return np.block([[T, -a * I], [a * I, dense_T_second(prob)]])


def dense_P_S(prob):
    S = dense_calS(prob); a = prob.alpha; I = np.eye(S.shape[0])
    return np.block([[S, -a * I], [a * I, dense_calS_second(prob)]])


def _sqrtm_herm(H):
    w, U = np.linalg.eigh(H)
    return (U * np.sqrt(np.maximum(w, 0.0))) @ U.conj().T


def dense_abs_P_S(prob):
    """|P_S| = blockdiag(sqrt(S*S + alpha^2 I), sqrt(SS* + alpha^2 I))   (Eq. matrix_P)."""
    S = dense_calS(prob); a2 = prob.alpha ** 2; I = np.eye(S.shape[0])
    top = _sqrtm_herm(S.conj().T @ S + a2 * I)
    bot = _sqrtm_herm(S @ S.conj().T + a2 * I)
    Z = np.zeros_like(top)
    return np.block([[top, Z], [Z, bot]])


def dense_P_MS(prob):
    """P_MS of Eq. (matrix_P_MS)."""
    Sn = dense_Sn(prob); a2 = prob.alpha ** 2; In = np.eye(prob.n); Im = np.eye(prob.m)
    K = dense_K(prob)
    top = np.kron(_sqrtm_herm(Sn.conj().T @ Sn + a2 * In), Im) + prob.tau * np.kron(In, K)
    bot = np.kron(_sqrtm_herm(Sn @ Sn.conj().T + a2 * In), Im) + prob.tau * np.kron(In, K)
    Z = np.zeros_like(top)
    return np.block([[top, Z], [Z, bot]])


def dense_abs_A(prob):
    """|A| = sqrt(A^2)   (Eq. abs_ideal_matrix_H)."""
    A = dense_A(prob)
    return _sqrtm_herm(A @ A)

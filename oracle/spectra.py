"""Spectral data of the preconditioners (paper Sec. 1 and Sec. 3.5).

omega-circulant factors (Eq. matrix_strang_1): S^(1) = B^(1) with top-right entry -omega,
S^(2) = B^(2) with top-right entry omega (1 - theta), omega = exp(i zeta).

Factorisation used here (reading of Eq. decompositiob_S12): with D = diag(exp(i zeta t / n)),
t = 0..n-1, and F the forward DFT matrix (entries exp(-2 pi i k t / n)),
    C = D^{-1} F^{-1} diag(lambda) F D,   lambda_k = sum_d c_d exp(i d phi_k),
    phi_k = (zeta - 2 pi k) / n,
for an omega-circulant C with first column c.  This is the paper's set of eigenvalues
f((zeta + 2 pi k)/n) re-indexed k -> -k (mod n).

Spatial factor (Sec. 3.5): for a = 1, K = -L_m = (S_N (x) S_N) diag(kappa_p + kappa_q) (S_N (x) S_N),
S_N[i, p] = sqrt(2/(N+1)) sin(i p pi/(N+1)) (orthogonal, symmetric, involutory),
kappa_p = (4/h^2) sin^2(p pi h / 2).  A constant coefficient a0 scales kappa.

Neumann (Example 3, the "minimal modification" of Sec. 1 with a cosine transform in place of the
sine transform): the mirrored second difference on N nodes (h = 1/(N-1)) is K1 = W^{-1} K1s with
W = diag(1/2, 1, .., 1, 1/2) and K1s symmetric, so W^{1/2} K1 W^{-1/2} is symmetric and is
diagonalised by the orthonormal DCT-I matrix C (C = C^T = C^{-1}):
    K1 = V diag(kappa) V^{-1},  V = W^{-1/2} C,  V^{-1} = C W^{1/2},
    kappa_k = (4/h^2) sin^2(k pi / (2 (N-1))), k = 0..N-1.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft


def omega(zeta):
    return complex(math.cos(zeta), math.sin(zeta))


def S1_dense(n, zeta):
    S = (np.eye(n) - np.eye(n, k=-1)).astype(complex)
    S[0, n - 1] = -omega(zeta)
    return S


def S2_dense(n, theta, zeta):
    S = (theta * np.eye(n) + (1.0 - theta) * np.eye(n, k=-1)).astype(complex)
    S[0, n - 1] = omega(zeta) * (1.0 - theta)
    return S


def phi(n, zeta):
    return (zeta - 2.0 * math.pi * np.arange(n)) / n


def lam_S1(n, zeta):
    """lambda_k(S^(1)) = f1(phi_k) = 1 - exp(i phi_k)   (Eq. functionB1)."""
    return 1.0 - np.exp(1j * phi(n, zeta))


def lam_S2(n, theta, zeta, remedy=True):
    """lambda_k(S^(2)) = f2(phi_k) = theta + (1 - theta) exp(i phi_k)   (Eq. functionB2).
    A zero eigenvalue (theta = 1/2 with exp(i phi_k) = -1) is replaced by 1, the value of f2 at
    phi = 0 (Remark 1 leaves the nonzero replacement unspecified)."""
    lam = theta + (1.0 - theta) * np.exp(1j * phi(n, zeta))
    if remedy:
        lam = np.where(np.abs(lam) < 1e-14, 1.0 + 0j, lam)
    return lam


def lam_Sn(n, theta, zeta):
    """lambda_k(S_n) = lambda_k(S^(1)) / lambda_k(S^(2))   (proof of Lemma 3.4)."""
    return lam_S1(n, zeta) / lam_S2(n, theta, zeta)


def D_omega(n, zeta):
    return np.exp(1j * zeta * np.arange(n) / n)


def kappa(N):
    """Eigenvalues of the 1D Dirichlet second-difference matrix, p = 1..N."""
    h = 1.0 / (N + 1)
    p = np.arange(1, N + 1)
    return (4.0 / h ** 2) * np.sin(p * math.pi * h / 2.0) ** 2


def kappa_neumann(N):
    """Eigenvalues of the 1D mirrored (Neumann) second-difference matrix, k = 0..N-1, h = 1/(N-1)."""
    h = 1.0 / (N - 1)
    k = np.arange(N)
    return (4.0 / h ** 2) * np.sin(k * math.pi / (2.0 * (N - 1))) ** 2


def mass_eigenvalues(N):
    """Eigenvalues of the 1D linear-element mass matrix (h/6) tridiag(1, 4, 1), p = 1..N (the
    same sine eigenvectors as the second difference): (h/6)(4 + 2 cos(p pi h))."""
    h = 1.0 / (N + 1)
    p = np.arange(1, N + 1)
    return (h / 6.0) * (4.0 + 2.0 * np.cos(p * math.pi * h))


def stiffness_eigenvalues(N):
    """Eigenvalues of the 1D linear-element stiffness matrix (1/h) tridiag(-1, 2, -1), p = 1..N."""
    h = 1.0 / (N + 1)
    p = np.arange(1, N + 1)
    return (2.0 - 2.0 * np.cos(p * math.pi * h)) / h


def mass_eigenvalues_2d(N):
    """Eigenvalues of M1 (x) M1 laid out [q, p]."""
    mu = mass_eigenvalues(N)
    return mu[None, :] * mu[:, None]


def kappa_fem(N):
    """Eigenvalues of M1^{-1/2} K1 M1^{-1/2} (the 1D factor of K~ = M^{-1/2} K M^{-1/2}): since
    M1 and K1 share their eigenvectors, kappa1_p / mu_p."""
    return stiffness_eigenvalues(N) / mass_eigenvalues(N)


def kappa2d(N, bc="dirichlet", fem=False):
    """kappa_p + kappa_q laid out [q, p] (x1-mode p fastest), matching the spatial vector layout.
    With fem: the eigenvalues of K~ = M^{-1/2} K M^{-1/2} / a0 (K = a0 (K1 (x) M1 + M1 (x) K1) gives
    K~ = a0 (K1^ (x) I + I (x) K1^) with K1^ = M1^{-1/2} K1 M1^{-1/2})."""
    k = kappa_neumann(N) if bc == "neumann" else (kappa_fem(N) if fem else kappa(N))
    return k[None, :] + k[:, None]


def dst_matrix(N):
    i = np.arange(1, N + 1)
    return math.sqrt(2.0 / (N + 1)) * np.sin(np.outer(i, i) * math.pi / (N + 1))


# ---- fast transforms (library FFT / DST as single steps) --------------------------------

def time_forward(v, zeta):
    """(F D (x) I) v along axis 0 of v with shape (n, ...)."""
    n = v.shape[0]
    d = D_omega(n, zeta).reshape((n,) + (1,) * (v.ndim - 1))
    return np.fft.fft(d * v, axis=0)


def time_inverse(w, zeta):
    """(D^{-1} F^{-1} (x) I) w."""
    n = w.shape[0]
    d = D_omega(n, zeta).reshape((n,) + (1,) * (w.ndim - 1))
    return np.fft.ifft(w, axis=0) / d


def dst2(u, N):
    """(S_N (x) S_N) u for u of shape (..., N*N) (applied on the [j, i] grid)."""
    U = u.reshape(u.shape[:-1] + (N, N))
    U = scipy.fft.dst(U, type=1, axis=-1, norm="ortho")
    U = scipy.fft.dst(U, type=1, axis=-2, norm="ortho")
    return U.reshape(u.shape)


def _wsqrt(N):
    w = np.ones(N)
    w[0] = w[-1] = math.sqrt(0.5)
    return w


def dct1_forward2(u, N):
    """(V^{-1} (x) V^{-1}) u = (C (x) C)(W^{1/2} (x) W^{1/2}) u for u of shape (..., N*N)."""
    w = _wsqrt(N)
    U = u.reshape(u.shape[:-1] + (N, N)) * w[:, None] * w[None, :]
    U = scipy.fft.dct(U, type=1, axis=-1, norm="ortho")
    U = scipy.fft.dct(U, type=1, axis=-2, norm="ortho")
    return U.reshape(u.shape)


def dct1_inverse2(v, N):
    """(V (x) V) v = (W^{-1/2} (x) W^{-1/2})(C (x) C) v."""
    w = _wsqrt(N)
    V = v.reshape(v.shape[:-1] + (N, N))
    V = scipy.fft.dct(V, type=1, axis=-1, norm="ortho")
    V = scipy.fft.dct(V, type=1, axis=-2, norm="ortho")
    return (V / w[:, None] / w[None, :]).reshape(v.shape)


def space_forward(u, N, bc="dirichlet"):
    """Spatial eigenbasis coordinates: S_N (x) S_N (Dirichlet) or V^{-1} (x) V^{-1} (Neumann)."""
    return dct1_forward2(u, N) if bc == "neumann" else dst2(u, N)


def space_inverse(v, N, bc="dirichlet"):
    return dct1_inverse2(v, N) if bc == "neumann" else dst2(v, N)

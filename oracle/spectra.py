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
kappa_p = (4/h^2) sin^2(p pi h / 2).
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


def kappa2d(N):
    """kappa_p + kappa_q laid out [q, p] (x1-mode p fastest), matching the spatial vector layout."""
    k = kappa(N)
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

"""All-at-once matrix-vector products (paper Sec. 1 and Sec. 3.5):
  A     = [[alpha I, T^T], [T, -alpha I]]      (Eq. matrix_A, MINRES)
  A_hat = [[T, -alpha I], [alpha I, T^T]]      (Eq. matrix_A_hat, GMRES)
  T     = B_n (x) I_m + tau I_n (x) M^{-1/2} K M^{-1/2}   (Eq. matrix_T; K itself when M = I)
written from the definitions; B_n is applied as B^(1) followed by (B^(2))^{-1}.
"""
from __future__ import annotations

import numpy as np

from .discretisation import apply_Bn, apply_K_tilde


def apply_T(prob, x, transpose=False):
    """T x (or T^T x) for x of shape (n, m)."""
    return apply_Bn(prob.theta, x, transpose) + prob.tau * apply_K_tilde(prob, x)


def matvec_A(prob, x):
    """A x for x of length 2mn: [alpha x1 + T^T x2 ; T x1 - alpha x2]."""
    mn = prob.m * prob.n
    x1 = x[:mn].reshape(prob.n, prob.m); x2 = x[mn:].reshape(prob.n, prob.m)
    a = prob.alpha
    top = a * x1 + apply_T(prob, x2, transpose=True)
    bot = apply_T(prob, x1) - a * x2
    return np.concatenate([top.ravel(), bot.ravel()])


def matvec_A_hat(prob, x):
    """A_hat x: [T x1 - alpha x2 ; alpha x1 + T^T x2]."""
    mn = prob.m * prob.n
    x1 = x[:mn].reshape(prob.n, prob.m); x2 = x[mn:].reshape(prob.n, prob.m)
    a = prob.alpha
    top = apply_T(prob, x1) - a * x2
    bot = a * x1 + apply_T(prob, x2, transpose=True)
    return np.concatenate([top.ravel(), bot.ravel()])

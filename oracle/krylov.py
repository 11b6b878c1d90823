"""Krylov solvers used in Sec. 4 (zero initial guess, relative-residual tolerance):

  minres : preconditioned MINRES (Paige & Saunders, 1975) -- Lanczos three-term recurrence in the
           preconditioner's inner product, Givens QR of the tridiagonal matrix, three-term
           direction update.  The preconditioner must be symmetric positive definite.
  fgmres : right-preconditioned restarted GMRES in the flexible form (Saad, 1993): the
           preconditioned basis Z is stored, Arnoldi uses classical Gram-Schmidt applied twice,
           Givens rotations on the Hessenberg matrix.  With a fixed preconditioner this is
           right-preconditioned GMRES(m).

Stopping rule (reading of "reduction in relative residual norms", Sec. 4): a solve succeeds when
the true relative residual ||b - A x||_2 / ||b||_2 <= tol, evaluated in float64; the
recurrence's residual estimate only decides when to evaluate it.

stall (off by default): for solves asked to go below the attainable accuracy of float64, stop
once the true residual no longer follows -- MINRES when the recurrence's estimate has dropped
below stall x the last true residual evaluated, FGMRES when a restart cycle reduced the true
residual by less than a factor 2.  The result is then returned unconverged with its true relres.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Info:
    iterations: int = 0
    relres: float = float("nan")
    converged: bool = False
    history: list = None
    breakdown: bool = False


def minres(A, b, M=None, tol=1e-8, maxit=500, fixed_iterations=None, stall=None):
    """Solve A x = b (A symmetric) with SPD preconditioner M (callable returning M^{-1} r).
    fixed_iterations: run exactly that many iterations (for same-algorithm comparisons)."""
    if M is None:
        M = lambda r: r.copy()
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    info = Info(history=[])
    if bnorm == 0.0:
        info.relres, info.converged = 0.0, True
        return x, info
    r1 = b.copy()
    y = M(r1)
    beta1 = float(r1 @ y)
    if beta1 <= 0.0:
        info.breakdown = True
        return x, info
    beta1 = math.sqrt(beta1)
    oldb, beta, dbar, epsln, phibar = 0.0, beta1, 0.0, 0.0, beta1
    cs, sn = -1.0, 0.0
    w = np.zeros_like(b); w2 = np.zeros_like(b)
    r2 = r1.copy()
    limit = fixed_iterations if fixed_iterations is not None else maxit
    for itn in range(1, limit + 1):
        v = y / beta
        y = A(v)
        if itn >= 2:
            y = y - (beta / oldb) * r1
        alfa = float(v @ y)
        y = y - (alfa / beta) * r2
        r1, r2 = r2, y
        y = M(r2)
        oldb = beta
        bb = float(r2 @ y)
        if bb < 0.0:
            info.breakdown = True
            break
        beta = math.sqrt(bb)
        oldeps = epsln
        delta = cs * dbar + sn * alfa
        gbar = sn * dbar - cs * alfa
        epsln = sn * beta
        dbar = -cs * beta
        gamma = math.hypot(gbar, beta)
        if gamma == 0.0:
            info.breakdown = True
            break
        cs, sn = gbar / gamma, beta / gamma
        phi = cs * phibar
        phibar = sn * phibar
        w1, w2 = w2, w
        w = (v - oldeps * w1 - delta * w2) / gamma
        x = x + phi * w
        info.iterations = itn
        info.history.append(phibar / beta1)
        if fixed_iterations is None and phibar / beta1 <= tol:
            rel = float(np.linalg.norm(b - A(x))) / bnorm
            if rel <= tol:
                info.relres, info.converged = rel, True
                return x, info
            if stall is not None and phibar / beta1 <= stall * rel:
                info.relres = rel
                return x, info
        if beta == 0.0:
            break
    info.relres = float(np.linalg.norm(b - A(x))) / bnorm
    info.converged = info.relres <= tol
    return x, info


def _givens(a, b):
    """(c, s) with [c s; -s c] [a; b] = [r; 0]; real arithmetic."""
    if b == 0.0:
        return 1.0, 0.0
    r = math.hypot(a, b)
    return a / r, b / r


def fgmres(A, b, M=None, tol=1e-8, restart=30, maxit=500, fixed_iterations=None, stall=None):
    """Right-preconditioned restarted (F)GMRES with CGS2 orthogonalisation."""
    if M is None:
        M = lambda r: r.copy()
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    info = Info(history=[])
    if bnorm == 0.0:
        info.relres, info.converged = 0.0, True
        return x, info
    total = 0
    limit = fixed_iterations if fixed_iterations is not None else maxit
    last = math.inf
    while total < limit:
        r = b - A(x)
        beta = float(np.linalg.norm(r))
        if fixed_iterations is None and beta / bnorm <= tol:
            info.relres, info.converged = beta / bnorm, True
            return x, info
        if stall is not None and total > 0 and beta > 0.5 * last:
            info.relres = beta / bnorm
            return x, info
        last = beta
        mres = min(restart, limit - total)
        V = np.zeros((mres + 1, b.size)); Z = np.zeros((mres, b.size))
        H = np.zeros((mres + 1, mres)); g = np.zeros(mres + 1)
        cs = np.zeros(mres); sn = np.zeros(mres)
        V[0] = r / beta; g[0] = beta
        k = 0
        for j in range(mres):
            Z[j] = M(V[j])
            wv = A(Z[j])
            h = V[: j + 1] @ wv
            wv = wv - V[: j + 1].T @ h
            h2 = V[: j + 1] @ wv
            wv = wv - V[: j + 1].T @ h2
            h = h + h2
            hn = float(np.linalg.norm(wv))
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            k = j + 1
            info.history.append(abs(g[j + 1]) / bnorm)
            if hn == 0.0:
                break
            V[j + 1] = wv / hn
            if fixed_iterations is None and abs(g[j + 1]) / bnorm <= tol:
                break
        yk = np.zeros(k)
        for i in range(k - 1, -1, -1):
            yk[i] = (g[i] - H[i, i + 1: k] @ yk[i + 1:]) / H[i, i]
        x = x + Z[:k].T @ yk
        info.iterations = total
        if fixed_iterations is None and abs(g[k]) / bnorm <= tol:
            rel = float(np.linalg.norm(b - A(x))) / bnorm
            if rel <= tol:
                info.relres, info.converged = rel, True
                return x, info
    info.relres = float(np.linalg.norm(b - A(x))) / bnorm
    info.converged = info.relres <= tol
    return x, info

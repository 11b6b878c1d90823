"""Geometric multigrid V-cycle for the per-frequency shifted spatial systems (mu I + tau K) z = r
named in Sec. 3.5 (Step 2 of the P_S^{-1} and P_MS^{-1} applications) and Sec. 4.

The paper does not specify its multigrid.  Reading used here (parity against the paper unpinned;
pinned only by convergence to the exact shifted solve):
  * vertex-centred coarsening N -> (N-1)/2 (N = 2^k - 1 down to N = 1), spacing doubles;
  * coarse edge coefficient = mean of the two collinear fine edge coefficients it spans;
  * full-weighting restriction ([1 2 1; 2 4 2; 1 2 1]/16), bilinear prolongation;
  * damped Jacobi smoother, weight 4/5, nu1 pre- and nu2 post-sweeps;
  * exact solve on the single-unknown coarsest grid;
  * zero initial guess, a fixed number of cycles, so the solver is a fixed linear operator.
The shift mu is complex in general; K is real.

Neumann grids (Example 3, solved with "GMRES-P_S + MG" in Sec. 4): N = 2^k + 1 nodes per side
including the boundary, h = 1/(N-1), constant coefficient a0 and the mirrored second difference of
discretisation.apply_K.  Reading (the paper gives no details): coarse nodes are the even fine nodes
(boundary included), N -> (N+1)/2 down to N = 3; full weighting with the same mirrored ghost values
as the stencil; bilinear prolongation (every odd fine node lies between two coarse nodes); the same
damped Jacobi (the diagonal is 4 a0/h^2 at every node); an exact dense solve on the 3 x 3 grid.
"""
from __future__ import annotations

import numpy as np

JACOBI_WEIGHT = 0.8


class Level:
    def __init__(self, N, ax, ay, tau):
        self.N, self.ax, self.ay, self.tau = N, ax, ay, tau
        self.h = 1.0 / (N + 1)
        self.diagK = (ax[:, :-1] + ax[:, 1:] + ay[:-1, :] + ay[1:, :]) / self.h ** 2

    def K(self, U):
        """K applied to U[..., j, i] with zero Dirichlet boundary."""
        N = self.N
        P = np.zeros(U.shape[:-2] + (N + 2, N + 2), dtype=U.dtype)
        P[..., 1:-1, 1:-1] = U
        c = P[..., 1:-1, 1:-1]
        return (self.ax[:, :-1] * (c - P[..., 1:-1, :-2]) + self.ax[:, 1:] * (c - P[..., 1:-1, 2:])
                + self.ay[:-1, :] * (c - P[..., :-2, 1:-1]) + self.ay[1:, :] * (c - P[..., 2:, 1:-1])) / self.h ** 2


class NeumannLevel:
    """One level of a Neumann grid: N nodes per side with the boundary, mirrored stencil."""

    def __init__(self, N, a0, tau):
        self.N, self.a0, self.tau = N, a0, tau
        self.h = 1.0 / (N - 1)
        self.diagK = np.full((N, N), 4.0 * a0 / self.h ** 2)

    def K(self, U):
        P = np.pad(U, [(0, 0)] * (U.ndim - 2) + [(1, 1), (1, 1)], mode="reflect")
        c = P[..., 1:-1, 1:-1]
        nb = P[..., 1:-1, :-2] + P[..., 1:-1, 2:] + P[..., :-2, 1:-1] + P[..., 2:, 1:-1]
        return self.a0 * (4.0 * c - nb) / self.h ** 2


def hierarchy_neumann(N, a0, tau):
    """Levels from fine (N nodes) to the 3 x 3 grid; requires N = 2^k + 1, k >= 1."""
    if N < 3 or (N - 1) & (N - 2):
        raise ValueError("the Neumann multigrid needs N = 2^k + 1 nodes per side")
    levels = [NeumannLevel(N, a0, tau)]
    while levels[-1].N > 3:
        levels.append(NeumannLevel((levels[-1].N + 1) // 2, a0, tau))
    return levels


def restrict_neumann(R):
    """Full weighting onto the even fine nodes, with mirrored ghost values at the boundary."""
    P = np.pad(R, [(0, 0)] * (R.ndim - 2) + [(1, 1), (1, 1)], mode="reflect")
    c = slice(1, -1, 2)        # padded index of even fine nodes
    cm = slice(0, -2, 2)
    cp = slice(2, None, 2)
    return (4 * P[..., c, c] + 2 * (P[..., c, cm] + P[..., c, cp] + P[..., cm, c] + P[..., cp, c])
            + P[..., cm, cm] + P[..., cm, cp] + P[..., cp, cm] + P[..., cp, cp]) / 16.0


def prolong_neumann(E, Nf):
    """Bilinear interpolation from the coarse nodes (even fine nodes) to the fine Neumann grid."""
    out = np.zeros(E.shape[:-2] + (Nf, Nf), dtype=E.dtype)
    out[..., 0::2, 0::2] = E
    out[..., 0::2, 1::2] = 0.5 * (E[..., :, :-1] + E[..., :, 1:])
    out[..., 1::2, 0::2] = 0.5 * (E[..., :-1, :] + E[..., 1:, :])
    out[..., 1::2, 1::2] = 0.25 * (E[..., :-1, :-1] + E[..., :-1, 1:] + E[..., 1:, :-1] + E[..., 1:, 1:])
    return out


def _coarsest_solve_neumann(L, mu, R):
    """Exact solve of (mu I + tau K) Z = R on the 3 x 3 grid (dense, per system)."""
    N = L.N
    eye = np.eye(N * N).reshape(N * N, N, N)
    Kd = np.stack([L.K(e).ravel() for e in eye], axis=1)            # K as a dense 9 x 9 matrix
    mu_b = np.broadcast_to(np.asarray(mu), R.shape[:-2] + (1, 1))[..., 0, 0]
    A = mu_b[..., None, None] * np.eye(N * N) + L.tau * Kd
    Z = np.linalg.solve(A, R.reshape(R.shape[:-2] + (N * N,))[..., None])[..., 0]
    return Z.reshape(R.shape)


def hierarchy(N, ax, ay, tau):
    """Levels from fine (N) to the 1 x 1 grid; requires N = 2^k - 1."""
    if N < 1 or (N + 1) & N:
        raise ValueError("multigrid needs N = 2^k - 1")
    levels = [Level(N, ax, ay, tau)]
    while levels[-1].N > 1:
        f = levels[-1]
        Nc = (f.N - 1) // 2
        # coarse x1-edge e (between coarse nodes e, e+1) on coarse row J spans fine edges 2e, 2e+1 on fine row 2J+1
        axc = 0.5 * (f.ax[1::2, 0::2] + f.ax[1::2, 1::2])
        ayc = 0.5 * (f.ay[0::2, 1::2] + f.ay[1::2, 1::2])
        levels.append(Level(Nc, axc, ayc, tau))
    return levels


def restrict(R):
    """Full weighting from a fine (Nf x Nf) grid to the coarse ((Nf-1)/2)^2 grid."""
    Nf = R.shape[-1]
    P = np.zeros(R.shape[:-2] + (Nf + 2, Nf + 2), dtype=R.dtype)
    P[..., 1:-1, 1:-1] = R
    c = slice(2, Nf, 2)          # padded index of fine node 2J (1-based), J = 1..Nc
    cm = slice(1, Nf - 1, 2)
    cp = slice(3, Nf + 1, 2)
    return (4 * P[..., c, c] + 2 * (P[..., c, cm] + P[..., c, cp] + P[..., cm, c] + P[..., cp, c])
            + P[..., cm, cm] + P[..., cm, cp] + P[..., cp, cm] + P[..., cp, cp]) / 16.0


def prolong(E, Nf):
    """Bilinear interpolation from the coarse grid to the fine (Nf x Nf) grid."""
    Nc = E.shape[-1]
    P = np.zeros(E.shape[:-2] + (Nc + 2, Nc + 2), dtype=E.dtype)
    P[..., 1:-1, 1:-1] = E
    out = np.zeros(E.shape[:-2] + (Nf, Nf), dtype=E.dtype)
    # fine 1-based index 2J sits on coarse node J; odd fine indices lie between coarse nodes
    out[..., 1::2, 1::2] = E
    out[..., 1::2, 0::2] = 0.5 * (P[..., 1:-1, :-1] + P[..., 1:-1, 1:])
    out[..., 0::2, 1::2] = 0.5 * (P[..., :-1, 1:-1] + P[..., 1:, 1:-1])
    out[..., 0::2, 0::2] = 0.25 * (P[..., :-1, :-1] + P[..., :-1, 1:] + P[..., 1:, :-1] + P[..., 1:, 1:])
    return out


def smooth(L, mu, Z, R, sweeps):
    """`sweeps` damped Jacobi sweeps on (mu I + tau K) Z = R at level L."""
    diag = mu + L.tau * L.diagK
    for _ in range(sweeps):
        Z = Z + JACOBI_WEIGHT * (R - (mu * Z + L.tau * L.K(Z))) / diag
    return Z


def vcycle(levels, mu, R, nu1=2, nu2=2, lev=0):
    """One V-cycle with zero initial guess for (mu I + tau K) Z = R; mu broadcasts against
    R[..., j, i] (shape (...,) -> use mu[..., None, None])."""
    L = levels[lev]
    neu = isinstance(L, NeumannLevel)
    if lev == len(levels) - 1:
        return _coarsest_solve_neumann(L, mu, R) if neu else R / (mu + L.tau * L.diagK)
    Z = smooth(L, mu, np.zeros_like(R), R, nu1)
    res = R - (mu * Z + L.tau * L.K(Z))
    Ec = vcycle(levels, mu, restrict_neumann(res) if neu else restrict(res), nu1, nu2, lev + 1)
    Z = Z + (prolong_neumann(Ec, L.N) if neu else prolong(Ec, L.N))
    return smooth(L, mu, Z, R, nu2)


def solve(levels, mu, R, cycles=2, nu1=2, nu2=2):
    """`cycles` V-cycles from a zero initial guess (each further cycle corrects the residual)."""
    L = levels[0]
    Z = np.zeros_like(R)
    for _ in range(cycles):
        res = R - (mu * Z + L.tau * L.K(Z))
        Z = Z + vcycle(levels, mu, res, nu1, nu2)
    return Z

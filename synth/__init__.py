"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle's tests.

This module holds input *data* only: grids, random target trajectories g(x, t), analytic
source samples f(x, t), coefficient samples a(x) at cell-edge midpoints, parameter draws and
arrival traces.  It contains none of the solver's arithmetic (no operators, no transforms,
no right-hand-side assembly), so both sides can draw identical inputs from it without
sharing any of the method.

Shapes follow the test problems of the paper's numerical section (unit square, T = 1,
smooth sine modes, gamma between 1e-10 and 1e-1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Instance:
    """One control problem: grid, horizon, scheme and data samples (all FP64, host)."""

    N: int                    # interior points per side, m = N*N
    n: int                    # time steps, tau = T/n
    theta: float              # 1 = backward Euler, 0.5 = Crank-Nicolson
    gamma: float              # regularisation parameter
    T: float = 1.0
    zeta: float = math.pi     # omega = exp(i*zeta); pi gives the skew-circulant choice
    a_edges: np.ndarray | None = None   # None => a(x) = 1, else 2*N*(N+1) edge values
    g: np.ndarray | None = None         # (n+1, m) samples of g at t_k = k*tau
    f: np.ndarray | None = None         # (n+1, m) samples of f at t_k
    y0: np.ndarray | None = None        # (m,) initial state, None => 0
    tag: str = ""

    @property
    def m(self) -> int:
        return self.N * self.N

    @property
    def unknowns(self) -> int:
        return 2 * self.m * self.n


def grid(N: int) -> tuple[np.ndarray, np.ndarray]:
    """Interior node coordinates x1[j, i], x2[j, i] (i fastest), h = 1/(N+1)."""
    h = 1.0 / (N + 1)
    x = h * np.arange(1, N + 1)
    x2, x1 = np.meshgrid(x, x, indexing="ij")
    return x1, x2


def times(n: int, T: float = 1.0) -> np.ndarray:
    return (T / n) * np.arange(n + 1)


def random_target(N: int, n: int, seed: int, T: float = 1.0, modes: int = 8, kmax: int = 4) -> np.ndarray:
    """g(x, t) = e^{-t} sum_k c_k sin(pi i_k x1) sin(pi j_k x2), i_k, j_k ~ U{1..kmax},
    c_k ~ N(0,1)/(i_k^2 + j_k^2); returns (n+1, N*N) samples at t_k = k*T/n."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ik = rng.integers(1, kmax + 1, size=modes)
    jk = rng.integers(1, kmax + 1, size=modes)
    ck = rng.standard_normal(modes) / (ik.astype(float) ** 2 + jk.astype(float) ** 2)
    x1, x2 = grid(N)
    space = np.zeros_like(x1)
    for c, i, j in zip(ck, ik, jk):
        space += c * np.sin(math.pi * i * x1) * np.sin(math.pi * j * x2)
    t = times(n, T)
    return np.exp(-t)[:, None] * space.reshape(1, -1)


def manufactured_source(N: int, n: int, T: float = 1.0) -> np.ndarray:
    """Analytic source samples f = (1 + 2 pi^2 t) sin(pi x1) sin(pi x2): the state equation's
    forcing for y = t sin sin when the adjoint coupling is ignored.  Used as a smooth,
    paper-shaped source for the large synthetic workloads; (n+1, N*N)."""
    x1, x2 = grid(N)
    s = (np.sin(math.pi * x1) * np.sin(math.pi * x2)).reshape(1, -1)
    t = times(n, T)[:, None]
    return (1.0 + 2.0 * math.pi ** 2 * t) * s


def example1_data(N: int, n: int, T: float = 1.0):
    """Example 1 of the paper's numerical section (a = 1): f = (2 pi^2 - 1) e^{-t} sin sin,
    g = e^{-t} sin sin, exact y = e^{-t} sin sin, p = 0.  Returns (g, f, y_exact, p_exact),
    each (n+1, N*N)."""
    x1, x2 = grid(N)
    s = (np.sin(math.pi * x1) * np.sin(math.pi * x2)).reshape(1, -1)
    e = np.exp(-times(n, T))[:, None]
    y = e * s
    return y.copy(), (2.0 * math.pi ** 2 - 1.0) * y, y, np.zeros_like(y)


EXAMPLE2_EPS = 1e-5


def example2_coefficient(x1, x2):
    """a(x1, x2) = 1e-5 sin(pi x1 x2) of Example 2."""
    return EXAMPLE2_EPS * np.sin(math.pi * x1 * x2)


def example2_data(N: int, n: int, gamma: float, T: float = 1.0):
    """Example 2 of the paper's numerical section (variable a = 1e-5 sin(pi x1 x2)), with the exact
    solution y = e^{-t} x1(1-x1) x2(1-x2), p = gamma sin(pi t) sin(pi x1) sin(pi x2).  The printed
    f and g are partly garbled; they are the data that make (y, p) solve the optimality system
    y_t - div(a grad y) = f + p/gamma, -p_t - div(a grad p) = g - y, i.e.
      f = y_t - div(a grad y) - p/gamma,   g = -p_t - div(a grad p) + y,
    with div(a grad u) = a_x1 u_x1 + a u_x1x1 + a_x2 u_x2 + a u_x2x2 written out below (they agree
    term by term with the legible parts of the printed formulas).  Returns (g, f, y_exact,
    p_exact, a_edges), the first four (n+1, N*N) at t_k = k tau on the interior nodes."""
    X, Y = grid(N)
    X, Y = X.reshape(1, -1), Y.reshape(1, -1)
    t = times(n, T)[:, None]
    eps, pi = EXAMPLE2_EPS, math.pi
    q = lambda s: s * (1.0 - s)
    sxy, cxy = np.sin(pi * X * Y), np.cos(pi * X * Y)
    a, ax, ay = eps * sxy, eps * pi * Y * cxy, eps * pi * X * cxy
    Q = q(X) * q(Y)
    # y = e^{-t} Q: y_x1 = e^{-t} (1 - 2 x1) q(x2), y_x1x1 = -2 e^{-t} q(x2) (and symmetrically)
    div_a_grad_Q = ax * (1 - 2 * X) * q(Y) + a * (-2.0) * q(Y) + ay * q(X) * (1 - 2 * Y) + a * (-2.0) * q(X)
    S = np.sin(pi * X) * np.sin(pi * Y)
    # p = gamma sin(pi t) S: S_x1 = pi cos(pi x1) sin(pi x2), S_x1x1 = -pi^2 S (and symmetrically)
    div_a_grad_S = (ax * pi * np.cos(pi * X) * np.sin(pi * Y) + ay * pi * np.sin(pi * X) * np.cos(pi * Y)
                    - 2.0 * pi ** 2 * a * S)
    et = np.exp(-t)
    y = et * Q
    p = gamma * np.sin(pi * t) * S
    f = -et * Q - et * div_a_grad_Q - np.sin(pi * t) * S
    g = -gamma * pi * np.cos(pi * t) * S - gamma * np.sin(pi * t) * div_a_grad_S + et * Q
    return g, f, y, p, variable_coefficient_edges(N, example2_coefficient)


def neumann_grid(N: int) -> tuple[np.ndarray, np.ndarray]:
    """Node coordinates x1[j, i], x2[j, i] (i fastest) of the Neumann grid: N nodes per side
    including the boundary, x = i h, h = 1/(N-1)."""
    x = np.arange(N) / (N - 1)
    x2, x1 = np.meshgrid(x, x, indexing="ij")
    return x1, x2


def example3_data(N: int, n: int, a0: float = 1e-3, T: float = 1.0):
    """Example 3 of the paper's numerical section (homogeneous Neumann, constant a = a0):
    f = (8 pi^2 a0 - 1) e^{-t} cos(2 pi x1) cos(2 pi x2), g = e^{-t} cos cos, exact y = g, p = 0.
    Returns (g, f, y_exact, p_exact), each (n+1, N*N), on neumann_grid(N)."""
    x1, x2 = neumann_grid(N)
    s = (np.cos(2.0 * math.pi * x1) * np.cos(2.0 * math.pi * x2)).reshape(1, -1)
    y = np.exp(-times(n, T))[:, None] * s
    return y.copy(), (8.0 * math.pi ** 2 * a0 - 1.0) * y, y, np.zeros_like(y)


def variable_coefficient_edges(N: int, fn=None) -> np.ndarray:
    """a(x) at cell-edge midpoints, flattened as [ax (N rows x (N+1)), ay ((N+1) rows x N)].

    ax[j, e] is the x1-edge between nodes e and e+1 of row j+1 (x1 = (e + 1/2) h),
    ay[e, i] is the x2-edge between nodes e and e+1 of column i+1 (x2 = (e + 1/2) h).
    Default a(x) = 1 + 0.5 sin(pi x1) sin(pi x2)."""
    if fn is None:
        fn = lambda x1, x2: 1.0 + 0.5 * np.sin(math.pi * x1) * np.sin(math.pi * x2)
    h = 1.0 / (N + 1)
    node = h * np.arange(1, N + 1)
    mid = h * (np.arange(0, N + 1) + 0.5)
    X1, X2 = np.meshgrid(mid, node, indexing="xy")      # ax: rows j (x2 = node), cols e (x1 = mid)
    ax = fn(X1, X2)
    Y1, Y2 = np.meshgrid(node, mid, indexing="xy")      # ay: rows e (x2 = mid), cols i (x1 = node)
    ay = fn(Y1, Y2)
    return np.concatenate([ax.ravel(), ay.ravel()])


def random_vector(size: int, seed: int, dtype=np.float64) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size).astype(dtype)


# --------------------------------------------------------------------------------------
# Workload configurations
# --------------------------------------------------------------------------------------

def config0() -> Instance:
    """N=15, n=16, backward Euler, gamma=1e-2, a=1, y0=0, g random (seed 0)."""
    N, n = 15, 16
    return Instance(N=N, n=n, theta=1.0, gamma=1e-2, g=random_target(N, n, seed=0),
                    f=manufactured_source(N, n), tag="cfg0")


def config1(gamma: float = 1e-2, N: int = 511, n: int = 512) -> Instance:
    """N=511, n=512, backward Euler, gamma in {1e-2, 1e-6}, a=1, g random (seed 1)."""
    return Instance(N=N, n=n, theta=1.0, gamma=gamma, g=random_target(N, n, seed=1),
                    f=manufactured_source(N, n), tag=f"cfg1-g{gamma:g}")


def config2(N: int = 255, n: int = 256) -> Instance:
    """Crank-Nicolson, gamma=1e-4, a = 1 + 0.5 sin sin, g random (seed 2)."""
    return Instance(N=N, n=n, theta=0.5, gamma=1e-4, a_edges=variable_coefficient_edges(N),
                    g=random_target(N, n, seed=2), f=manufactured_source(N, n), tag="cfg2")


def config3(count: int = 64, seed: int = 3, with_data: bool = True,
            Ns=(63, 127, 191, 255), ns=(32, 64, 128, 256)) -> list[Instance]:
    """Uneven batch: N ~ U(Ns), n ~ U(ns), theta ~ U{1, 1/2}, log10 gamma ~ U[-6, -1], a = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        N = int(rng.choice(Ns)); n = int(rng.choice(ns))
        theta = float(rng.choice([1.0, 0.5]))
        gamma = float(10.0 ** rng.uniform(-6.0, -1.0))
        gseed = int(rng.integers(0, 2 ** 31 - 1))
        inst = Instance(N=N, n=n, theta=theta, gamma=gamma, tag=f"cfg3-{k}")
        if with_data:
            inst.g = random_target(N, n, seed=gseed)
            inst.f = manufactured_source(N, n)
        out.append(inst)
    return out


@dataclass
class Request:
    rid: int
    arrival_s: float
    inst: Instance


def serving_trace(rate_hz: float = 200.0, duration_s: float = 60.0, seed: int = 4,
                  large_frac: float = 0.05, Ns=(63, 127, 191, 255), ns=(32, 64, 128, 256),
                  large=(511, 512), with_data: bool = False) -> list[Request]:
    """Poisson arrivals; 95% sized like the uneven batch, the rest large (N=511, n=512)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    rid = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        if rng.uniform() < large_frac:
            N, n = large
        else:
            N = int(rng.choice(Ns)); n = int(rng.choice(ns))
        theta = float(rng.choice([1.0, 0.5]))
        gamma = float(10.0 ** rng.uniform(-6.0, -1.0))
        gseed = int(rng.integers(0, 2 ** 31 - 1))
        inst = Instance(N=N, n=n, theta=theta, gamma=gamma, tag=f"req{rid}")
        inst._gseed = gseed  # data drawn lazily by the caller
        if with_data:
            inst.g = random_target(N, n, seed=gseed)
            inst.f = manufactured_source(N, n)
        out.append(Request(rid=rid, arrival_s=t, inst=inst))
        rid += 1
    return out

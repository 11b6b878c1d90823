"""Pins of the oracle's multigrid (oracle/multigrid.py) against the mathematics of its parts.

The paper names a multigrid V-cycle for the shifted spatial systems (mu I + tau K) z = r of
Sec. 3.5 and Sec. 4 but gives no details; the oracle's reading (vertex-centred coarsening, damped
Jacobi with weight 4/5, full weighting, bilinear prolongation, rediscretised coarse operator with
averaged edge coefficients) is pinned here part by part, each against a fact that a plausible
mistake in that part would break:
  * the Jacobi sweep multiplies every sine mode by 1 - w (mu + tau kappa_pq)/(mu + 4 tau a/h^2), and
    its local-Fourier-analysis smoothing factor over the high frequencies is 3/5 (w = 4/5);
  * bilinear prolongation reproduces bilinear functions, full weighting restricts them exactly;
  * for an affine a(x) the averaged coarse edge coefficients equal a at the coarse edge midpoints;
  * the two-grid error operator assembled from the oracle's parts, and the oracle's own two-level
    V-cycle (N = 3), equal their Fourier (4 x 4 harmonic block) analysis to rounding.
"""
import math

import numpy as np
import pytest

from oracle import multigrid as mg
from oracle import spectra as spc


def _const_level(N, a=1.0, tau=1.0):
    return mg.Level(N, a * np.ones((N, N + 1)), a * np.ones((N + 1, N)), tau)


def _sine_modes(N):
    """phi[p-1, q-1] = sin(p pi x1) sin(q pi x2) on the [j, i] grid (x1 = i h, x2 = j h)."""
    S = spc.dst_matrix(N)                     # S[i-1, p-1] = sqrt(2/(N+1)) sin(i p pi h)
    return np.einsum("ip,jq->pqji", S, S)     # (p, q, j, i)


@pytest.mark.parametrize("mu", [0.0, 3.7, 2.0 + 5.0j])
@pytest.mark.parametrize("a", [1.0, 0.3])
def test_jacobi_sweep_multiplies_sine_modes(mu, a):
    N, tau = 31, 0.05
    L = _const_level(N, a, tau)
    h = 1.0 / (N + 1)
    phi = _sine_modes(N).astype(complex)
    out = mg.smooth(L, mu, phi, np.zeros_like(phi), 1)
    kap = a * spc.kappa2d(N)                  # [q, p]
    lam = mu + tau * kap.T                    # [p, q]
    s = 1.0 - mg.JACOBI_WEIGHT * lam / (mu + 4.0 * tau * a / h ** 2)
    assert np.abs(out - s[:, :, None, None] * phi).max() < 1e-12


def test_jacobi_smoothing_factor_is_three_fifths():
    """Local Fourier analysis of damped Jacobi for the 5-point Laplacian: the multiplier is
    1 - w (1 - (cos t1 + cos t2)/2); over the high frequencies (max |t| >= pi/2) its largest modulus
    is max(|1 - 2w|, 1 - w/2) = 3/5 at w = 4/5 (the optimal weight).  On the grid, the largest high-
    frequency multiplier of the oracle's sweep approaches 3/5 from below as h -> 0."""
    for N in (31, 63, 127):
        L = _const_level(N)
        h = 1.0 / (N + 1)
        p = np.arange(1, N + 1)
        sp = np.sin(p * math.pi * h / 2) ** 2
        mult = 1.0 - mg.JACOBI_WEIGHT * (sp[:, None] + sp[None, :])    # the sweep's multipliers (test above)
        high = (p[:, None] >= (N + 1) // 2) | (p[None, :] >= (N + 1) // 2)
        mu_s = np.abs(mult[high]).max()
        assert 0.6 - 4 * h ** 2 * 10 <= mu_s <= 0.6 + 1e-12, (N, mu_s)
        # the sweep itself on the worst high-frequency mode
        phi = _sine_modes(N)
        k = np.unravel_index(np.argmax(np.where(high, np.abs(mult), 0)), mult.shape)
        z = mg.smooth(L, 0.0, phi[k], np.zeros_like(phi[k]), 1)
        assert abs(np.sum(z * phi[k]) - mult[k]) < 1e-12
    # w = 4/5 is the weight that balances the two ends; another weight gives a larger factor
    for w in (2.0 / 3.0, 0.9, 1.0):
        assert max(abs(1 - 2 * w), 1 - w / 2) > 0.6


def _grid(N):
    h = 1.0 / (N + 1)
    x = np.arange(1, N + 1) * h
    return x[None, :], x[:, None]             # (x1 over i, x2 over j) on the [j, i] grid


def _bilinear(x1, x2):
    return 0.3 + 1.7 * x1 - 0.9 * x2 + 2.3 * x1 * x2


@pytest.mark.parametrize("Nf", [7, 31, 63])
def test_prolongation_reproduces_bilinear_functions(Nf):
    Nc = (Nf - 1) // 2
    E = _bilinear(*_grid(Nc))
    fine = mg.prolong(E, Nf)
    want = _bilinear(*_grid(Nf))
    # every fine node whose interpolation stencil uses interior coarse nodes only (the outermost
    # fine rows and columns lean on the zero boundary)
    assert np.abs(fine[1:-1, 1:-1] - want[1:-1, 1:-1]).max() < 1e-13
    # coarse nodes are copied
    assert np.abs(fine[1::2, 1::2] - E).max() == 0.0


@pytest.mark.parametrize("Nf", [7, 31, 63])
def test_full_weighting_restricts_bilinear_functions_exactly(Nf):
    R = _bilinear(*_grid(Nf))
    Nc = (Nf - 1) // 2
    assert np.abs(mg.restrict(R) - _bilinear(*_grid(Nc))).max() < 1e-13


def test_coarse_edge_coefficients_of_an_affine_a():
    """a(x) = c0 + c1 x1 + c2 x2 sampled at the fine edge midpoints: every coarser level's edge
    coefficients equal a at that level's own edge midpoints (the mean of two collinear fine edges
    is a at their common midpoint)."""
    def a_fun(x1, x2):
        return 1.1 + 0.7 * x1 - 0.4 * x2

    def edges(N):
        h = 1.0 / (N + 1)
        e = np.arange(N + 1)
        i = np.arange(1, N + 1)
        ax = a_fun((e[None, :] + 0.5) * h, i[:, None] * h)     # x1-edge e of row j (x2 = j h)
        ay = a_fun(i[None, :] * h, (e[:, None] + 0.5) * h)     # x2-edge e of column i
        return ax, ay

    N = 63
    ax, ay = edges(N)
    levels = mg.hierarchy(N, ax, ay, 1.0)
    assert [L.N for L in levels] == [63, 31, 15, 7, 3, 1]
    for L in levels[1:]:
        axw, ayw = edges(L.N)
        assert np.abs(L.ax - axw).max() < 1e-14 and np.abs(L.ay - ayw).max() < 1e-14, L.N


def _lfa_two_grid(N, a, tau, mu, nu1, nu2):
    """The two-grid error operator in the sine basis, block by block: harmonics (p, q), (p', q),
    (p, q'), (p', q') with p' = N + 1 - p are coupled by full weighting and bilinear prolongation,
    whose 1D weights on the pair (p, p') are (cos^2(p pi h/2), -sin^2(p pi h/2)); the coarse
    operator is the 5-point one on H = 2h, eigenvalues mu + tau a (4/H^2)(sin^2(p pi H/2) + ...).
    Returns the (N^2 x N^2) matrix indexed [(p-1) N + (q-1)]."""
    h = 1.0 / (N + 1)
    Nc = (N - 1) // 2
    p = np.arange(1, N + 1)
    kap = 4.0 / h ** 2 * np.sin(p * math.pi * h / 2) ** 2
    D = mu + 4.0 * tau * a / h ** 2
    lam = mu + tau * a * (kap[:, None] + kap[None, :])
    s = 1.0 - mg.JACOBI_WEIGHT * lam / D
    E = np.diag((s ** (nu1 + nu2)).ravel()).astype(complex)
    idx = lambda pp, qq: (pp - 1) * N + (qq - 1)
    for pc in range(1, Nc + 1):
        for qc in range(1, Nc + 1):
            ps, qs = (pc, N + 1 - pc), (qc, N + 1 - qc)
            harm = [(ps[0], qs[0]), (ps[1], qs[0]), (ps[0], qs[1]), (ps[1], qs[1])]
            w = np.array([(math.cos(pc * math.pi * h / 2) ** 2 if kp == 0 else -math.sin(pc * math.pi * h / 2) ** 2)
                          * (math.cos(qc * math.pi * h / 2) ** 2 if kq == 0 else -math.sin(qc * math.pi * h / 2) ** 2)
                          for kq in (0, 1) for kp in (0, 1)])
            lam_h = np.array([lam[pp - 1, qq - 1] for pp, qq in harm])
            s_h = np.array([s[pp - 1, qq - 1] for pp, qq in harm])
            lam_c = mu + tau * a / h ** 2 * (math.sin(pc * math.pi * h) ** 2 + math.sin(qc * math.pi * h) ** 2)
            cgc = np.eye(4) - np.outer(w, w * lam_h) / lam_c
            blk = np.diag(s_h ** nu2) @ cgc @ np.diag(s_h ** nu1)
            ids = [idx(pp, qq) for pp, qq in harm]
            E[np.ix_(ids, ids)] = blk
    return E


def _to_sine_basis(E_apply, N):
    """Matrix of a grid operator in the orthonormal sine basis, indexed [(p-1) N + (q-1)]."""
    phi = _sine_modes(N).reshape(N * N, N, N)
    cols = np.stack([E_apply(phi[k].astype(complex)) for k in range(N * N)])   # (mode, j, i)
    return (cols.reshape(N * N, N * N) @ phi.reshape(N * N, N * N).T).T


@pytest.mark.parametrize("N,a,tau,mu", [(15, 1.0, 0.01, 0.0), (15, 0.4, 0.02, 7.5), (15, 1.0, 0.003, 2.0 + 30.0j)])
def test_two_grid_from_the_oracles_parts_matches_fourier_analysis(N, a, tau, mu):
    L = _const_level(N, a, tau)
    levels = mg.hierarchy(N, L.ax, L.ay, tau)
    C = levels[1]
    Nc = C.N
    # the coarse operator mu I + tau K_c as a dense matrix (from the coarse level's own stencil)
    eye = np.eye(Nc * Nc).reshape(Nc * Nc, Nc, Nc)
    Ac = np.stack([(mu * e + tau * C.K(e)).ravel() for e in eye], axis=1)

    def two_grid(e):
        z = mg.smooth(L, mu, e, np.zeros_like(e), 2)
        r = -(mu * z + tau * L.K(z))
        ec = np.linalg.solve(Ac, mg.restrict(r).ravel()).reshape(Nc, Nc)
        z = z + mg.prolong(ec, N)
        return mg.smooth(L, mu, z, np.zeros_like(z), 2)

    E = _to_sine_basis(two_grid, N)
    F = _lfa_two_grid(N, a, tau, mu, 2, 2)
    assert np.abs(E - F).max() < 1e-10, np.abs(E - F).max()
    rho = np.abs(np.linalg.eigvals(F)).max()
    assert rho < 0.2, rho                    # a good two-grid method for these operators


@pytest.mark.parametrize("mu", [0.0, 5.0, 1.0 + 4.0j])
def test_two_level_vcycle_matches_fourier_analysis(mu):
    """N = 3 has two levels (3 -> 1, exact coarse solve): the oracle's V-cycle is the two-grid
    method, so its error operator I - V A must equal the Fourier analysis exactly."""
    N, a, tau = 3, 1.0, 0.25
    L = _const_level(N, a, tau)
    levels = mg.hierarchy(N, L.ax, L.ay, tau)

    def err_op(e):
        return e - mg.vcycle(levels, mu, mu * e + tau * L.K(e), 2, 2)

    E = _to_sine_basis(err_op, N)
    assert np.abs(E - _lfa_two_grid(N, a, tau, mu, 2, 2)).max() < 1e-12


def test_multigrid_operator_and_diagonal_match_the_discretisation():
    """With a variable a(x) the finest level's operator and the Jacobi diagonal are those of the
    assembled K of the discretisation (Sec. 1, conservative 5-point stencil), entry by entry."""
    import synth
    from oracle import discretisation as ds
    N = 31
    prob = ds.Problem(N, 4, 1.0, 1e-2, a_edges=synth.variable_coefficient_edges(N))
    ax, ay = prob.edges()
    L = mg.hierarchy(N, ax, ay, prob.tau)[0]
    K = ds.K_sparse(prob)
    assert np.abs(L.diagK.ravel() - K.diagonal()).max() < 1e-10 * np.abs(K.diagonal()).max()
    U = np.random.default_rng(3).standard_normal((5, N, N))
    KU = np.stack([(K @ u.ravel()).reshape(N, N) for u in U])
    assert np.abs(L.K(U) - KU).max() < 1e-12 * np.abs(KU).max()


# ---------------------------------------------------------------- Neumann grids (Example 3's route)
def _neumann_grid(N):
    x = np.arange(N) / (N - 1)
    return x[None, :], x[:, None]


@pytest.mark.parametrize("Nf", [5, 17, 65])
def test_neumann_prolongation_reproduces_bilinear_functions(Nf):
    """Coarse nodes are the even fine nodes, boundary included, so bilinear interpolation is exact
    for bilinear functions on the whole fine grid."""
    Nc = (Nf + 1) // 2
    E = _bilinear(*_neumann_grid(Nc))
    assert np.abs(mg.prolong_neumann(E, Nf) - _bilinear(*_neumann_grid(Nf))).max() < 1e-13


def test_neumann_restriction_is_second_order_on_compatible_functions():
    """Full weighting with mirrored ghosts reproduces a smooth function with zero normal derivative
    (cos(pi x1) cos(pi x2)) at the coarse nodes to O(h^2), boundary nodes included."""
    errs = []
    for Nf in (17, 33, 65):
        X, Y = _neumann_grid(Nf)
        Xc, Yc = _neumann_grid((Nf + 1) // 2)
        f = lambda x, y: np.cos(math.pi * x) * np.cos(math.pi * y)
        errs.append(np.abs(mg.restrict_neumann(f(X, Y)) - f(Xc, Yc)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_neumann_operator_matches_the_discretisation():
    """Every level's operator is the mirrored stencil of the discretisation on that level's grid."""
    from oracle import discretisation as ds
    for L in mg.hierarchy_neumann(33, 1e-3, 0.01):
        prob = ds.Problem(L.N, 4, 1.0, 1e-2, bc="neumann", a0=1e-3)
        U = np.random.default_rng(L.N).standard_normal((2, L.N, L.N))
        ref = np.stack([(ds.K_sparse(prob) @ u.ravel()).reshape(L.N, L.N) for u in U])
        assert np.abs(L.K(U) - ref).max() <= 1e-12 * np.abs(ref).max()
    assert [L.N for L in mg.hierarchy_neumann(65, 1e-3, 0.01)] == [65, 33, 17, 9, 5, 3]


@pytest.mark.parametrize("mu", [0.5 + 3.0j, 4.0])
def test_neumann_vcycles_converge_to_the_exact_shifted_solve(mu):
    """The V-cycle on the Neumann grid contracts the error by a factor that stays bounded as the grid
    is refined, towards the exact shifted solve of the DCT-I route; on the 3 x 3 grid the cycle is
    the exact solve."""
    from oracle import spectra as spc
    rates = []
    for N in (17, 33, 65):
        tau, a0 = 0.02, 0.3
        levels = mg.hierarchy_neumann(N, a0, tau)
        L = levels[0]
        R = np.random.default_rng(N).standard_normal((N, N)) + 1j * np.random.default_rng(N + 1).standard_normal((N, N))
        # exact solve through the DCT-I eigenbasis of the mirrored stencil (the oracle's pinned route)
        kap = a0 * spc.kappa2d(N, "neumann")
        Z = spc.space_inverse(spc.space_forward(R.ravel(), N, "neumann") / (mu + tau * kap.ravel()), N, "neumann")
        Z = Z.reshape(N, N)
        e1 = np.abs(mg.solve(levels, mu, R, 1) - Z).max() / np.abs(Z).max()
        e4 = np.abs(mg.solve(levels, mu, R, 4) - Z).max() / np.abs(Z).max()
        rates.append((e4 / e1) ** (1 / 3))
        assert e4 < e1
    # measured: 0.04-0.18 from N = 17 to 257, levelling off
    assert max(rates) < 0.25, rates
    levels = mg.hierarchy_neumann(3, 0.3, 0.02)
    R = np.random.default_rng(3).standard_normal((3, 3)) + 0j
    Z = mg.vcycle(levels, mu, R)
    assert np.abs(mu * Z + 0.02 * levels[0].K(Z) - R).max() < 1e-12

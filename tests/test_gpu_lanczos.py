"""The product of a MINRES iteration with its Lanczos epilogue (C-ABI pcb_lanczos_product):
out = A y / beta - (beta/oldb) r1 and y . out / beta, against the FP64 oracle's A (Eq. matrix_A).

FP64: within 1e-13 (relative 2-norm and max-norm, tests/closeness.py).  Two-word FP32 (the inner
iterations of a mixed-precision solve): every value within 2^-44 of the magnitude of its terms,
|out - ref| <= 2^-44 (|A| |y| / beta + (beta/oldb) |r1|) componentwise (the arithmetic carries
47 significand bits of each input, 2^-46 relative, and rounds each operation to about 2^-48), and the dot within
2^-44 of sum |y| (|A| |y| / beta + ...) / beta.  Shapes span several 32 x 4 patches with ragged
edges, several time chunks with a ragged last chunk, n = 2, and Neumann grids."""
import numpy as np
import pytest
import torch

import synth
from closeness import assert_close
from oracle import discretisation as ds
from oracle import operators as op

pytestmark = pytest.mark.gpu
TOL_TW = 2.0 ** -44


@pytest.fixture(scope="module")
def P():
    from paper_2406_00952_gb300 import _build
    _build.build()
    import paper_2406_00952_gb300 as P
    return P


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def abs_A(prob, y):
    """|A| |y| for theta = 1 and a constant coefficient: the operator of Eq. matrix_A with every
    coefficient replaced by its absolute value (zero or mirrored neighbours as in A)."""
    N, n, m = prob.N, prob.n, prob.m
    c = prob.tau * prob.a0 / prob.h ** 2
    u1 = np.abs(y[:m * n]).reshape(n, N, N)
    u2 = np.abs(y[m * n:]).reshape(n, N, N)

    def absK(u):
        p = np.zeros((n, N + 2, N + 2))
        p[:, 1:-1, 1:-1] = u
        if prob.bc == "neumann":
            p[:, 0, 1:-1] = u[:, 1]; p[:, -1, 1:-1] = u[:, -2]
            p[:, 1:-1, 0] = u[:, :, 1]; p[:, 1:-1, -1] = u[:, :, -2]
        return c * (4 * u + p[:, 1:-1, :-2] + p[:, 1:-1, 2:] + p[:, :-2, 1:-1] + p[:, 2:, 1:-1])

    z = np.zeros((1, N, N))
    T1 = u1 + np.concatenate([z, u1[:-1]]) + absK(u1)           # |T| |x1|
    TT2 = u2 + np.concatenate([u2[1:], z]) + absK(u2)           # |T^T| |x2|
    a = prob.alpha
    return np.concatenate([(a * u1 + TT2).ravel(), (T1 + a * u2).ravel()])


CASES = [  # (N, n, bc): 511 = 15 * 32 + 31 = 127 * 4 + 3 (ragged patches); n = 8 at N = 511 and
           # n = 64 at N = 255 run time chunks of 3 and 6 (ragged last chunk); n = 2: one chunk of two levels
    (5, 2, "dirichlet"), (31, 16, "dirichlet"), (47, 8, "dirichlet"), (95, 32, "dirichlet"),
    (255, 64, "dirichlet"), (511, 8, "dirichlet"), (31, 2, "dirichlet"),
    (33, 16, "neumann"), (65, 8, "neumann"), (257, 4, "neumann")]


def _setup(P, N, n, bc, precision, seed):
    gamma = 1e-2
    prob = ds.Problem(N, n, 1.0, gamma, bc=bc)
    gp = P.Problem(N, n, 1.0, gamma, precision=precision, bc=bc)
    rng = np.random.default_rng(seed)
    L = 2 * prob.m * n
    # a smooth field plus noise (the cancellation of smooth vectors), some exact zeros
    y = synth.random_vector(L, seed=seed) * 1e-3 + np.sin(np.arange(L) * 1e-3) * 0.5
    y[rng.integers(0, L, max(1, L // 50))] = 0.0
    r1 = synth.random_vector(L, seed=seed + 1)
    return prob, gp, y, r1


@pytest.mark.parametrize("case", CASES)
def test_lanczos_product(P, case):
    N, n, bc = case
    for k, (beta, oldb) in enumerate(((0.37, 0.0), (2.3e-3, 4.1e-3))):
        prob, gp, y, r1 = _setup(P, N, n, bc, "mixed", 11 + k)
        ref = op.matvec_A(prob, y) / beta - ((beta / oldb) * r1 if oldb > 0 else 0.0)
        dref = float(y @ ref) / beta
        mag = abs_A(prob, y) / beta + ((beta / oldb) * np.abs(r1) if oldb > 0 else 0.0)
        yd, rd = dev(y), (dev(r1) if oldb > 0 else None)
        o64, d64 = gp.lanczos_product(yd, beta, rd, oldb, precision="fp64")
        assert_close(o64.cpu().numpy(), ref, 1e-13, what="fp64 product")
        assert abs(d64 - dref) <= 1e-13 * float(np.abs(y) @ mag) / beta
        otw, dtw = gp.lanczos_product(yd, beta, rd, oldb, precision="mixed")
        err = np.abs(otw.cpu().numpy() - ref)
        worst = float(np.max(err / np.maximum(mag, 1e-300)))
        assert np.all(err <= TOL_TW * mag), (case, k, worst, int(np.argmax(err / np.maximum(mag, 1e-300))))
        assert abs(dtw - dref) <= TOL_TW * float(np.abs(y) @ mag) / beta, (dtw, dref)
        gp.close()


# The states a MINRES iteration produces: in the first iteration y = P^-1 b and beta carry the scale
# of b and there is no r1 term; later y and beta are free of it, while r1 = b and oldb still carry
# it in the second iteration.  The output is free of the scale in every case.
@pytest.mark.parametrize("scale", [(1e-200, 0.0), (1e200, 0.0), (2.0 ** -1000, 0.0), (1.0, 1e200), (1.0, 1e-200)])
def test_lanczos_product_scale_invariance(P, scale):
    """The two-word split is taken relative to the binades of beta and oldb: inputs far outside
    the FP32 range keep their accuracy."""
    sy, sr = scale
    N, n = 63, 16
    prob, gp, y, r1 = _setup(P, N, n, "dirichlet", "mixed", 5)
    beta, oldb = 0.37 * sy, 0.59 * sr
    # the reference from the unscaled inputs (the same values; FP64 itself would lose digits to
    # subnormal intermediates at 2^-1000)
    kr1 = (0.37 * sy / 0.59) * r1 if sr else 0.0
    ref = op.matvec_A(prob, y) / 0.37 - kr1
    mag = abs_A(prob, y) / 0.37 + np.abs(kr1)
    out, dot = gp.lanczos_product(dev(y * sy), beta, dev(r1 * sr) if sr else None, oldb, precision="mixed")
    err = np.abs(out.cpu().numpy() - ref)
    assert np.all(err <= TOL_TW * mag), float(np.max(err / mag))
    assert abs(dot - float(y @ ref) / 0.37) <= TOL_TW * float(np.abs(y) @ mag) / 0.37
    gp.close()


def test_lanczos_product_nonfinite_and_arguments(P):
    prob, gp, y, r1 = _setup(P, 31, 8, "dirichlet", "mixed", 3)
    y[17] = np.nan
    for prec in ("mixed", "fp64"):
        out, dot = gp.lanczos_product(dev(y), 1.0, None, 0.0, precision=prec)
        assert not np.isfinite(dot)
    with pytest.raises(RuntimeError):
        gp.lanczos_product(dev(y), 0.0)
    with pytest.raises(RuntimeError):
        gp.lanczos_product(dev(y), 1.0, None, 2.0)      # oldb > 0 needs r1
    gp.close()

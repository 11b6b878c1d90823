"""Where the FP32 preconditioner costs MINRES iterations (a study, run by hand; not collected by
pytest).  The oracle's |P_S|^{-1} (Sec. 3.5: DST-I in x1 and x2, the zeta = pi time DFT, the weight
1/sqrt(|lambda_k + tau kappa_pq|^2 + alpha^2), the inverse transforms) is re-run with every stage
in FP32 (library single-precision transforms) except the stages named on the command line, inside
the same FP64 iterative refinement the library runs (inner MINRES to tol ||b||/||r||, FP64 true
residual, x += d), on the bench family's problem (backward Euler, a = 1, seed-1 target).

    python tests/fp32_rounding_study.py N gamma 'exact;;t,ti;x1,x2,x2i,x1i;@split47;@split47+noise=4e-15'

Each ';'-separated variant lists the stages kept in FP64: x1, x2 (forward DSTs), t (forward time
DFT), w (weights), ti (inverse time DFT), x2i, x1i (inverse DSTs); 'exact' is the FP64 oracle;
'noise=E' is the FP64 oracle with a relative perturbation of size E (random sign, seeded) on every
output value, which measures how much inexactness the solve tolerates.  A suffix '@split47' makes
the inner iterations' product act on its input truncated to 47 significand bits (the two FP32
words of the mixed solve's two-word product: the leading 24 bits and the next 23, both
truncated), '@split47+noise=E' adds a perturbation of E |A| |z| with random signs to it; the
refinement's true residuals keep the FP64 product.
Prints one JSON line per variant: total inner iterations and the iterations of each sweep.
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np
import scipy.fft as sf

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synth  # noqa: E402
from oracle import discretisation as ds  # noqa: E402
from oracle import operators as op  # noqa: E402
from oracle import precond as pc  # noqa: E402
from oracle import spectra as spc  # noqa: E402


def make_apply(prob, fp64_stages=()):
    """|P_S|^{-1} with the listed stages in FP64 and the rest in FP32 (zeta = pi, a = 1)."""
    N, n = prob.N, prob.n
    lam = spc.lam_Sn(n, prob.theta, prob.zeta)
    kap = spc.kappa2d(N)
    W64 = 1.0 / np.sqrt(np.abs(lam[:, None, None] + prob.tau * kap[None]) ** 2 + prob.alpha ** 2)
    W32 = W64.astype(np.float32)
    d64 = spc.D_omega(n, prob.zeta)
    d32 = d64.astype(np.complex64)

    def dst(u, ax, stage):
        if stage in fp64_stages:
            return sf.dst(u.astype(np.complex128 if np.iscomplexobj(u) else np.float64), type=1, axis=ax, norm="ortho")
        return sf.dst(u.astype(np.complex64 if np.iscomplexobj(u) else np.float32), type=1, axis=ax, norm="ortho")

    def apply(v):
        mn = prob.m * n
        h0 = v[:mn].reshape(n, N, N); h1 = v[mn:].reshape(n, N, N)
        a0 = dst(dst(h0, -1, "x1"), -2, "x2"); a1 = dst(dst(h1, -1, "x1"), -2, "x2")
        # the two real halves as one complex line (the operator is real at zeta = pi)
        if "t" in fp64_stages:
            Z = np.fft.fft((a0.astype(np.float64) + 1j * a1.astype(np.float64)) * d64[:, None, None], axis=0)
        else:
            Z = sf.fft((a0.astype(np.float32) + 1j * a1.astype(np.float32)).astype(np.complex64) * d32[:, None, None], axis=0)
        Z = Z * (W64 if "w" in fp64_stages else W32)
        if "ti" in fp64_stages:
            z = np.fft.ifft(Z.astype(np.complex128), axis=0) / d64[:, None, None]
        else:
            z = sf.ifft(Z.astype(np.complex64), axis=0) / d32[:, None, None]
        b0 = dst(dst(np.real(z), -2, "x2i"), -1, "x1i"); b1 = dst(dst(np.imag(z), -2, "x2i"), -1, "x1i")
        return np.concatenate([b0.astype(np.float64).ravel(), b1.astype(np.float64).ravel()])
    return apply


def minres_inner(A, b, M, tol, maxit):
    """Preconditioned MINRES (Paige-Saunders) from zero, stopped when its residual estimate reaches
    tol (the library's inner solve of a refinement sweep)."""
    x = np.zeros_like(b)
    r1 = b.copy(); y = M(r1); beta1 = math.sqrt(r1 @ y)
    oldb, beta, dbar, epsln, phibar = 0.0, beta1, 0.0, 0.0, beta1
    cs, sn = -1.0, 0.0
    w = np.zeros_like(b); w2 = np.zeros_like(b); r2 = r1.copy()
    for itn in range(1, maxit + 1):
        v = y / beta; y = A(v)
        if itn >= 2:
            y = y - (beta / oldb) * r1
        alfa = v @ y; y = y - (alfa / beta) * r2
        r1, r2 = r2, y; y = M(r2); oldb = beta
        beta = math.sqrt(r2 @ y)
        oldeps = epsln; delta = cs * dbar + sn * alfa; gbar = sn * dbar - cs * alfa
        epsln = sn * beta; dbar = -cs * beta; gamma = math.hypot(gbar, beta)
        cs, sn = gbar / gamma, beta / gamma; phi = cs * phibar; phibar = sn * phibar
        w1, w2 = w2, w; w = (v - oldeps * w1 - delta * w2) / gamma; x = x + phi * w
        if phibar / beta1 <= tol:
            return x, itn
    return x, maxit


def split47(x):
    """The value the two FP32 words hold: the leading 24 significand bits and the next 23, i.e. x
    with the last 6 of its 52 stored mantissa bits cleared (normal values)."""
    return (x.view(np.uint64) & np.uint64(0xFFFFFFFFFFFFFFC0)).view(np.float64)


def refine(A, b, M, tol=1e-8, maxit=400, A_inner=None):
    A_inner = A_inner or A
    x = np.zeros_like(b); bn = np.linalg.norm(b); r = b.copy(); rn = bn; its = 0; sweeps = []
    while rn / bn > tol and its < maxit:
        d, k = minres_inner(A_inner, r, M, min(0.5, tol * bn / rn), maxit - its)
        its += k; sweeps.append(k)
        x = x + d; r = b - A(x); rn = np.linalg.norm(r)
    return x, its, sweeps, rn / bn


def main(N, gamma, variants):
    n = N + 1
    prob = ds.Problem(N, n, 1.0, gamma)
    b = ds.rhs_minres(prob, synth.random_target(N, n, seed=1), synth.manufactured_source(N, n))
    A = lambda z: op.matvec_A(prob, z)
    for var in variants:
        var, _, inner = var.partition("@")
        A_inner = None
        if inner.startswith("split47"):
            eps = float(inner.split("noise=")[1]) if "noise=" in inner else 0.0
            rng_i = np.random.default_rng(3)

            def A_inner(z, eps=eps, rng_i=rng_i):
                y = A(split47(z))
                if eps:   # the size of the terms taken as |A |z||
                    y = y + eps * np.abs(A(np.abs(z))) * rng_i.choice([-1.0, 1.0], z.size)
                return y
        if var == "exact":
            M = lambda r: pc.apply_abs_ps_inv(prob, r)
        elif var.startswith("noise="):
            eps, rng = float(var[6:]), np.random.default_rng(7)
            M = lambda r, eps=eps, rng=rng: (lambda z: z * (1.0 + eps * rng.choice([-1.0, 1.0], z.size)))(
                pc.apply_abs_ps_inv(prob, r))
        else:
            M = make_apply(prob, tuple(v for v in var.split(",") if v))
        t0 = time.time()
        _, its, sw, rr = refine(A, b, M, A_inner=A_inner)
        print(json.dumps({"N": N, "gamma": gamma, "fp64_stages": var, "inner_product": inner or "fp64",
                          "iterations": its, "sweeps": sw,
                          "relres": rr, "seconds": round(time.time() - t0, 1)}), flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]), float(sys.argv[2]), sys.argv[3].split(";"))

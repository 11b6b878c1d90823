"""Element-wise comparison of a GPU result with the oracle's.

Every parity test checks two figures, so that neither a spread-out error nor one confined to a few
values passes unseen:
  rel2   = ||out - ref||_2 / ||ref||_2                 (relative 2-norm)
  relmax = max_i |out_i - ref_i| / max_i |ref_i|       (relative max-norm)
Structured checks (`assert_close_by_parts`) add the worst relative 2-norm over each part of a
partition (one time slice, one grid line, one half), so that a defect confined to one boundary line,
one frequency slot or one instance does not hide under the whole vector's norm.
"""
from __future__ import annotations

import numpy as np


def rel2(out, ref) -> float:
    return float(np.linalg.norm(out - ref) / max(np.linalg.norm(ref), 1e-300))


def relmax(out, ref) -> float:
    return float(np.max(np.abs(out - ref)) / max(np.max(np.abs(ref)), 1e-300)) if ref.size else 0.0


def errors(out, ref) -> dict:
    out = np.asarray(out, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    assert out.shape == ref.shape, (out.shape, ref.shape)
    assert np.all(np.isfinite(out)), "non-finite values in the result"
    return {"rel2": rel2(out, ref), "relmax": relmax(out, ref)}


def assert_close(out, ref, tol2, tolmax=None, what=""):
    """rel2 <= tol2 and relmax <= tolmax (default: tol2)."""
    e = errors(out, ref)
    tolmax = tol2 if tolmax is None else tolmax
    assert e["rel2"] <= tol2 and e["relmax"] <= tolmax, (what, e, tol2, tolmax)
    return e


def worst_part(out, ref, shape, axes) -> float:
    """Largest relative 2-norm error over the parts of `shape` that keep `axes` fixed: e.g.
    shape (2, n, N, N) with axes (0, 1) compares each (half, time) slice on its own."""
    o = np.asarray(out, dtype=np.float64).reshape(shape)
    r = np.asarray(ref, dtype=np.float64).reshape(shape)
    red = tuple(a for a in range(len(shape)) if a not in axes)
    num = np.sqrt(np.sum((o - r) ** 2, axis=red))
    den = np.sqrt(np.sum(r ** 2, axis=red))
    return float(np.max(num / np.maximum(den, 1e-300)))


def assert_close_by_parts(out, ref, shape, tol, partitions, what=""):
    """For every partition (a tuple of kept axes) the worst part's relative 2-norm is <= tol."""
    worst = {str(ax): worst_part(out, ref, shape, ax) for ax in partitions}
    assert all(v <= tol for v in worst.values()), (what, worst, tol)
    return worst

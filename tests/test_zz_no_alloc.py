"""The allocation-free preconditioner apply (pcb_precond_apply_noalloc) against the allocating
entry point (pcb_precond_apply) through the C ABI, for callers that cannot use cudaMalloc.
Collected last on purpose; passes alone in a fresh process and after the other tests."""
import ctypes
import math

import numpy as np
import pytest
import torch

import synth
from closeness import assert_close
from oracle import discretisation as ds
from oracle import precond as pc

pytestmark = pytest.mark.gpu
ORACLE = {"abs_ps": pc.apply_abs_ps_inv, "ps": pc.apply_ps_inv, "pms": pc.apply_pms_inv}

KIND = {"abs_ps": 1, "ps": 2, "pms": 3}
PREC = {"fp64": 0, "mixed": 1}
TOL = {"fp64": 1e-12, "mixed": 2e-6}       # same bounds as the oracle parity tests


@pytest.fixture(scope="module")
def lib():
    from paper_2406_00952_gb300 import _build, _lib
    _build.build()
    return _lib.load()


def _desc(N, n, theta, gamma, zeta=math.pi):
    from paper_2406_00952_gb300 import _lib
    s = torch.cuda.current_stream().cuda_stream
    return _lib.PcbDesc(N, n, theta, 1.0, gamma, zeta, None, 0, 2, ctypes.c_void_p(s))


# (N, n, theta, gamma, kind, precision, seed, zeta)
CASES = [(63, 64, 1.0, 1e-2, "abs_ps", "mixed", 1, math.pi), (31, 16, 0.5, 1e-4, "ps", "fp64", 2, math.pi),
         (95, 32, 0.75, 1e-3, "pms", "mixed", 3, math.pi), (63, 64, 1.0, 1e-2, "abs_ps", "mixed", 4, math.pi / 2),
         (31, 32, 0.5, 1e-3, "ps", "mixed", 5, 0.4)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "N%d-n%d-%s-%s-z%.2f" % (c[0], c[1], c[4], c[5], c[7]))
def test_noalloc_matches_allocating_apply_two_calls_in_a_row(lib, case):
    """Two calls in a row give the allocating entry point's result (and the oracle's), including a
    general zeta, whose unpadded scratch runs the general-zeta time pass."""
    import paper_2406_00952_gb300 as P
    N, n, theta, gamma, kind, prec, seed, zeta = case
    size = 2 * N * N * n
    v = synth.random_vector(size, seed=seed)
    x = torch.from_numpy(v).cuda()
    ref = P.Problem(N, n, theta, gamma, zeta=zeta).precond_apply(x, kind=kind, precision=prec).cpu().numpy()
    oracle = ORACLE[kind](ds.Problem(N, n, theta, gamma, zeta=zeta), v)
    d = _desc(N, n, theta, gamma, zeta)
    for call in range(2):
        y = torch.full((size,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.pcb_precond_apply_noalloc(ctypes.byref(d), KIND[kind], PREC[prec], x.data_ptr(), y.data_ptr())
        assert rc == 0, rc
        out = y.cpu().numpy()
        assert_close(out, ref, TOL[prec], what=("allocating", call))
        assert_close(out, oracle, TOL[prec], what=("oracle", call))


def test_noalloc_in_place(lib):
    """x and y the same buffer, as the header allows."""
    N, n, theta, gamma = 63, 64, 1.0, 1e-3
    v = synth.random_vector(2 * N * N * n, seed=6)
    oracle = pc.apply_abs_ps_inv(ds.Problem(N, n, theta, gamma), v)
    d = _desc(N, n, theta, gamma)
    for prec in ("fp64", "mixed"):
        t = torch.from_numpy(v).cuda()
        assert lib.pcb_precond_apply_noalloc(ctypes.byref(d), KIND["abs_ps"], PREC[prec], t.data_ptr(), t.data_ptr()) == 0
        assert_close(t.cpu().numpy(), oracle, TOL[prec], what=prec)


def test_noalloc_neumann_ps(lib):
    """Example 3's Neumann grid through the allocation-free entry: the DCT-I passes; |P_S| refused."""
    import paper_2406_00952_gb300 as P
    from paper_2406_00952_gb300 import _lib
    N, n = 33, 32
    size = 2 * N * N * n
    x = torch.from_numpy(synth.random_vector(size, seed=9)).cuda()
    ref = P.Problem(N, n, 0.5, 1e-3, bc="neumann", a=1e-3).precond_apply(x, kind="ps", precision="mixed").cpu().numpy()
    s = torch.cuda.current_stream().cuda_stream
    d = _lib.PcbDesc(N, n, 0.5, 1.0, 1e-3, math.pi, None, 0, 2, ctypes.c_void_p(s), 1, 1e-3)
    y = torch.full((size,), float("nan"), dtype=torch.float64, device="cuda")
    assert lib.pcb_precond_apply_noalloc(ctypes.byref(d), KIND["ps"], PREC["mixed"], x.data_ptr(), y.data_ptr()) == 0
    assert_close(y.cpu().numpy(), ref, TOL["mixed"])
    oracle = pc.apply_ps_inv(ds.Problem(N, n, 0.5, 1e-3, bc="neumann", a0=1e-3), x.cpu().numpy())
    assert_close(y.cpu().numpy(), oracle, TOL["mixed"])
    assert lib.pcb_precond_apply_noalloc(ctypes.byref(d), KIND["abs_ps"], PREC["mixed"], x.data_ptr(), y.data_ptr()) == -2


def test_noalloc_rejects_sizes_beyond_the_arena(lib):
    d = _desc(511, 512, 1.0, 1e-2)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert lib.pcb_precond_apply_noalloc(ctypes.byref(d), 1, 1, x.data_ptr(), x.data_ptr()) == -9
    assert lib.pcb_precond_apply_noalloc(None, 1, 1, x.data_ptr(), x.data_ptr()) == -1

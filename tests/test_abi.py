"""The C-ABI library builds for sm_103a, loads, and exports every function include/pcb.h declares
(no compute calls: this runs without a GPU)."""
import ctypes

from paper_2406_00952_gb300 import _build, _lib


def test_library_builds_and_exports_header_symbols():
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = _lib.header_functions()
    assert len(names) >= 10
    missing = [f for f in names if not hasattr(lib, f)]
    assert not missing, missing


def test_status_strings():
    lib = _lib.load()
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8, -9):
        assert lib.pcb_status_str(code)
    assert lib.pcb_status_str(-1) == b"invalid argument"


def test_create_rejects_invalid_descriptors_without_touching_the_gpu():
    """Argument validation happens before any CUDA call."""
    lib = _lib.load()
    bad = [dict(N=0, n=4, theta=1.0, gamma=1.0), dict(N=3, n=1, theta=1.0, gamma=1.0),
           dict(N=3, n=4, theta=0.4, gamma=1.0), dict(N=3, n=4, theta=1.0, gamma=0.0),
           dict(N=3, n=4, theta=1.0, gamma=-1.0)]
    for b in bad:
        d = _lib.PcbDesc(b["N"], b["n"], b["theta"], 1.0, b["gamma"], 3.141592653589793, None, 0, 2, None)
        h = ctypes.c_void_p()
        assert lib.pcb_create(ctypes.byref(d), ctypes.byref(h)) == -1
    # unsupported: n not a power of two, N+1 not 2^a 3^b
    for N, n, z in ((3, 6, 3.141592653589793), (4, 4, 3.141592653589793)):
        d = _lib.PcbDesc(N, n, 1.0, 1.0, 1e-2, z, None, 0, 2, None)
        h = ctypes.c_void_p()
        assert lib.pcb_create(ctypes.byref(d), ctypes.byref(h)) == -2
    # unsupported: variable a(x) with zeta != pi (the multigrid route pairs conjugate slots)
    a = (ctypes.c_double * (2 * 3 * 4))(*([1.0] * 24))
    d = _lib.PcbDesc(3, 4, 1.0, 1.0, 1e-2, 0.4, a, 0, 2, None)
    h = ctypes.c_void_p()
    assert lib.pcb_create(ctypes.byref(d), ctypes.byref(h)) == -2
    # Neumann: N-1 must be 2^a 3^b (DCT-I radices), 3 <= N <= 513, no a_edges; bc outside the enum
    for N in (2, 6, 514, 1025):
        d = _lib.PcbDesc(N, 4, 0.5, 1.0, 1e-2, 3.141592653589793, None, 0, 2, None, 1, 1e-3)
        assert lib.pcb_create(ctypes.byref(d), ctypes.byref(h)) == -2, N
    a = (ctypes.c_double * (2 * 3 * 4))(*([1.0] * 24))
    d = _lib.PcbDesc(3, 4, 0.5, 1.0, 1e-2, 3.141592653589793, a, 0, 2, None, 1, 0.0)
    assert lib.pcb_create(ctypes.byref(d), ctypes.byref(h)) == -2
    d = _lib.PcbDesc(5, 4, 0.5, 1.0, 1e-2, 3.141592653589793, None, 0, 2, None, 2, 1.0)
    assert lib.pcb_create(ctypes.byref(d), ctypes.byref(h)) == -1
    assert lib.pcb_create(None, None) == -1


def test_entry_points_reject_null_problems_without_touching_the_gpu():
    """Calls on a NULL problem handle return INVALID_ARG before any CUDA call."""
    lib = _lib.load()
    dot = ctypes.c_double()
    assert lib.pcb_lanczos_product(None, 1, None, None, 1.0, 0.0, None, ctypes.byref(dot)) == -1
    assert lib.pcb_matvec(None, 0, None, None) == -1
    assert lib.pcb_precond_apply(None, 1, 1, None, None) == -1

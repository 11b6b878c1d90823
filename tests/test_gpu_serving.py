"""Continuous batching: requests that arrive while others are on the GPU join the shared launches as
slots and budget free up; each result equals the same request solved alone (within 1e-12: the same
rounds and per-request fixed-order reductions), and meets the FP64 residual checked by the oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import discretisation as ds
from oracle import operators as op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2406_00952_gb300 import _build
    _build.build()
    import paper_2406_00952_gb300 as P
    return P


def _requests(P):
    from paper_2406_00952_gb300 import serve
    shapes = [(15, 16, 1.0, 1e-2), (31, 8, 0.5, 1e-4), (23, 32, 1.0, 1e-5), (15, 64, 0.5, 1e-2),
              (47, 16, 1.0, 1e-1), (31, 32, 0.5, 1e-3), (7, 128, 1.0, 1e-6), (63, 8, 0.5, 1e-2),
              (31, 16, 1.0, 1e-3), (15, 32, 0.5, 1e-5)]
    out = []
    for k, (N, n, th, gm) in enumerate(shapes):
        prob = ds.Problem(N, n, th, gm)
        g = synth.random_target(N, n, seed=70 + k); f = synth.manufactured_source(N, n)
        b = ds.rhs_minres(prob, g, f) if th == 1.0 else ds.rhs_gmres(prob, g, f)
        out.append((serve.Request(k, 0.002 * k, N, n, th, gm, torch.from_numpy(b).pin_memory()), prob, b))
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_served_results_equal_alone(P, precision):
    from paper_2406_00952_gb300 import serve
    reqs = _requests(P)
    res = serve.run([r for r, _, _ in reqs], budget_bytes=8 << 30, max_slots=3, precision=precision)
    assert res["failed"] == 0 and res["max_relres"] <= 1e-8
    for r, prob, b in reqs:
        x = r.x.numpy()
        A = (lambda z: op.matvec_A(prob, z)) if r.theta == 1.0 else (lambda z: op.matvec_A_hat(prob, z))
        assert np.linalg.norm(b - A(x)) / np.linalg.norm(b) <= 1.5e-8
        gp = P.Problem(r.N, r.n, r.theta, r.gamma, precision=precision)
        xa, ia = P.batch_solve([gp], [torch.from_numpy(b).cuda()], tol=1e-8, restart=16)
        assert np.linalg.norm(xa[0].cpu().numpy() - x) <= 1e-12 * np.linalg.norm(x)
        assert ia[0]["iterations"] == res["results"][r.tag].iterations


def test_budget_admission_and_rejection(P):
    from paper_2406_00952_gb300 import serve
    reqs = _requests(P)[:4]
    # a budget that holds one request at a time still serves all of them, with the same results
    big = max(2 * r.N * r.N * r.n for r, _, _ in reqs) * 8 * 60 + (8 << 20)
    res = serve.run([r for r, _, _ in reqs], budget_bytes=big, max_slots=8, precision="mixed")
    assert res["failed"] == 0 and res["max_relres"] <= 1e-8
    # the budget is reserved up front and each request takes exactly its workspace (about 0.7 MB
    # here): 256 KB holds none
    srv = serve.Server(budget_bytes=1 << 18, max_slots=2)
    t = torch.zeros(2 * 15 * 15 * 16, dtype=torch.float64).pin_memory()
    with pytest.raises(Exception) as e:
        srv.submit(15, 16, 1.0, 1e-2, t, t.clone(), 0)
    assert "too large" in str(e.value)
    srv.close()


def test_served_neumann_requests_beside_dirichlet(P):
    """Neumann requests (Example 3's grid, GMRES-P_S with the DCT-I passes) served in the same
    shared launches as Dirichlet ones; each equals the request solved alone."""
    from paper_2406_00952_gb300 import serve
    specs = [(33, 32, 1.0, 1e-3, "neumann", 1e-3), (31, 16, 1.0, 1e-2, "dirichlet", 1.0),
             (17, 64, 0.5, 1e-5, "neumann", 0.1), (15, 32, 0.5, 1e-3, "dirichlet", 1.0)]
    reqs = []
    for k, (N, n, th, gm, bc, a) in enumerate(specs):
        prob = ds.Problem(N, n, th, gm, bc=bc, a0=a)
        g = synth.random_target(N, n, seed=90 + k); f = synth.manufactured_source(N, n)
        gmres = th != 1.0 or bc == "neumann"
        b = ds.rhs_gmres(prob, g, f) if gmres else ds.rhs_minres(prob, g, f)
        reqs.append((serve.Request(k, 0.0, N, n, th, gm, torch.from_numpy(b).pin_memory(), bc=bc, a=a), prob, b, gmres))
    res = serve.run([r for r, _, _, _ in reqs], budget_bytes=8 << 30, max_slots=4, precision="mixed")
    assert res["failed"] == 0 and res["max_relres"] <= 1e-8
    for r, prob, b, gmres in reqs:
        x = r.x.numpy()
        A = (lambda z: op.matvec_A_hat(prob, z)) if gmres else (lambda z: op.matvec_A(prob, z))
        assert np.linalg.norm(b - A(x)) / np.linalg.norm(b) <= 1.5e-8
        gp = P.Problem(r.N, r.n, r.theta, r.gamma, precision="mixed", bc=r.bc, a=r.a)
        xa, ia = P.batch_solve([gp], [torch.from_numpy(b).cuda()], tol=1e-8, restart=16)
        assert np.linalg.norm(xa[0].cpu().numpy() - x) <= 1e-12 * np.linalg.norm(x)
        assert ia[0]["iterations"] == res["results"][r.tag].iterations

"""FP64 products emulated on the BF16 tensor cores (RANDUTV_FP64_EMULATED):
the same oracle parity and UTV bounds as the DMMA path, on shapes where the
emulated products run (at least 128 x 64 x 64) and where they fall back."""
import numpy as np
import pytest

import oracle
import synthetic
from conftest import utv_bound

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rutv():
    import paper_2104_05782_gb300 as r
    from paper_2104_05782_gb300 import build
    build.build()
    r.load()
    return r


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()


def host(X):
    return None if X is None else X.t().contiguous().cpu().numpy().T


@pytest.mark.parametrize("m,n,b,q,kind,seed", [
    (1000, 1000, 64, 1, "geometric10", 0),   # the 1000^2 parity workload
    (640, 400, 128, 2, "normal", 3),         # tall, b = 128
    (333, 200, 48, 1, "geometric10", 7),     # ragged; small steps fall back to DMMA
])
@pytest.mark.parametrize("prec_name", ["RANDUTV_FP64_EMULATED", "RANDUTV_EMULATED_SKETCH_BF16"])
def test_emulated_parity(rutv, m, n, b, q, kind, seed, prec_name):
    prec = getattr(rutv, prec_name)
    A = synthetic.test_matrix(m, n, kind, 10 + seed, 20 + seed)
    U, T, V = rutv.factor(dev(A), b, q, seed, prec=prec)
    torch.cuda.synchronize()
    U, T, V = host(U), host(T), host(V)
    nrm = np.linalg.norm(A)
    assert np.linalg.norm(A - U @ T @ V.T) / nrm <= utv_bound(n)
    assert np.linalg.norm(U.T @ U - np.eye(m)) <= utv_bound(m)
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= utv_bound(n)
    assert np.array_equal(np.tril(T, -1), np.zeros_like(T))
    if prec == rutv.RANDUTV_FP64_EMULATED:
        Uo, To, Vo, _ = oracle.randutv(A, b, q, seed)
        assert np.abs(T - To).max() <= 1e-10 * nrm
        assert np.abs(U @ T - Uo @ To).max() <= 1e-10 * nrm
        assert np.abs(T @ V.T - To @ Vo.T).max() <= 1e-10 * nrm


@pytest.mark.parametrize("prec_name", ["RANDUTV_FP64_EMULATED", "RANDUTV_EMULATED_SKETCH_BF16"])
def test_emulated_wide_updates(rutv, prec_name):
    """Trailing updates large enough (over 600 tiles of 128 x 64) for the
    32-column, two-CTAs-per-SM product; ragged in both dimensions. Two block
    steps of the factorization, checked against two steps of the oracle."""
    prec = getattr(rutv, prec_name)
    m, n, b, q, seed, steps = 4000, 3000, 128, 1, 4, 2
    A = synthetic.test_matrix(m, n, "geometric10", 31, 32)
    U, T, V = rutv.factor(dev(A), b, q, seed, prec=prec, stop_after=steps)
    torch.cuda.synchronize()
    U, T, V = host(U), host(T), host(V)
    nrm = np.linalg.norm(A)
    assert np.linalg.norm(A - U @ T @ V.T) / nrm <= utv_bound(n)
    assert np.linalg.norm(U.T @ U - np.eye(m)) <= utv_bound(m)
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= utv_bound(n)
    assert np.array_equal(np.tril(T[:, :b * steps], -1), np.zeros((m, b * steps)))
    if prec == rutv.RANDUTV_FP64_EMULATED:
        Uo, To, Vo, _ = oracle.randutv(A, b, q, seed, stop_after=steps)
        assert np.abs(T - To).max() <= 1e-10 * nrm
        assert np.abs(U @ T - Uo @ To).max() <= 1e-10 * nrm
        assert np.abs(T @ V.T - To @ Vo.T).max() <= 1e-10 * nrm

"""The host BLAS/LAPACK randUTV that bench.py times as its CPU comparison run
computes the same factorization as the oracle (same Gaussian draws, sign
rules and steps), to the tolerance the GPU path is held to."""
import numpy as np
import pytest

import bench
import oracle
import synthetic
from conftest import utv_bound


@pytest.mark.parametrize("m,n,b,q,kind,seed", [
    (200, 150, 32, 1, "geometric10", 3),   # ragged final block of 22
    (128, 128, 24, 2, "normal", 1),        # final block of 8
    (90, 60, 64, 1, "geometric10", 2),     # b >= n': one sketch step, then the final block
    (70, 40, 64, 0, "normal", 5),          # b >= n: final block only
])
def test_blas_randutv_matches_oracle(m, n, b, q, kind, seed):
    A = synthetic.test_matrix(m, n, kind, 40 + seed, 50 + seed)
    U, T, V = bench.blas_randutv(A, b, q, seed, oracle.gaussian)
    Uo, To, Vo, rc = oracle.randutv(A, b, q, seed)
    assert rc == 0
    nrm = np.linalg.norm(A)
    assert np.abs(T - To).max() <= 1e-10 * nrm
    assert np.abs(U @ T - Uo @ To).max() <= 1e-10 * nrm
    assert np.abs(T @ V.T - To @ Vo.T).max() <= 1e-10 * nrm
    assert np.linalg.norm(A - U @ T @ V.T) / nrm <= utv_bound(n)
    assert np.linalg.norm(U.T @ U - np.eye(m)) <= utv_bound(m)
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= utv_bound(n)
    assert np.array_equal(np.tril(T, -1), np.zeros_like(T))


def test_blas_randutv_t_only():
    A = synthetic.test_matrix(120, 100, "geometric10", 1, 2)
    U, T, V = bench.blas_randutv(A, 16, 1, 0, oracle.gaussian, want_uv=False)
    assert U is None and V is None
    _, To, _, _ = oracle.randutv(A, 16, 1, 0, want_uv=False)
    assert np.abs(T - To).max() <= 1e-10 * np.linalg.norm(A)


def test_cpu_blas_sample_reports_a_rate():
    val, secs, cores = bench.cpu_blas_sample(256, 32, 1, "gap")
    assert val > 0 and secs > 0 and cores >= 1

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


def test_diag_quality_reports_the_spread_beside_the_median():
    """A run of repeated sigma found exactly can hold the median of
    T_ii / sigma_i at 1 while the other ratios spread by percents."""
    n, b = 1000, 100
    sigma = np.concatenate([np.ones(100), np.geomspace(1e-3, 1e-12, n - 100)])
    r = np.concatenate([np.ones(100), 1 + 0.03 * np.where(np.arange(n - 100) % 2, 1, -1)])
    q = bench.diag_quality(r * sigma, sigma, b)
    assert q["Tii_over_sigma_median"] == 1.0
    assert abs(q["Tii_over_sigma_median_abs_dev"] - 0.03) < 1e-12
    assert q["Tii_within_5pct_of_sigma"] == 1.0
    assert q["Tii_over_sigma_first_block_max_dev"] == 0.0


def test_diag_quality_of_the_cpu_run_on_the_gap_spectrum():
    """randUTV's own rank-revealing quality on the gap spectrum (q = 2): the
    sigma = 1 block exactly, the decaying part within a few percent."""
    n, b = 2048, 128          # the sigma = 1 cluster (n / 10) fills the first block
    A = synthetic.test_matrix(n, n, "gap", 1, 2)
    _, T, _ = bench.blas_randutv(A, b, 2, 0, oracle.gaussian, want_uv=False)
    q = bench.diag_quality(np.abs(np.diag(T)), synthetic.spectrum("gap", n), b)
    assert q["Tii_over_sigma_first_block_max_dev"] <= 1e-13
    assert q["Tii_over_sigma_median_abs_dev"] <= 0.1

"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks one oracle routine against something other than itself: a
library implementation of the same definition (numpy Philox, LAPACK dgeqrf /
dgeqrt, LAPACK SVD), a closed form, an invariant of the UTV factorization
(Sec. 1.1 and 3.1: A = U T V^T, T upper triangular, U and V orthogonal) or a
special case that reduces to a textbook routine.  No GPU needed.
"""
import os

import numpy as np
import pytest
import scipy.linalg.lapack as lapack
import scipy.stats

import oracle
import synthetic
from conftest import EPS, utv_bound

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- Philox
def _numpy_philox_block(counter, key):
    """numpy's Philox4x64-10 pre-increments the 256-bit counter: feed counter-1."""
    c = sum(int(x) << (64 * i) for i, x in enumerate(counter))
    c = (c - 1) % (1 << 256)
    cp = np.array([(c >> (64 * i)) & (2 ** 64 - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=cp)
    return bg.random_raw(4)


def test_philox_known_answer():
    with open(os.path.join(GOLDEN, "philox4x64_10_kat.txt")) as f:
        rows = [line.split() for line in f if line.strip() and not line.startswith("#")]
    for row in rows:
        ctr = [int(x) for x in row[:4]]
        key = [int(x) for x in row[4:6]]
        want = [int(x, 16) for x in row[6:10]]
        got = oracle.philox4x64_10(ctr, key)
        assert [int(x) for x in got] == want


@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((5, 7, 3, 0), (123456789, 0)),
    ((2 ** 64 - 1,) * 4, (2 ** 64 - 1, 2 ** 64 - 1)),
    ((17, 3, 250, 0), (0xDEADBEEF, 0)),
])
def test_philox_matches_numpy(ctr, key):
    assert (oracle.philox4x64_10(ctr, key) == _numpy_philox_block(ctr, key)).all()


def test_gaussian_is_standard_normal_and_independent():
    G = oracle.gaussian(7, 3, 4001, 64)
    x = G.ravel()
    assert abs(x.mean()) < 5.0 / np.sqrt(x.size)
    assert abs(x.var() - 1.0) < 8.0 * np.sqrt(2.0 / x.size)
    assert scipy.stats.kstest(x, "norm").pvalue > 1e-3
    # different steps, seeds and columns give uncorrelated draws
    G2 = oracle.gaussian(7, 4, 4001, 64)
    G3 = oracle.gaussian(8, 3, 4001, 64)
    for other in (G2, G3):
        c = np.corrcoef(G.ravel(), other.ravel())[0, 1]
        assert abs(c) < 5.0 / np.sqrt(x.size)
    cc = np.corrcoef(G.T)
    off = cc - np.diag(np.diag(cc))
    assert np.abs(off).max() < 6.0 / np.sqrt(G.shape[0])


def test_gaussian_prefix_consistent():
    """G(r, c) depends on (seed, step, r, c) only, not on the requested shape."""
    big = oracle.gaussian(3, 2, 103, 9)
    small = oracle.gaussian(3, 2, 50, 4)
    assert np.array_equal(big[:50, :4], small)


# --------------------------------------------------------------------------- HQR
@pytest.mark.parametrize("shape,seed", [((50, 20), 0), ((20, 20), 1), ((7, 1), 2), ((300, 64), 3)])
def test_householder_qr_matches_lapack(shape, seed):
    A = np.random.default_rng(seed).standard_normal(shape)
    R, tau = oracle.householder_qr(A)
    ref, tau_ref, _, info = lapack.dgeqrf(A)
    assert info == 0
    scale = np.abs(A).max()
    assert np.abs(R - ref).max() <= 200 * EPS * scale * shape[0]
    assert np.abs(tau - tau_ref).max() <= 200 * EPS * shape[0]


def test_householder_zero_subcolumn_and_signs():
    # column 0 already upper triangular -> tau = 0, R(0,0) unchanged (dlarfg rule)
    A = np.array([[3.0, 1.0], [0.0, 2.0], [0.0, 5.0]])
    R, tau = oracle.householder_qr(A)
    assert tau[0] == 0.0 and R[0, 0] == 3.0
    # column 1: alpha = 2 > 0 -> beta = -hypot(2, 5)
    assert np.isclose(R[1, 1], -np.hypot(2.0, 5.0))
    # alpha < 0 -> beta > 0
    R2, _ = oracle.householder_qr(np.array([[-1.0], [1.0]]))
    assert np.isclose(R2[0, 0], np.sqrt(2.0))


def _explicit_q(W, tau):
    M, k = W.shape
    Q = np.eye(M)
    for j in range(k):
        Q = Q @ (np.eye(M) - tau[j] * np.outer(W[:, j], W[:, j]))
    return Q


@pytest.mark.parametrize("shape,seed", [((40, 12), 0), ((12, 12), 4), ((200, 32), 5)])
def test_larft_matches_lapack_and_explicit_product(shape, seed):
    A = np.random.default_rng(seed).standard_normal(shape)
    M, k = shape
    R, tau = oracle.householder_qr(A)
    W = np.tril(R, -1)[:, :k] + np.eye(M, k)
    Tf = oracle.larft(W, tau)
    _, t_ref, info = lapack.dgeqrt(k, A)
    assert info == 0
    assert np.abs(Tf - t_ref).max() <= 1e-12
    assert np.allclose(np.tril(Tf, -1), 0.0)
    Q = _explicit_q(W, tau)
    assert np.abs((np.eye(M) - W @ Tf @ W.T) - Q).max() <= 1e-13
    # Q^T A = [R; 0]
    QtA = Q.T @ A
    assert np.abs(np.triu(QtA[:k]) - np.triu(R[:k])).max() <= 1e-12
    if M > k:
        assert np.abs(QtA[k:]).max() <= 1e-12


# --------------------------------------------------------------------------- Jacobi SVD
@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (17, 2), (64, 3)])
def test_jacobi_svd_random(n, seed):
    R = np.triu(np.random.default_rng(seed).standard_normal((n, n)))
    D, Us, Vs, sweeps, rc = oracle.jacobi_svd(R)
    assert rc == 0
    s_ref = np.linalg.svd(R, compute_uv=False)
    assert np.abs(D - s_ref).max() <= 50 * n * EPS * s_ref[0]
    assert np.all(np.diff(D) <= 0)
    assert np.abs(Us @ np.diag(D) @ Vs.T - R).max() <= 50 * n * EPS * s_ref[0]
    assert np.abs(Us.T @ Us - np.eye(n)).max() <= 50 * n * EPS
    assert np.abs(Vs.T @ Vs - np.eye(n)).max() <= 50 * n * EPS
    for j in range(n):  # canonical sign
        i = np.argmax(np.abs(Vs[:, j]))
        assert Vs[i, j] > 0


def test_jacobi_svd_diagonal_closed_form():
    d = np.array([0.5, -3.0, 2.0, 1e-9])
    D, Us, Vs, sweeps, rc = oracle.jacobi_svd(np.diag(d))
    assert rc == 0 and sweeps == 1
    assert np.array_equal(D, np.array([3.0, 2.0, 0.5, 1e-9]))
    P = np.zeros((4, 4))
    P[1, 0] = P[2, 1] = P[0, 2] = P[3, 3] = 1.0
    assert np.array_equal(Vs, P)
    assert np.array_equal(Us, P * np.sign(d)[:, None])


def test_jacobi_svd_rank_deficient_completes_u():
    R = np.zeros((3, 3))
    R[0, 0] = 2.0
    R[0, 2] = 1.0
    D, Us, Vs, _, rc = oracle.jacobi_svd(R)
    assert rc == 0
    assert np.isclose(D[0], np.sqrt(5.0)) and D[1] == 0.0 and D[2] == 0.0
    assert np.abs(Us.T @ Us - np.eye(3)).max() < 1e-15
    assert np.abs(Us @ np.diag(D) @ Vs.T - R).max() < 1e-15


def test_jacobi_svd_sweep_cap_reports_status():
    R = np.triu(np.random.default_rng(0).standard_normal((16, 16)))
    *_, sweeps, rc = oracle.jacobi_svd(R, max_sweeps=1)
    assert rc == 1 and sweeps == 1


# --------------------------------------------------------------------------- randUTV
def _check_utv(A, U, T, V, triangular=True):
    m, n = A.shape
    nrm = np.linalg.norm(A)
    bound = utv_bound(n)
    assert np.linalg.norm(A - U @ T @ V.T) / nrm <= bound
    assert np.linalg.norm(U.T @ U - np.eye(m)) <= utv_bound(m)
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= bound
    if triangular:
        assert np.array_equal(np.tril(T, -1), np.zeros_like(T))  # exact zeros
    # unitary invariance of the Frobenius norm
    assert abs(np.linalg.norm(T) - nrm) <= bound * nrm


@pytest.mark.parametrize("m,n,b,q,kind", [
    (64, 64, 16, 0, "normal"),
    (64, 64, 16, 1, "geometric10"),
    (96, 40, 16, 2, "geometric10"),   # tall, b does not divide n
    (128, 64, 24, 3, "gap"),          # m = 2n, final block of 16
    (50, 50, 7, 1, "normal"),
    (33, 33, 64, 1, "normal"),        # b >= n: one final block
])
def test_randutv_brute_force_small(m, n, b, q, kind):
    A = synthetic.test_matrix(m, n, kind, 11, 12)
    U, T, V, rc = oracle.randutv(A, b, q, seed=5)
    assert rc == 0
    _check_utv(A, U, T, V)
    s = np.linalg.svd(A, compute_uv=False)
    d = np.diag(T)
    # every diagonal block is nonnegative and descending (its SVD)
    for k0 in range(0, n, b):
        blk = d[k0:k0 + b]
        assert np.all(blk >= 0) and np.all(np.diff(blk) <= 0)
    # interlacing for the first block: T_jj <= sigma_j(A)
    w = min(b, n)
    assert np.all(d[:w] <= s[:w] * (1 + 1e-12))
    # |det A| = prod |T_ii| for square A
    if m == n:
        assert abs(np.sum(np.log10(d)) - np.sum(np.log10(s))) <= 1e-6 * n


def test_randutv_b_ge_n_gives_singular_values():
    A = synthetic.test_matrix(40, 30, "geometric10", 3, 4)
    U, T, V, rc = oracle.randutv(A, 30, 2, seed=1)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.abs(np.diag(T) - s).max() <= 1e-14
    assert np.abs(np.triu(T, 1)).max() <= 1e-14 * s[0]
    _check_utv(A, U, T, V)


@pytest.mark.parametrize("kind", ["normal", "geometric10"])
def test_randutv_step0_matches_sketch_subspace(kind):
    """After step 0, V(:, 0:b) spans Y = (A^T A)^q A^T G and T_11 = sigma(A Q1).

    The subspace of Y is determined to about eps * cond(Y), which sets the tolerance.
    """
    m, n, b, q, seed = 80, 60, 12, 2, 9
    A = synthetic.test_matrix(m, n, kind, 1, 2)
    U, T, V, _ = oracle.randutv(A, b, q, seed, stop_after=1)
    G = oracle.gaussian(seed, 0, m, b)
    Y = A.T @ G
    for _ in range(q):
        Y = A.T @ (A @ Y)
    Q1 = np.linalg.qr(Y)[0]
    # span equality: projector difference
    P1 = Q1 @ Q1.T
    P2 = V[:, :b] @ V[:, :b].T
    tol = 100 * EPS * np.linalg.cond(Y)
    assert np.abs(P1 - P2).max() <= tol
    s1 = np.linalg.svd(A @ Q1, compute_uv=False)
    assert np.abs(np.diag(T)[:b] - s1).max() <= max(tol, 1e-13) * s1[0]
    # partial factorization is still exact
    _check_utv(A, U, T, V, triangular=False)
    assert np.abs(np.tril(T[:, :b], -1)).max() == 0.0


def test_randutv_power_iteration_sharpens_gap_spectrum():
    n, b = 120, 12
    A = synthetic.test_matrix(n, n, "gap", 5, 6)
    s = np.linalg.svd(A, compute_uv=False)
    ratios = []
    for q in (0, 2):
        _, T, _, _ = oracle.randutv(A, b, q, seed=2, want_uv=False)
        ratios.append(np.diag(T)[:b] / s[:b])
    # sigma = 1 repeated over the first block: q = 2 recovers it to ~1e-12
    assert np.abs(ratios[1] - 1).max() < 1e-8
    assert np.abs(ratios[1] - 1).max() <= np.abs(ratios[0] - 1).max()


def test_randutv_rank_deficient():
    n, k, b = 64, 16, 8
    rng = np.random.default_rng(3)
    A = rng.standard_normal((n, k)) @ rng.standard_normal((k, n))
    U, T, V, rc = oracle.randutv(A, b, 1, seed=4)
    assert rc == 0
    d = np.diag(T)
    assert np.all(d[k:] <= 1e-12 * np.linalg.norm(A))
    assert np.all(d[:k] > 1e-3)
    _check_utv(A, U, T, V)


def test_randutv_t_only_mode_matches():
    A = synthetic.test_matrix(70, 50, "normal", 7, 0)
    _, T1, _, _ = oracle.randutv(A, 16, 1, seed=3)
    U, T2, V, _ = oracle.randutv(A, 16, 1, seed=3, want_uv=False)
    assert U is None and V is None
    assert np.array_equal(T1, T2)


@pytest.mark.parametrize("m,n,b,q,kind", [
    (300, 100, 16, 1, "geometric10"),   # m = 3n, b does not divide n
    (160, 40, 12, 2, "normal"),          # m = 4n
    (64, 64, 16, 1, "normal"),           # square: the QR is of a square matrix
    (90, 30, 40, 1, "normal"),           # b >= n: the SVD of R
])
def test_randutv_qrfirst_against_lapack_qr_and_identities(m, n, b, q, kind):
    """QR first (Sec. 5.1): T must be [T_R; 0] where T_R is randUTV of the R
    factor of A, here taken from LAPACK's dgeqrf (an independent QR with the
    same sign rule), and (U, T, V) must be a UTV factorization of A."""
    from scipy.linalg import lapack

    A = synthetic.test_matrix(m, n, kind, 21, 22)
    nrm = np.linalg.norm(A)
    U, T, V, rc = oracle.randutv_qrfirst(A, b, q, seed=3)
    assert rc == 0
    _check_utv(A, U, T, V)
    qr, _, _, info = lapack.dgeqrf(np.asfortranarray(A))
    assert info == 0
    R = np.triu(qr[:n, :n])
    UR, TR, VR, _ = oracle.randutv(R, b, q, 3)
    assert np.abs(T[:n] - TR).max() <= 1e-10 * nrm
    assert np.array_equal(T[n:], np.zeros((m - n, n)))
    assert np.abs(T @ V.T - np.vstack([TR @ VR.T, np.zeros((m - n, n))])).max() <= 1e-10 * nrm
    # U^T A = T V^T by definition of the factorization
    assert np.abs(U.T @ A - T @ V.T).max() <= 50 * m * EPS * nrm
    if b >= n:
        s = np.linalg.svd(A, compute_uv=False)
        assert np.abs(np.diag(T) - s).max() <= 1e-13 * s[0]


def test_randutv_qrfirst_t_only_and_stop():
    A = synthetic.test_matrix(200, 60, "normal", 5, 6)
    U, T, V, _ = oracle.randutv_qrfirst(A, 16, 1, seed=2, want_uv=False)
    assert U is None and V is None
    _, T2, _, _ = oracle.randutv_qrfirst(A, 16, 1, seed=2)
    assert np.array_equal(T, T2)
    U, T, V, _ = oracle.randutv_qrfirst(A, 16, 1, seed=2, stop_after=2)
    _check_utv(A, U, T, V, triangular=False)
    assert np.array_equal(np.tril(T[:, :32], -1), np.zeros((200, 32)))
    with pytest.raises(ValueError):
        oracle.randutv_qrfirst(np.zeros((3, 5)), 2, 1, 0)


def test_randutv_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.randutv(np.zeros((3, 5)), 2, 1, 0)  # m < n
    with pytest.raises(ValueError):
        oracle.randutv(np.zeros((5, 3)), 0, 1, 0)  # b < 1
    with pytest.raises(ValueError):
        oracle.randutv(np.zeros((5, 3)), 2, -1, 0)  # q < 0


def test_randutv_empty():
    U, T, V, rc = oracle.randutv(np.zeros((4, 0)), 2, 1, 0)
    assert rc == 0 and T.shape == (4, 0)
    assert np.array_equal(U, np.eye(4))


@pytest.mark.slow
def test_randutv_config1_invariants():
    """1000 x 1000, sigma_i = 10^(-10 (i-1)/999), b = 64, q = 1, seed 0."""
    A = synthetic.test_matrix(1000, 1000, "geometric10", 1, 2)
    U, T, V, rc = oracle.randutv(A, 64, 1, seed=0)
    assert rc == 0
    _check_utv(A, U, T, V)
    d = np.diag(T)
    # prod sigma_i = 10^-5000 exactly for this spectrum
    assert abs(np.sum(np.log10(d)) + 5000.0) < 1e-2
    s = synthetic.spectrum("geometric10", 1000)
    assert np.all(d[:64] <= s[:64] * (1 + 1e-9))
    assert np.median(np.abs(d / s - 1)) < 0.2

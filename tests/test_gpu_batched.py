"""Batched randUTV (one persistent, graph-captured launch over many matrices)
against the CPU oracle and the single-matrix path."""
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
    return X.t().contiguous().cpu().numpy().T


def make_batch(shapes, kind="geometric8"):
    mats = []
    for k, (m, n) in enumerate(shapes):
        mats.append(synthetic.test_matrix(m, n, kind if n > 1 else "normal", 100 + k, 200 + k))
    return mats


def run_batch(rutv, mats, b, q, prec=0, seeds=None, table=None, want_uv=True):
    A = [dev(M) for M in mats]
    T = [rutv.colmajor_empty(M.shape[0], M.shape[1]) for M in mats]
    U = [rutv.colmajor_empty(M.shape[0], M.shape[0]) for M in mats] if want_uv else None
    V = [rutv.colmajor_empty(M.shape[1], M.shape[1]) for M in mats] if want_uv else None
    seeds = seeds if seeds is not None else list(range(len(mats)))
    tab = table if table is not None else "0 100000 -1 %d" % b
    status = [0] * len(mats)
    r = rutv.randutv_batched([M.shape[0] for M in mats], [M.shape[1] for M in mats], A,
                             [M.shape[0] for M in mats], U, T, V, seeds, q, prec, tab, status)
    torch.cuda.synchronize()
    return r, status, [host(x) for x in U] if U else None, [host(x) for x in T], [host(x) for x in V] if V else None


SHAPES = [(40, 40), (96, 48), (130, 130), (64, 64), (33, 17), (200, 100), (150, 150), (17, 17), (8, 3), (256, 128),
          (100, 100), (70, 35)]


@pytest.mark.parametrize("b", [16, 32])
def test_batched_matches_oracle(rutv, b):
    """Entrywise parity needs a sketch that rounding does not decide: with
    q = 2 the condition number of Y grows like (sigma_1 / sigma_b)^5 within a
    block, so the parity batch uses i.i.d. Gaussian matrices (well separated
    singular values); the steep 1e-8 workload spectrum is covered by
    test_batched_workload_spectrum_invariants."""
    mats = make_batch(SHAPES, kind="normal")
    r, status, U, T, V = run_batch(rutv, mats, b, 2)
    assert r == rutv.RANDUTV_OK and all(s == 0 for s in status)
    for k, A in enumerate(mats):
        Uo, To, Vo, _ = oracle.randutv(A, b, 2, k)
        nrm = np.linalg.norm(A)
        assert np.abs(T[k] - To).max() <= 1e-10 * nrm, k
        assert np.abs(U[k] @ T[k] - Uo @ To).max() <= 1e-10 * nrm, k
        assert np.abs(T[k] @ V[k].T - To @ Vo.T).max() <= 1e-10 * nrm, k
        m, n = A.shape
        assert np.linalg.norm(A - U[k] @ T[k] @ V[k].T) / nrm <= utv_bound(n)
        assert np.linalg.norm(U[k].T @ U[k] - np.eye(m)) <= utv_bound(m)
        assert np.array_equal(np.tril(T[k], -1), np.zeros_like(T[k]))


def test_batched_workload_spectrum_invariants(rutv):
    mats = make_batch(SHAPES, kind="geometric8")
    r, status, U, T, V = run_batch(rutv, mats, 16, 2)
    assert r == rutv.RANDUTV_OK
    for k, A in enumerate(mats):
        m, n = A.shape
        nrm = np.linalg.norm(A)
        assert np.linalg.norm(A - U[k] @ T[k] @ V[k].T) / nrm <= utv_bound(n)
        assert np.linalg.norm(U[k].T @ U[k] - np.eye(m)) <= utv_bound(m)
        assert np.linalg.norm(V[k].T @ V[k] - np.eye(n)) <= utv_bound(n)
        assert np.array_equal(np.tril(T[k], -1), np.zeros_like(T[k]))
        d = np.diag(T[k])
        for k0 in range(0, n, 16):
            assert np.all(np.diff(d[k0:k0 + 16]) <= 0) and np.all(d >= 0)
        if m == n:
            s = np.linalg.svd(A, compute_uv=False)
            assert abs(np.sum(np.log10(d)) - np.sum(np.log10(s))) <= 1e-3 * n


def test_batched_matches_single_path(rutv):
    mats = make_batch([(300, 200), (180, 180), (64, 32)])
    _, _, _, T, _ = run_batch(rutv, mats, 32, 1, seeds=[5, 6, 7])
    for k, A in enumerate(mats):
        _, Ts, _ = rutv.factor(dev(A), 32, 1, 5 + k)
        torch.cuda.synchronize()
        assert np.abs(T[k] - host(Ts)).max() <= 1e-10 * np.linalg.norm(A)


def test_batched_t_only_and_status(rutv):
    mats = make_batch([(50, 50), (60, 40), (80, 80)])
    mats[1][3, 4] = np.nan
    r, status, U, T, V = run_batch(rutv, mats, 16, 1, want_uv=False)
    assert status[1] == rutv.RANDUTV_ENONFINITE
    assert status[0] == 0 and status[2] == 0
    assert r == rutv.RANDUTV_ENONFINITE
    _, To, _, _ = oracle.randutv(mats[2], 16, 1, 2, want_uv=False)
    assert np.abs(T[2] - To).max() <= 1e-10 * np.linalg.norm(mats[2])


def test_batched_plan_replay_deterministic(rutv):
    mats = make_batch([(120, 60), (90, 90), (256, 256), (40, 20)])
    A = [dev(M) for M in mats]
    T = [rutv.colmajor_empty(*M.shape) for M in mats]
    plan = rutv.BatchPlan([M.shape[0] for M in mats], [M.shape[1] for M in mats], A, [M.shape[0] for M in mats],
                          None, T, None, [1, 2, 3, 4], 2, 0, "0 100000 -1 32")
    r1, s1 = plan.run()
    T1 = [host(x) for x in T]
    r2, s2 = plan.run()
    T2 = [host(x) for x in T]
    plan.close()
    assert r1 == r2 == 0
    for x, y in zip(T1, T2):
        assert np.array_equal(x, y)


def test_batched_fp32_sketch_quality(rutv):
    mats = make_batch([(256, 256), (300, 150), (128, 128)], kind="geometric8")
    _, _, U, T, V = run_batch(rutv, mats, 32, 2, prec=rutv.RANDUTV_SKETCH_FP32)
    _, _, _, T64, _ = run_batch(rutv, mats, 32, 2, prec=rutv.RANDUTV_FP64)
    for k, A in enumerate(mats):
        m, n = A.shape
        nrm = np.linalg.norm(A)
        assert np.linalg.norm(A - U[k] @ T[k] @ V[k].T) / nrm <= utv_bound(n)
        assert np.linalg.norm(V[k].T @ V[k] - np.eye(n)) <= utv_bound(n)
        s = np.linalg.svd(A, compute_uv=False)
        keep = s > 1e3 * 2.0 ** -53 * s[0]
        dev_ = np.abs((np.diag(T[k])[keep] / s[keep]) / (np.diag(T64[k])[keep] / s[keep]) - 1)
        assert dev_.max() <= 0.05


def test_batched_autotune_table(rutv):
    mats = make_batch([(40, 40), (80, 40), (200, 200)])
    A = [dev(M) for M in mats]
    T = [rutv.colmajor_empty(*M.shape) for M in mats]
    r, table = rutv.randutv_batched_autotune([M.shape[0] for M in mats], [M.shape[1] for M in mats], A,
                                             [M.shape[0] for M in mats], None, T, None, [0, 1, 2], 1)
    assert r == 0
    lines = table.strip().splitlines()
    assert lines[-1] in ("threads 128", "threads 256")
    rows = [list(map(int, line.split())) for line in lines[:-1]]
    assert len(rows) == 3 and all(row[3] in (16, 32, 64) and row[4] in (32, 64) for row in rows)
    # the table drives a run
    r2, status, _, T2, _ = run_batch(rutv, mats, 0, 1, table=table, want_uv=False)
    assert r2 == 0


def _check_against_oracle(mats, b_of, q, U, T, V, seeds):
    for k, A in enumerate(mats):
        Uo, To, Vo, rc = oracle.randutv(A, b_of(k), q, seeds[k])
        assert rc == 0
        nrm = np.linalg.norm(A)
        m, n = A.shape
        assert np.abs(T[k] - To).max() <= 1e-10 * nrm, (k, A.shape)
        assert np.abs(U[k] @ T[k] - Uo @ To).max() <= 1e-10 * nrm, (k, A.shape)
        assert np.abs(T[k] @ V[k].T - To @ Vo.T).max() <= 1e-10 * nrm, (k, A.shape)
        assert np.linalg.norm(A - U[k] @ T[k] @ V[k].T) / nrm <= utv_bound(n)
        assert np.linalg.norm(U[k].T @ U[k] - np.eye(m)) <= utv_bound(m)
        assert np.linalg.norm(V[k].T @ V[k] - np.eye(n)) <= utv_bound(n)
        assert np.array_equal(np.tril(T[k], -1), np.zeros_like(T[k]))


def test_batched_b64_large_and_tall_match_oracle(rutv):
    """b = 64 (the block size the autotuner picks from n = 256 up) on the
    largest square size of the workload (512), a ragged 300, and tall
    m = 2n matrices up to 1024 x 512, each against the oracle."""
    shapes = [(300, 300), (512, 512), (600, 300), (1024, 512), (520, 260), (384, 192)]
    mats = make_batch(shapes, kind="normal")
    seeds = [11 + k for k in range(len(mats))]
    r, status, U, T, V = run_batch(rutv, mats, 64, 2, seeds=seeds)
    assert r == rutv.RANDUTV_OK and all(s == 0 for s in status)
    _check_against_oracle(mats, lambda k: 64, 2, U, T, V, seeds)


def test_batched_autotuned_workload_slice_matches_oracle(rutv):
    """The autotuner's table, run on a 32-matrix slice of the 4096-matrix
    workload's shapes (n log-uniform in [32, 512], 25% with m = 2n), with the
    block size the table picks for each matrix, against the oracle."""
    import bench

    ms, ns = bench.batched_shapes(4096)
    shapes = list(zip(ms, ns))[:32]
    mats = make_batch(shapes, kind="normal")
    seeds = list(range(100, 100 + len(mats)))
    A = [dev(M) for M in mats]
    T0 = [rutv.colmajor_empty(*M.shape) for M in mats]
    r, table = rutv.randutv_batched_autotune([M.shape[0] for M in mats], [M.shape[1] for M in mats], A,
                                             [M.shape[0] for M in mats], None, T0, None, seeds, 2)
    assert r == 0
    lines = table.strip().splitlines()
    assert lines[-1].startswith("threads ")
    rows = [tuple(map(int, line.split())) for line in lines[:-1]]
    assert rows and all(row[3] in (16, 32, 64) and row[4] in (32, 64) for row in rows)

    def b_of(k):
        m, n = mats[k].shape
        tall = 1 if m > n else 0
        hits = [row[3] for row in rows if row[0] <= n <= row[1] and row[2] in (tall, -1)]
        assert hits, (m, n, table)
        return hits[0]

    r, status, U, T, V = run_batch(rutv, mats, 0, 2, seeds=seeds, table=table)
    assert r == rutv.RANDUTV_OK and all(s == 0 for s in status)
    _check_against_oracle(mats, b_of, 2, U, T, V, seeds)


@pytest.mark.parametrize("threads,tile", [(128, 32), (128, 64), (256, 32), (256, 64)])
def test_batched_threads_and_tiles_match_oracle(rutv, threads, tile):
    """Every shape the autotuner can pick (threads per matrix, GEMM tile)
    computes the same factorization as the oracle."""
    shapes = [(96, 48), (130, 130), (33, 17), (200, 100), (300, 300), (70, 35)]
    mats = make_batch(shapes, kind="normal")
    seeds = [40 + k for k in range(len(mats))]
    table = "0 100000 -1 32 %d\nthreads %d\n" % (tile, threads)
    r, status, U, T, V = run_batch(rutv, mats, 0, 2, seeds=seeds, table=table)
    assert r == rutv.RANDUTV_OK and all(s == 0 for s in status)
    _check_against_oracle(mats, lambda k: 32, 2, U, T, V, seeds)

"""randutv_factor_opt against the oracle: the tolerance-driven stop and resume
of a partial factorization (early termination, Sec. 1.1 and Sec. 3.2) and
randUTV with a QR first for tall inputs (Sec. 5.1).  Needs a GB300."""
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


def check_parity(A, got, want, tol=1e-10):
    Ug, Tg, Vg = got
    Uo, To, Vo = want
    nrm = np.linalg.norm(A)
    assert np.abs(Tg - To).max() <= tol * nrm
    if Uo is not None and Ug is not None:
        assert np.abs(Ug @ Tg - Uo @ To).max() <= tol * nrm
        assert np.abs(Tg @ Vg.T - To @ Vo.T).max() <= tol * nrm


def check_utv(A, U, T, V):
    m, n = A.shape
    nrm = np.linalg.norm(A)
    assert np.linalg.norm(A - U @ T @ V.T) / nrm <= utv_bound(n)
    assert np.linalg.norm(U.T @ U - np.eye(m)) <= utv_bound(m)
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= utv_bound(n)


PRECS = ["RANDUTV_FP64", "RANDUTV_FP64_EMULATED"]


@pytest.mark.parametrize("prec_name", PRECS)
@pytest.mark.parametrize("m,n,b,q,parts", [
    (400, 300, 40, 1, [3]),          # stop after 3 steps, resume to the end
    (640, 512, 128, 2, [1, 2]),      # three calls: 1 step, 2 steps, the rest (emulated products run)
    (1024, 1024, 64, 1, [5]),        # geometric decay of 10^-0.63 per block
    (333, 200, 48, 1, [4]),          # the resumed call has only the ragged final block left
])
def test_resume_equals_uninterrupted(rutv, prec_name, m, n, b, q, parts):
    prec = getattr(rutv, prec_name)
    # entrywise parity needs a sketch that rounding does not decide: N(0,1)
    # entries at b = 128 (the geometric spectrum falls 10^-2.5 per block of 128
    # at n = 512, which makes the q = 2 sketch's condition number ~1e12)
    kind = "normal" if b >= 128 else "geometric10"
    A = synthetic.test_matrix(m, n, kind, 70, 71)
    seed = 5
    U, T, V, cols, _ = rutv.factor_opt(dev(A), b, q, seed, prec=prec, stop_after=parts[0])
    assert cols == min(n, parts[0] * b)
    for extra in parts[1:]:
        cols2, _ = rutv.resume(U, T, V, b, q, seed, cols, prec=prec, stop_after=extra)
        assert cols2 == min(n, cols + extra * b)
        cols = cols2
    cols_end, rank = rutv.resume(U, T, V, b, q, seed, cols, prec=prec)
    assert cols_end == n and rank == n
    torch.cuda.synchronize()
    got = (host(U), host(T), host(V))
    check_utv(A, *got)
    assert np.array_equal(np.tril(got[1], -1), np.zeros_like(got[1]))
    check_parity(A, got, oracle.randutv(A, b, q, seed)[:3])
    # and equal to one uninterrupted call of the library
    Uf, Tf, Vf = rutv.factor(dev(A), b, q, seed, prec=prec)
    torch.cuda.synchronize()
    check_parity(A, got, (host(Uf), host(Tf), host(Vf)))


def _expected_stop(To, b, tol):
    """First block step whose smallest diagonal entry is <= tol |T_00| (from
    the oracle's complete factorization), as (columns done, rank count)."""
    d = np.abs(np.diag(To))
    n = d.size
    for k0 in range(0, n, b):
        blk = d[k0:k0 + b]
        if blk.min() <= tol * d[0]:
            cols = min(n, k0 + b)
            return cols, int((d[:cols] > tol * d[0]).sum())
    return n, int((d > tol * d[0]).sum())


@pytest.mark.parametrize("prec_name", PRECS)
@pytest.mark.parametrize("case", ["rank100", "geometric"])
def test_rank_tolerance_stop(rutv, prec_name, case):
    prec = getattr(rutv, prec_name)
    rng = np.random.default_rng(7)
    if case == "rank100":     # exact rank 100: the third block of 40 holds the boundary
        m, n, b, q, tol = 300, 260, 40, 1, 1e-10
        A = np.asfortranarray(rng.standard_normal((m, 100)) @ rng.standard_normal((100, n)))
    else:                     # sigma_i = 10^(-10 (i-1)/(n-1)): crosses 1e-5 halfway, 10^-0.63 per block
        m, n, b, q, tol = 1024, 1024, 64, 1, 1e-5
        A = synthetic.test_matrix(m, n, "geometric10", 72, 73)
    seed = 3
    _, To_full, _, _ = oracle.randutv(A, b, q, seed, want_uv=False)
    cols_want, rank_want = _expected_stop(To_full, b, tol)
    assert cols_want < n
    U, T, V, cols, rank = rutv.factor_opt(dev(A), b, q, seed, prec=prec, rank_tol=tol)
    torch.cuda.synchronize()
    assert cols == cols_want and rank == rank_want
    got = (host(U), host(T), host(V))
    check_utv(A, *got)
    assert np.array_equal(np.tril(got[1][:, :cols], -1), np.zeros((m, cols)))
    check_parity(A, got, oracle.randutv(A, b, q, seed, stop_after=cols // b)[:3])
    # a resume from there completes the same factorization as one call
    cols_end, _ = rutv.resume(U, T, V, b, q, seed, cols, prec=prec)
    torch.cuda.synchronize()
    assert cols_end == n
    check_parity(A, (host(U), host(T), host(V)), oracle.randutv(A, b, q, seed)[:3])


@pytest.mark.parametrize("prec_name", PRECS)
@pytest.mark.parametrize("m,n,b,q,kind", [
    (1200, 300, 64, 1, "geometric10"),   # m = 4n
    (900, 300, 128, 2, "normal"),        # m = 3n, b = 128 (emulated products run)
    (333, 200, 48, 1, "geometric10"),    # ragged panels and final block
    (256, 40, 64, 1, "normal"),          # b >= n: one panel, the SVD of R
])
def test_qr_first_matches_oracle(rutv, prec_name, m, n, b, q, kind):
    prec = getattr(rutv, prec_name)
    A = synthetic.test_matrix(m, n, kind, 74, 75)
    seed = 9
    U, T, V, cols, _ = rutv.factor_opt(dev(A), b, q, seed, prec=prec, qr_first=True)
    torch.cuda.synchronize()
    assert cols == n
    got = (host(U), host(T), host(V))
    check_utv(A, *got)
    assert np.array_equal(np.tril(got[1], -1), np.zeros_like(got[1]))
    check_parity(A, got, oracle.randutv_qrfirst(A, b, q, seed)[:3])


def test_qr_first_t_only_and_stop(rutv):
    A = synthetic.test_matrix(800, 200, "geometric10", 76, 77)
    _, T, _, _, _ = rutv.factor_opt(dev(A), 32, 1, 2, want_uv=False, qr_first=True)
    torch.cuda.synchronize()
    _, To, _, _ = oracle.randutv_qrfirst(A, 32, 1, 2, want_uv=False)
    assert np.abs(host(T) - To).max() <= 1e-10 * np.linalg.norm(A)
    U, T, V, cols, _ = rutv.factor_opt(dev(A), 32, 1, 2, qr_first=True, stop_after=2)
    torch.cuda.synchronize()
    assert cols == 64
    got = (host(U), host(T), host(V))
    check_utv(A, *got)
    check_parity(A, got, oracle.randutv_qrfirst(A, 32, 1, 2, stop_after=2)[:3])


def test_options_rejected_on_host(rutv):
    fake = 256
    bad = [rutv.randutv_options(start_col=30), rutv.randutv_options(start_col=64, qr_first=True),
           rutv.randutv_options(rank_tol=-1.0), rutv.randutv_options(start_col=400)]
    for o in bad:
        assert rutv.randutv_factor_opt(300, 200, fake, 300, 32, 1, 0, fake, fake, fake, o) == rutv.RANDUTV_EINVAL

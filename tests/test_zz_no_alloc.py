"""The allocation-free SVD entry point (randutv_svd_small_noalloc) against the
existing path and the CPU oracle.  Callers that cannot allocate device memory
(strict memory pools, allocation-free real-time code, plugins whose host owns
all memory) use it; its scratch is a fixed device array inside the library.

Two references:
  - randutv_factor on the same upper triangular w x w matrix with b >= w: that
    call runs the library's own Jacobi SVD on the block (its Householder panel
    leaves a triangular input unchanged), so T = diag(D), U = Us and V = Vs;
  - the oracle's one-sided Jacobi SVD (plain C, FP64), which shares no code
    with the library.
Both have the same canonical order and signs (descending D, the largest entry
of each column of Vs positive).  Orders up to the documented maximum
w = 256 run, including 128 < w <= 256 (the two-hundred-and-fifty-six-thread
variant of the kernel) and a padded leading dimension whose padding and
strictly lower triangle hold NaN, which must never be read.
Two calls in a row check that the shared scratch carries nothing over.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()


def host(X):
    return X.t().contiguous().cpu().numpy().T


@pytest.fixture(scope="module")
def rutv():
    import paper_2104_05782_gb300 as r
    from paper_2104_05782_gb300 import build
    build.build()
    r.load()
    return r


def reference(rutv, R):
    w = R.shape[0]
    U, T, V = rutv.factor(dev(R), w, 0, 0)
    torch.cuda.synchronize()
    return np.diag(host(T)), host(U), host(V)


def padded(R, ldr):
    """Column-major device copy of R with leading dimension ldr; the padding
    rows and the strictly lower triangle are NaN."""
    w = R.shape[0]
    big = np.full((ldr, w), np.nan)
    big[:w, :] = np.where(np.triu(np.ones((w, w))) > 0, R, np.nan)
    return torch.from_numpy(np.ascontiguousarray(big.T)).cuda().t()


def check_against(d, Uh, Vh, d_ref, U_ref, V_ref, nrm):
    assert np.abs(d - d_ref).max() <= 1e-10 * nrm
    assert np.abs(Uh * d - U_ref * d_ref).max() <= 1e-10 * nrm
    assert np.abs(d[:, None] * Vh.T - d_ref[:, None] * V_ref.T).max() <= 1e-10 * nrm


@pytest.mark.parametrize("w,ldr_pad,seed", [(128, 0, 1), (77, 0, 2), (256, 0, 3), (200, 0, 4), (150, 9, 5),
                                            (64, 3, 6)])
def test_noalloc_svd_matches_factor_and_oracle_twice(rutv, w, ldr_pad, seed):
    rng = np.random.default_rng(seed)
    for call in range(2):
        # diagonal entries kept away from zero so that the singular values are
        # well separated and every singular vector is determined
        R = np.triu(rng.standard_normal((w, w))) * 0.1 + np.diag(1.0 + rng.uniform(size=w)) * (1.0 + call)
        ldr = w + ldr_pad
        dR = padded(R, ldr) if ldr_pad else dev(R)
        D = torch.zeros(w, dtype=torch.float64, device="cuda")
        Us = rutv.colmajor_empty(w, w)
        Vs = rutv.colmajor_empty(w, w)
        st = rutv.randutv_svd_small_noalloc(w, dR, ldr, D, Us, Vs)
        assert st == rutv.RANDUTV_OK
        torch.cuda.synchronize()
        d, Uh, Vh = D.cpu().numpy(), host(Us), host(Vs)
        nrm = np.linalg.norm(R)
        check_against(d, Uh, Vh, *reference(rutv, R), nrm)
        d_o, U_o, V_o, _, rc = oracle.jacobi_svd(R)
        assert rc == 0
        check_against(d, Uh, Vh, d_o, U_o, V_o, nrm)
        assert np.abs(Uh @ np.diag(d) @ Vh.T - R).max() <= 1e-12 * nrm
        assert np.linalg.norm(Uh.T @ Uh - np.eye(w)) <= 50 * w * 2.0 ** -53
        assert np.linalg.norm(Vh.T @ Vh - np.eye(w)) <= 50 * w * 2.0 ** -53


def test_noalloc_rejects_too_large(rutv):
    w = 257
    assert rutv.randutv_svd_small_noalloc(w, 256, w, 256, 256, 256) == rutv.RANDUTV_EINVAL

"""Failure detection on the GPU without a fault: a bounded device wait that
gives up, and a Jacobi SVD that hits its sweep cap, each reported as a status
while the context stays usable.  The limits are lowered for the process with
randutv_set_limits and restored afterwards.  Needs a GB300."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rutv():
    import paper_2104_05782_gb300 as r
    from paper_2104_05782_gb300 import build
    build.build()
    r.load()
    yield r
    r.randutv_set_limits(0, 0)


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()


def host(X):
    return X.t().contiguous().cpu().numpy().T


def _still_usable(rutv):
    A = synthetic.test_matrix(200, 150, "geometric10", 3, 4)
    _, T, _ = rutv.factor(dev(A), 32, 1, 0)
    torch.cuda.synchronize()
    _, To, _, _ = oracle.randutv(A, 32, 1, 0, want_uv=False)
    assert np.abs(host(T) - To).max() <= 1e-10 * np.linalg.norm(A)


def test_grid_barrier_wait_gives_up(rutv):
    """One poll per grid barrier: blocks of the cooperative panel QR that
    arrive before the others give up at once, record the timeout and return;
    the call reports RANDUTV_ETIMEOUT instead of waiting."""
    m, n = 4000, 256
    A = synthetic.test_matrix(m, n, "normal", 5, 6)
    U, T, V = rutv.colmajor_empty(m, m), rutv.colmajor_empty(m, n), rutv.colmajor_empty(n, n)
    rutv.randutv_set_limits(1, 0)
    try:
        st = rutv.randutv_factor_ex(m, n, dev(A), m, 64, 1, 0, U, T, V)
    finally:
        rutv.randutv_set_limits(0, 0)
    assert st == rutv.RANDUTV_ETIMEOUT
    _still_usable(rutv)


def test_jacobi_sweep_cap_reports_noconv(rutv):
    """A sweep cap of one: the b x b Jacobi SVDs stop unconverged and the call
    reports RANDUTV_ENOCONV; so does the allocation-free SVD (the grid variant
    of the kernel)."""
    A = synthetic.test_matrix(200, 150, "normal", 7, 8)
    w = 96
    R = np.triu(np.random.default_rng(1).standard_normal((w, w)))
    D = torch.zeros(w, dtype=torch.float64, device="cuda")
    Us = rutv.colmajor_empty(w, w)
    Vs = rutv.colmajor_empty(w, w)
    rutv.randutv_set_limits(0, 1)
    try:
        T = rutv.colmajor_empty(200, 150)
        st = rutv.randutv_factor_ex(200, 150, dev(A), 200, 32, 1, 0, None, T, None)
        st_small = rutv.randutv_svd_small_noalloc(w, dev(R), w, D, Us, Vs)
    finally:
        rutv.randutv_set_limits(0, 0)
    assert st == rutv.RANDUTV_ENOCONV
    assert st_small == rutv.RANDUTV_ENOCONV
    _still_usable(rutv)

"""The allocation-free SVD entry point (randutv_svd_small_noalloc) against the
existing path.  Callers that cannot allocate device memory (strict memory
pools, allocation-free real-time code, plugins whose host owns all memory)
use it; its scratch is a fixed device array inside the library.

The reference is randutv_factor on the same upper triangular w x w matrix with
b >= w: that call runs the same Jacobi SVD on the block (its Householder panel
leaves a triangular input unchanged), so T = diag(D), U = Us and V = Vs.
Two calls in a row check that the shared scratch carries nothing over.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("w,seed", [(128, 1), (77, 2)])
def test_noalloc_svd_matches_factor_twice(rutv, w, seed):
    rng = np.random.default_rng(seed)
    for call in range(2):
        R = np.triu(rng.standard_normal((w, w))) * (1.0 + call)
        dR = dev(R)
        D = torch.zeros(w, dtype=torch.float64, device="cuda")
        Us = rutv.colmajor_empty(w, w)
        Vs = rutv.colmajor_empty(w, w)
        st = rutv.randutv_svd_small_noalloc(w, dR, w, D, Us, Vs)
        assert st == rutv.RANDUTV_OK
        d_ref, U_ref, V_ref = reference(rutv, R)
        nrm = np.linalg.norm(R)
        d = D.cpu().numpy()
        assert np.abs(d - d_ref).max() <= 1e-10 * nrm
        Uh, Vh = host(Us), host(Vs)
        assert np.abs(Uh * d - U_ref * d_ref).max() <= 1e-10 * nrm
        assert np.abs(d[:, None] * Vh.T - d_ref[:, None] * V_ref.T).max() <= 1e-10 * nrm
        assert np.abs(Uh @ np.diag(d) @ Vh.T - R).max() <= 1e-12 * nrm


def test_noalloc_rejects_too_large(rutv):
    w = 257
    assert rutv.randutv_svd_small_noalloc(w, 256, w, 256, 256, 256) == rutv.RANDUTV_EINVAL

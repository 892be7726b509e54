"""The full-size workload (16000 x 16000, gap spectrum, b = 128, q = 2, U and V
formed, FP64 emulated on the BF16 tensor cores), checked through properties
that hold at any size. Residual and orthogonality are taken on sampled
vectors, so no 16000^3 product is needed. Runs near the end (it holds the most
memory), before only the allocation-free entry point's test."""
import numpy as np
import pytest

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


def _colnorms(X):
    return X.pow(2).sum(dim=0).sqrt()


def test_full_size_emulated_factorization(rutv):
    n, b, q = 16000, 128, 2
    dev = torch.device("cuda", 0)
    A, sigma = synthetic.test_matrix_device(n, n, "gap", 1, 2, dev)
    U, T, V = rutv.factor(A, b, q, 0, prec=rutv.RANDUTV_FP64_EMULATED)
    torch.cuda.synchronize()
    bound = utv_bound(n)
    nrm = float(A.pow(2).sum().sqrt())
    # T upper triangular with exact zeros, and ||T||_F = ||A||_F (Sec. 3.1)
    assert int(torch.count_nonzero(torch.tril(T, -1))) == 0
    assert abs(float(T.pow(2).sum().sqrt()) - nrm) <= bound * nrm
    # A x = U T V^T x and U^T U x = x, V^T V x = x on sampled x
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    X = torch.randn(n, 4, generator=g, device=dev, dtype=torch.float64)
    xn = float(_colnorms(X).max())
    res = float(_colnorms(A @ X - U @ (T @ (V.t() @ X))).max())
    assert res <= bound * nrm * xn
    assert float(_colnorms(U.t() @ (U @ X) - X).max()) <= bound * xn
    assert float(_colnorms(V.t() @ (V @ X) - X).max()) <= bound * xn
    # the first block holds the sigma = 1 cluster exactly (Sec. 3.2.1 with q = 2)
    r = torch.diagonal(T).abs().cpu().numpy() / sigma
    assert np.abs(r[:b] - 1).max() <= 1e-10

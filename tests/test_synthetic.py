"""The seeded input generators: prescribed spectra, orthogonal factors and
layouts, on CPU. Both the oracle tests and the CUDA-path tests draw their
matrices here, so the recipe itself is pinned."""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")


def test_spectra_closed_forms():
    n = 101
    g10 = synthetic.spectrum("geometric10", n)
    assert g10[0] == 1.0 and np.isclose(g10[-1], 1e-10, rtol=1e-12)
    assert np.allclose(np.log10(g10), -10.0 * np.arange(n) / (n - 1), rtol=0, atol=1e-12)
    g8 = synthetic.spectrum("geometric8", n)
    assert np.isclose(g8[-1], 1e-8, rtol=1e-12)
    alg = synthetic.spectrum("algebraic", n)
    assert np.array_equal(alg, 1.0 / np.arange(1, n + 1))
    gap = synthetic.spectrum("gap", n)
    k = n // 10
    assert np.all(gap[:k] == 1.0)
    assert np.isclose(gap[k], 1e-3) and np.isclose(gap[-1], 1e-12)
    e32 = synthetic.spectrum("exp32", 1000)
    assert np.isclose(e32[32], 0.1, rtol=1e-12) and e32[-1] == 1e-15 and e32[479] > 1e-15
    e128 = synthetic.spectrum("exp128", n)
    assert np.allclose(np.log10(e128), -np.arange(n) / 128.0, rtol=0, atol=1e-12)
    for s in (g10, g8, alg, gap, e32, e128):
        assert np.all(np.diff(s) <= 0)
    with pytest.raises(ValueError):
        synthetic.spectrum("nope", 4)


@pytest.mark.parametrize("m,n,kind", [(60, 60, "geometric10"), (90, 45, "gap"), (40, 40, "algebraic"),
                                      (70, 50, "exp32")])
def test_small_matrix_has_the_prescribed_spectrum(m, n, kind):
    A = synthetic.test_matrix(m, n, kind, 3, 4)
    assert A.shape == (m, n) and A.flags["F_CONTIGUOUS"]
    s = np.linalg.svd(A, compute_uv=False)
    want = synthetic.spectrum(kind, n)
    assert np.abs(s - want).max() <= 100 * n * 2.0 ** -53
    assert np.array_equal(A, synthetic.test_matrix(m, n, kind, 3, 4))


def test_hartley_mix_is_orthogonal():
    n = 96
    gen = torch.Generator().manual_seed(5)
    Q = synthetic._hartley_mix(torch.eye(n, dtype=torch.float64), gen)
    assert torch.abs(Q.t() @ Q - torch.eye(n, dtype=torch.float64)).max() <= 50 * n * 2.0 ** -53
    # dense: every column mixes all rows
    assert int((Q.abs() > 0).sum()) > 0.9 * n * n


@pytest.mark.parametrize("m,n,kind", [(128, 128, "gap"), (160, 80, "geometric10")])
def test_large_recipe_has_the_prescribed_spectrum(m, n, kind):
    A, s = synthetic.test_matrix_device(m, n, kind, 1, 2, device="cpu")
    assert tuple(A.shape) == (m, n)
    assert A.stride() == (1, m)  # column-major: a transposed view of a row-major buffer
    got = np.linalg.svd(A.numpy(), compute_uv=False)
    assert np.array_equal(s, synthetic.spectrum(kind, n))
    assert np.abs(got - s).max() <= 100 * n * 2.0 ** -53
    B, _ = synthetic.test_matrix_device(m, n, kind, 1, 2, device="cpu")
    assert torch.equal(A, B)


def test_normal_kind_is_gaussian_entries():
    A, s = synthetic.test_matrix_device(300, 200, "normal", 7, 0, device="cpu")
    assert s is None and A.stride() == (1, 300)
    x = A.numpy().ravel()
    assert abs(x.mean()) < 5.0 / np.sqrt(x.size) and abs(x.var() - 1.0) < 0.02

"""Seeded synthetic test matrices A = U_A diag(sigma) V_A^T.

The paper factors "randomly generated" FP64 matrices without stating their
distribution (Sec. 6.1 and 6.2); these generators stand in for them.  The
module holds none of the factorization's arithmetic: only library QR/matmul
calls that draw orthogonal factors and a prescribed spectrum.  Both the CPU
oracle tests and the CUDA-path tests and benchmark draw their inputs here.
"""
from __future__ import annotations

import numpy as np

SPECTRA = ("geometric10", "gap", "algebraic", "geometric8", "normal")


def spectrum(kind: str, n: int) -> np.ndarray:
    """Singular values sigma_1 >= ... >= sigma_n of the synthetic workloads.

    geometric10: sigma_i = 10^(-10 (i-1)/(n-1))   (1 -> 1e-10)
    geometric8:  sigma_i = 10^(-8 (i-1)/(n-1))    (1 -> 1e-8)
    gap:         sigma_i = 1 for i <= n/10, then a gap to 1e-3 and geometric
                 decay to 1e-12 over the remaining indices
    algebraic:   sigma_i = 1 / i
    """
    i = np.arange(n, dtype=np.float64)
    if n == 0:
        return np.zeros(0)
    if kind == "geometric10":
        return 10.0 ** (-10.0 * i / max(n - 1, 1))
    if kind == "geometric8":
        return 10.0 ** (-8.0 * i / max(n - 1, 1))
    if kind == "algebraic":
        return 1.0 / (i + 1.0)
    if kind == "gap":
        k = n // 10
        s = np.empty(n)
        s[:k] = 1.0
        s[k:] = 10.0 ** np.linspace(-3.0, -12.0, n - k) if n - k > 1 else 1e-3
        return s
    raise ValueError("unknown spectrum %r" % kind)


def orthogonal(n: int, seed: int) -> np.ndarray:
    """Haar-distributed orthogonal n x n: Q of a seeded Gaussian, columns signed by diag(R)."""
    g = np.random.default_rng(seed).standard_normal((n, n))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return np.asfortranarray(q * d)


def test_matrix(m: int, n: int, kind: str = "geometric10", seed_u: int = 1, seed_v: int = 2) -> np.ndarray:
    """FP64 m x n (column-major) with prescribed singular values (numpy, small sizes).

    kind == "normal" gives i.i.d. N(0,1) entries drawn with seed_u instead.
    """
    if kind == "normal":
        return np.asfortranarray(np.random.default_rng(seed_u).standard_normal((m, n)))
    s = spectrum(kind, n)
    ua = orthogonal(m, seed_u)[:, :n]
    va = orthogonal(n, seed_v)
    return np.asfortranarray((ua * s) @ va.T)


def test_matrix_device(m: int, n: int, kind: str, seed_u: int, seed_v: int, device="cuda"):
    """Large synthetic matrix built on the GPU with torch (library QR and matmul).

    The orthogonal factors come from an FP32 QR of seeded Gaussians; the product
    is formed in FP64.  By multiplicative perturbation theory the singular values
    of the result equal the prescribed ones to a relative ~1e-6, which is what
    the quality ratios T_ii / sigma_i need.  Returns a column-major FP64 tensor
    (a transposed view of a row-major buffer) and the prescribed spectrum.
    """
    import torch

    gen = torch.Generator(device=device)
    if kind == "normal":
        gen.manual_seed(seed_u)
        a = torch.randn(n, m, generator=gen, device=device, dtype=torch.float64)
        return a.t(), None
    s = torch.from_numpy(spectrum(kind, n)).to(device)
    gen.manual_seed(seed_u)
    gu = torch.randn(m, m, generator=gen, device=device, dtype=torch.float32)
    qu = torch.linalg.qr(gu)[0][:, :n].to(torch.float64)
    del gu
    gen.manual_seed(seed_v)
    gv = torch.randn(n, n, generator=gen, device=device, dtype=torch.float32)
    qv = torch.linalg.qr(gv)[0].to(torch.float64)
    del gv
    # column-major A (m x n) == row-major A^T (n x m)
    at = (qv * s) @ qu.t()
    del qu, qv
    return at.t(), s.cpu().numpy()

"""Seeded synthetic test matrices A = U_A diag(sigma) V_A^T.

The paper factors "randomly generated" FP64 matrices without stating their
distribution (Sec. 6.1 and 6.2); these generators stand in for them.  The
module holds none of the factorization's arithmetic: only library QR/matmul
calls that draw orthogonal factors and a prescribed spectrum.  Both the CPU
oracle tests and the CUDA-path tests and benchmark draw their inputs here.
"""
from __future__ import annotations

import numpy as np

SPECTRA = ("geometric10", "gap", "algebraic", "geometric8", "normal", "exp32", "exp128")


def spectrum(kind: str, n: int) -> np.ndarray:
    """Singular values sigma_1 >= ... >= sigma_n of the synthetic workloads.

    geometric10: sigma_i = 10^(-10 (i-1)/(n-1))   (1 -> 1e-10)
    geometric8:  sigma_i = 10^(-8 (i-1)/(n-1))    (1 -> 1e-8)
    gap:         sigma_i = 1 for i <= n/10, then a gap to 1e-3 and geometric
                 decay to 1e-12 over the remaining indices
    algebraic:   sigma_i = 1 / i
    exp32, exp128: sigma_i = max(10^(-(i-1)/r), 1e-15), r = 32 or 128: a fixed
                 decay per index (four or one decade per 128 indices) down to a
                 floor near FP64 rounding, i.e. a numerically low-rank matrix
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
    if kind in ("exp32", "exp128"):
        r = 32.0 if kind == "exp32" else 128.0
        return np.maximum(10.0 ** (-i / r), 1e-15)
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


def _hartley_mix(X, gen, rounds: int = 2):
    """Apply an orthogonal Q = prod (P_r H D_r) to the columns of X (torch, FP64).

    D_r: random signs, H: orthonormal discrete Hartley transform
    (H x = (Re F x - Im F x) / sqrt(n), symmetric and orthogonal), P_r: random
    row permutation.  Every column of Q is dense; Q is orthogonal to FP64
    rounding, so the singular values of Q M equal those of M.
    """
    import torch

    n = X.shape[0]
    for _ in range(rounds):
        sg = torch.randint(0, 2, (n, 1), generator=gen, device=X.device, dtype=torch.int64) * 2 - 1
        X = X * sg.to(X.dtype)
        F = torch.fft.fft(X, dim=0)
        X = (F.real - F.imag) / (n ** 0.5)
        del F
        perm = torch.randperm(n, generator=gen, device=X.device)
        X = X[perm]
    return X


def test_matrix_device(m: int, n: int, kind: str, seed_u: int, seed_v: int, device="cuda"):
    """Large synthetic matrix A = Q_U [diag(sigma); 0] Q_V^T built on the device.

    Q_U, Q_V are FFT-based random orthogonal transforms (see _hartley_mix), so
    no dense QR is needed and the singular values of A are the prescribed ones
    to FP64 rounding.  kind == "normal" gives i.i.d. N(0,1) entries instead.
    Returns a column-major FP64 tensor (a transposed view of a row-major
    buffer) and the prescribed spectrum (None for "normal").
    """
    import torch

    gen = torch.Generator(device=device)
    if kind == "normal":
        gen.manual_seed(seed_u)
        a = torch.randn(n, m, generator=gen, device=device, dtype=torch.float64)
        return a.t(), None
    s = spectrum(kind, n)
    M0 = torch.zeros(m, n, dtype=torch.float64, device=device)
    M0.diagonal().copy_(torch.from_numpy(s))
    gen.manual_seed(seed_u)
    X = _hartley_mix(M0, gen)            # Q_U M0       (m x n)
    del M0
    gen.manual_seed(seed_v)
    At = _hartley_mix(X.t().contiguous(), gen)   # Q_V (Q_U M0)^T = A^T  (n x m, row-major)
    del X
    return At.t(), s


def graded(A: np.ndarray, span: float = 8.0, seed: int = 0) -> np.ndarray:
    """D_r A D_c with diagonal scalings whose entries run geometrically over
    [10^-span, 10^span] in a seeded random order, rows and columns drawn
    independently.  Rows and columns of the result then differ in scale by up
    to 10^(2 span), the case where scaling each row (or column) of a product
    operand by its largest entry truncates the small entries most."""
    m, n = A.shape
    g = np.random.default_rng(seed)
    dr = 10.0 ** g.permutation(np.linspace(-span, span, m)) if m > 1 else np.ones(m)
    dc = 10.0 ** g.permutation(np.linspace(-span, span, n)) if n > 1 else np.ones(n)
    return np.asfortranarray(dr[:, None] * np.asarray(A, dtype=np.float64) * dc[None, :])

"""A plain model of the emulated FP64 product, checked against exact
arithmetic (CPU).

The GPU path computes every FP64 product with the Ozaki scheme (Ozaki, Ogita,
Oishi & Rump 2012). This file restates its arithmetic in numpy and Python
integers, step by step:

- row and column scales from the largest exponent;
- 8 signed digits of 7 bits each;
- the 36 digit pairs with s + t <= 7 (0-based);
- exact integer digit sums over chunks of 128;
- a double-float FP32 fold of each chunk;
- the FP64 result.

It then checks the error bound stated for the scheme. It does not import or
run the CUDA code. It pins the design's arithmetic and error model; the GPU
tests pin the kernels against the oracle.
"""
from fractions import Fraction

import numpy as np
import pytest

S = 8          # digits per operand
W = 7          # bits per digit
CHUNK = 128    # k per exact FP32 chunk
NO_SCALE = np.iinfo(np.int64).min


def scales(X):
    """e_r with |X(r, :)| < 2^e_r from the largest biased exponent of row r (0-rows: NO_SCALE)."""
    be = ((X.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    m = be.max(axis=1)
    return np.where(m == 0, NO_SCALE, m - 1022)


def digits(X, e):
    """Signed digits D[s, r, k]: X(r, k) ~ 2^e_r sum_s D[s, r, k] 2^(-7(s+1)), truncated."""
    bits = X.view(np.uint64)
    be = ((bits >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    mant = (bits & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
    F = np.zeros(X.shape, dtype=np.uint64)
    ok = (be != 0) & (e[:, None] != NO_SCALE)
    sh = np.where(ok, be - 1075 - np.where(e == NO_SCALE, 0, e)[:, None] + W * S, -64)
    up = ok & (sh >= 0)
    dn = ok & (sh < 0) & (sh > -64)
    F[up] = mant[up] << sh[up].astype(np.uint64)
    F[dn] = mant[dn] >> (-sh[dn]).astype(np.uint64)
    sign = np.where((bits >> np.uint64(63)) != 0, -1, 1)
    return np.stack([((F >> np.uint64(W * (S - 1 - s))) & np.uint64(127)).astype(np.int64) * sign
                     for s in range(S)])


def f32(x):
    return np.float32(x)


def emulated_dot(da, db, er, ec):
    """One output element from the digits of a row (da[s, k]) and a column (db[t, k])."""
    if er == NO_SCALE or ec == NO_SCALE:
        return 0.0, 0
    K = da.shape[1]
    hi, lo = f32(0.0), f32(0.0)
    max_sum = 0
    for k0 in range(0, K, CHUNK):
        sl = slice(k0, min(K, k0 + CHUNK))
        sums = [sum(int(np.dot(da[s, sl], db[d - s, sl])) for s in range(d + 1)) for d in range(S)]
        max_sum = max(max_sum, max(abs(x) for x in sums))
        for d in range(S - 1, -1, -1):      # fold: two-sum into hi, errors into lo
            x = f32(f32(sums[d]) * f32(2.0 ** (-W * (d + 2))))
            s_ = f32(hi + x)
            bb = f32(s_ - hi)
            err = f32(f32(hi - f32(s_ - bb)) + f32(x - bb))
            hi, lo = s_, f32(lo + err)
        s_ = f32(hi + lo)                  # renormalise
        lo = f32(lo - f32(s_ - hi))
        hi = s_
    scale = 2.0 ** int(er + ec)
    return float(hi) * scale + float(lo) * scale, max_sum


def exact_dot(a, b):
    return sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))


def bound(a, b, er, ec):
    """Error bound of the scheme for one element.

    truncation of both operands and the dropped pairs (s + t >= 8):
        2^(er+ec) K (2 + 7.06) 2^-56
    rounding of lo in the fold, at most 8 per chunk, each below 9 2^-48 of
    the running sum (bounded by sum_k |a_k b_k| plus the truncation):
        72 ceil(K / 128) 2^-48 sum_k |a_k b_k|
    and the final FP64 addition: 2^-53 |result|.
    """
    K = len(a)
    sab = float(np.sum(np.abs(a) * np.abs(b)))
    trunc = 2.0 ** float(er + ec) * K * 9.06 * 2.0 ** -56
    fold = 72 * -(-K // CHUNK) * 2.0 ** -48 * (sab + trunc)
    return trunc + fold + 2.0 ** -53 * (sab + trunc)


def _cases():
    rng = np.random.default_rng(7)
    K = 700                                          # five full chunks and a ragged one
    normal = (rng.standard_normal((3, K)), rng.standard_normal((K, 3)))
    wide = (rng.standard_normal((3, K)) * 2.0 ** rng.integers(-40, 1, (3, K)),
            rng.standard_normal((K, 3)) * 2.0 ** rng.integers(-40, 1, (K, 3)))
    same_sign = (np.abs(rng.standard_normal((3, K))), np.abs(rng.standard_normal((K, 3))))
    cancel = (np.vstack([rng.standard_normal(K)] * 3), np.column_stack([rng.standard_normal(K)] * 3))
    cancel[1][:, 1] = -cancel[0][0] * (1 + 2.0 ** -30 * rng.standard_normal(K))   # sum near 0
    return {"normal": normal, "wide": wide, "same_sign": same_sign, "cancel": cancel}


def test_digits_are_bf16_exact_and_reconstruct_to_56_bits():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4, 300)) * 2.0 ** rng.integers(-60, 60, (4, 300))
    X[1, :5] = [0.0, -0.0, 5e-324, 2.0 ** -1022, -1.0]          # zeros and subnormals
    e = scales(X)
    D = digits(X, e)
    assert np.abs(D).max() <= 127                              # 7 bits: exact in BF16
    for r in range(X.shape[0]):
        assert np.abs(X[r]).max() < 2.0 ** int(e[r]) <= 2 * np.abs(X[r]).max()
        for k in range(X.shape[1]):
            x = Fraction(float(X[r, k]))
            y = Fraction(2) ** int(e[r]) * sum(Fraction(int(D[s, r, k]), 2 ** (W * (s + 1))) for s in range(S))
            if X[r, k] != 0 and abs(X[r, k]) >= 2.0 ** -1022:
                assert abs(x - y) < Fraction(2) ** (int(e[r]) - 56)
                assert y == 0 or (y > 0) == (x > 0)
            else:                                              # subnormals are dropped
                assert y == 0


def test_chunk_sums_are_exact_in_fp32():
    # the largest digit sum of a chunk: 8 pairs x 128 x 127^2 < 2^24
    assert 8 * CHUNK * 127 * 127 < 2 ** 24
    full = np.full((S, CHUNK), 127, dtype=np.int64)            # every digit at its largest
    _, m = emulated_dot(full, full, 0, 0)
    assert m == 8 * CHUNK * 127 * 127 and float(np.float32(m)) == m
    # a double has 53 significant bits, so its 56-bit digit string ends in 3 zero bits
    A = np.full((1, CHUNK), 1.0 - 2.0 ** -53)
    da = digits(A, scales(A))
    assert (da[:S - 1] == 127).all() and (da[S - 1] == 120).all()


@pytest.mark.parametrize("case", ["normal", "wide", "same_sign", "cancel"])
def test_emulated_product_within_its_bound(case):
    A, B = _cases()[case]
    er, ec = scales(A), scales(B.T)
    da, db = digits(A, er), digits(np.ascontiguousarray(B.T), ec)
    for r in range(A.shape[0]):
        for c in range(B.shape[1]):
            v, _ = emulated_dot(da[:, r], db[:, c], er[r], ec[c])
            exact = exact_dot(A[r], B[:, c])
            err = abs(Fraction(v) - exact)
            assert err <= Fraction(bound(A[r], B[:, c], er[r], ec[c])), (case, r, c, float(err))


def test_typical_error_against_fp64_dot():
    """On N(0,1) data the emulated product stays within a small factor of an
    FP64 dot product's own error (both against the exact sum)."""
    rng = np.random.default_rng(3)
    K, n = 1024, 24
    A, B = rng.standard_normal((n, K)), rng.standard_normal((K, n))
    er, ec = scales(A), scales(B.T)
    da, db = digits(A, er), digits(np.ascontiguousarray(B.T), ec)
    emu, f64 = [], []
    for i in range(n):
        exact = exact_dot(A[i], B[:, i])
        v, _ = emulated_dot(da[:, i], db[:, i], er[i], ec[i])
        sab = float(np.sum(np.abs(A[i] * B[:, i])))
        emu.append(float(abs(Fraction(v) - exact)) / sab)
        f64.append(float(abs(Fraction(float(np.dot(A[i], B[:, i]))) - exact)) / sab)
    assert np.median(emu) <= 2.0 ** -44
    assert np.median(emu) <= 64 * max(np.median(f64), 2.0 ** -53)

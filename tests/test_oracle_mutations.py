"""Planted mistakes in copies of the oracle: the pins must reject every one.

Each case rewrites one expression of ``oracle/randutv_oracle.c`` in a
temporary copy: a wrong sign, a dropped term, a transposed index, a wrong
constant or a skipped step. The test builds the copy and loads it in place of
the oracle. It then runs the pins of ``test_oracle_pins.py`` that cover the
changed routine, and at least one of them must fail. A copy with no change
must pass the same pins, so a failure comes from the planted mistake and not
from the harness. Every rewrite keeps each access inside its buffer. CPU only.
"""
import os

import pytest

import oracle.oracle as omod
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(omod.__file__), "randutv_oracle.c")


def _philox():
    pins.test_philox_known_answer()


def _gaussian():
    pins.test_gaussian_is_standard_normal_and_independent()


def _hqr():
    pins.test_householder_qr_matches_lapack((50, 20), 0)
    pins.test_householder_zero_subcolumn_and_signs()


def _larft():
    pins.test_larft_matches_lapack_and_explicit_product((40, 12), 0)


def _jacobi():
    pins.test_jacobi_svd_random(17, 2)
    pins.test_jacobi_svd_diagonal_closed_form()


def _utv():
    pins.test_randutv_brute_force_small(64, 64, 16, 1, "geometric10")
    pins.test_randutv_brute_force_small(96, 40, 16, 2, "geometric10")


def _sketch():
    pins.test_randutv_step0_matches_sketch_subspace("geometric10")
    pins.test_randutv_power_iteration_sharpens_gap_spectrum()


def _qrfirst():
    pins.test_randutv_qrfirst_against_lapack_qr_and_identities(300, 100, 16, 1, "geometric10")
    pins.test_randutv_qrfirst_against_lapack_qr_and_identities(160, 40, 12, 2, "normal")


# (what the mistake is, text in the oracle, its replacement, pins that must see it)
MUTANTS = [
    ("Philox key schedule constants swapped", "k0 += W0; k1 += W1;", "k0 += W1; k1 += W0;", _philox),
    ("Philox multiplier of the second lane", "mulhilo64(M1, x2, &hi1, &lo1);", "mulhilo64(M0, x2, &hi1, &lo1);",
     _philox),
    ("Box-Muller radius without the factor 2", "sqrt(-2.0 * log(u[2 * pair]))", "sqrt(-1.0 * log(u[2 * pair]))",
     _gaussian),
    ("dlarfg sign of beta", "(alpha >= 0.0) ? -h : h", "(alpha >= 0.0) ? h : -h", _hqr),
    ("reflector drops the pivot-row term", "double w = A[IDX(j, c, lda)];", "double w = 0.0;", _hqr),
    ("tau of the wrong form", "tau[j] = (beta - alpha) / beta;", "tau[j] = (beta - alpha) / alpha;", _hqr),
    ("T factor column of the wrong sign", "z[i] = -tau[j] * s;", "z[i] = tau[j] * s;", _larft),
    ("T factor with a transposed operand", "s += Tf[IDX(i, l, ldt)] * z[l];", "s += Tf[IDX(l, i, ldt)] * z[l];",
     _larft),
    ("Jacobi rotation of the wrong sign", "A[IDX(r, p, n)] = c * ap - s * aq;", "A[IDX(r, p, n)] = c * ap + s * aq;",
     _jacobi),
    ("Jacobi tangent of the wrong sign", "double t = (zeta >= 0.0 ? 1.0 : -1.0)",
     "double t = (zeta >= 0.0 ? -1.0 : 1.0)", _jacobi),
    ("singular values sorted ascending", "norms[order[b]] < norms[key]", "norms[order[b]] > norms[key]", _jacobi),
    ("canonical sign inverted", "if (Vs[IDX(imax, j, ldv)] < 0.0)", "if (Vs[IDX(imax, j, ldv)] > 0.0)", _jacobi),
    ("power iteration skipped", "for (int64_t it = 0; it < q; ++it)", "for (int64_t it = 0; it < 0; ++it)", _sketch),
    ("right update skips the rows above the block",
     "apply_wy_right(m, np, b, T + IDX(0, k0, m), m, W, np, Tf, b);",
     "apply_wy_right(mp, np, b, T + IDX(k0, k0, m), m, W, np, Tf, b);", _utv),
    ("V not updated by the right transform", "if (V) apply_wy_right(n, np, b, V + IDX(0, k0, n), n, W, np, Tf, b);",
     "", _utv),
    ("left update applies the transform, not its transpose",
     "oracle_gemm(1, 0, k, N, k, 1.0, Tf, ldt, X, k, 0.0, X2, k);",
     "oracle_gemm(0, 0, k, N, k, 1.0, Tf, ldt, X, k, 0.0, X2, k);", _utv),
    ("block row multiplied by Us instead of its transpose",
     "oracle_gemm(1, 0, w, nr, w, 1.0, Us, w, T + IDX(k0, k0 + w, m), m, 0.0, X, w);",
     "oracle_gemm(0, 0, w, nr, w, 1.0, Us, w, T + IDX(k0, k0 + w, m), m, 0.0, X, w);", _utv),
    ("columns above the block not multiplied by Vs", "    if (k0 > 0) {\n        double* X", "    if (0) {\n        double* X",
     _utv),
    ("U not multiplied by Us", "U[IDX(i, k0 + j, m)] = X[IDX(i, j, m)];", "(void)X;", _utv),
    ("QR-first: reflectors applied to U in the wrong order", "for (int64_t j = n - 1; j >= 0; --j) {",
     "for (int64_t j = 0; j < n; ++j) {", _qrfirst),
    ("QR-first: the pivot row of a reflector not updated", "                U[IDX(j, c, m)] -= s;\n", "\n",
     _qrfirst),
    ("QR-first: randUTV run on A instead of R", "int status = oracle_randutv(n, n, R, n, b, q, seed, UR, TR, V,",
     "int status = oracle_randutv(n, n, F, m, b, q, seed, UR, TR, V,", _qrfirst),
]


def _load_copy(tmp_path, name, text, monkeypatch):
    path = os.path.join(str(tmp_path), name + ".c")
    with open(path, "w") as f:
        f.write(text)
    lib = os.path.join(str(tmp_path), "lib" + name + ".so")
    omod.compile_source(path, lib)
    monkeypatch.setattr(omod, "_lib", omod.bind(lib))


def _rejected(check) -> bool:
    try:
        check()
    except Exception:  # an assertion, or a library routine refusing NaN input
        return True
    return False


def test_unchanged_copy_passes_the_pins(tmp_path, monkeypatch):
    with open(SRC) as f:
        _load_copy(tmp_path, "same", f.read(), monkeypatch)
    for check in (_philox, _gaussian, _hqr, _larft, _jacobi, _utv, _sketch, _qrfirst):
        check()


@pytest.mark.parametrize("what,old,new,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_rejected(what, old, new, check, tmp_path, monkeypatch):
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, "the rewritten text must occur once in the oracle: %r" % old
    _load_copy(tmp_path, "mutant", text.replace(old, new), monkeypatch)
    assert _rejected(check), "no pin rejects: " + what

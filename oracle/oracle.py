"""ctypes wrapper around ``randutv_oracle.c`` (plain FP64 CPU oracle).

TEST INFRASTRUCTURE ONLY: this module is the checker of the CUDA path and is
imported only by tests, the smoke check and the CPU-baseline leg of the
benchmark.  Every function mirrors one routine of the C file, which cites the
passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "randutv_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64


def compile_source(src: str, out: str) -> None:
    """gcc -O2 -fopenmp of one C source into the shared library ``out``."""
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (plain gcc, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


def bind(path: str):
    """Load a library built from the oracle's C source and declare its signatures."""
    lib = ctypes.CDLL(path)
    lib.oracle_philox4x64_10.argtypes = [ctypes.POINTER(ctypes.c_uint64)] * 3
    lib.oracle_gaussian.argtypes = [ctypes.c_uint64, _i64, _i64, _i64, _dp, _i64]
    lib.oracle_gemm.argtypes = [ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, ctypes.c_double,
                                _dp, _i64, _dp, _i64, ctypes.c_double, _dp, _i64]
    lib.oracle_householder_qr.argtypes = [_i64, _i64, _dp, _i64, _dp]
    lib.oracle_larft.argtypes = [_i64, _i64, _dp, _i64, _dp, _dp, _i64]
    lib.oracle_jacobi_svd.argtypes = [_i64, _dp, _i64, _dp, _dp, _i64, _dp, _i64, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]
    lib.oracle_jacobi_svd.restype = ctypes.c_int
    lib.oracle_randutv.argtypes = [_i64, _i64, _dp, _i64, _i64, _i64, ctypes.c_uint64,
                                   _dp, _dp, _dp, _i64, ctypes.c_int]
    lib.oracle_randutv.restype = ctypes.c_int
    lib.oracle_randutv_qrfirst.argtypes = [_i64, _i64, _dp, _i64, _i64, _i64, ctypes.c_uint64,
                                           _dp, _dp, _dp, _i64, ctypes.c_int]
    lib.oracle_randutv_qrfirst.restype = ctypes.c_int
    lib.oracle_num_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _fortran(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_num_threads())


def philox4x64_10(counter, key) -> np.ndarray:
    """Philox4x64-10 block function (Salmon et al., SC'11) -> four uint64."""
    ctr = (ctypes.c_uint64 * 4)(*[int(c) & (2**64 - 1) for c in counter])
    k = (ctypes.c_uint64 * 2)(*[int(c) & (2**64 - 1) for c in key])
    out = (ctypes.c_uint64 * 4)()
    _load().oracle_philox4x64_10(ctr, k, out)
    return np.array(list(out), dtype=np.uint64)


def gaussian(seed: int, step: int, rows: int, cols: int) -> np.ndarray:
    """G^(step) (rows x cols) of the sketch, Sec. 3.2.1 (Philox + Box-Muller)."""
    G = np.zeros((rows, cols), dtype=np.float64, order="F")
    _load().oracle_gaussian(seed, step, rows, cols, _ptr(G), max(rows, 1))
    return G


def gemm(A, B, transA=False, transB=False) -> np.ndarray:
    """Plain triple-loop product op(A) op(B)."""
    A = _fortran(A)
    B = _fortran(B)
    M = A.shape[1] if transA else A.shape[0]
    K = A.shape[0] if transA else A.shape[1]
    N = B.shape[0] if transB else B.shape[1]
    C = np.zeros((M, N), order="F")
    _load().oracle_gemm(int(transA), int(transB), M, N, K, 1.0, _ptr(A), max(A.shape[0], 1), _ptr(B),
                        max(B.shape[0], 1), 0.0, _ptr(C), max(M, 1))
    return C


def householder_qr(A):
    """HQR (Sec. 2.2) with the dlarfg sign rule -> (R_and_W storage, tau)."""
    A = _fortran(A).copy(order="F")
    M, N = A.shape
    tau = np.zeros(min(M, N))
    _load().oracle_householder_qr(M, N, _ptr(A), max(M, 1), _ptr(tau))
    return A, tau


def larft(W, tau) -> np.ndarray:
    """Upper triangular T of the compact WY form Q = I - W T W^T (Sec. 2.3)."""
    W = _fortran(W)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    M, k = W.shape
    Tf = np.zeros((k, k), order="F")
    _load().oracle_larft(M, k, _ptr(W), max(M, 1), _ptr(tau), _ptr(Tf), max(k, 1))
    return Tf


def jacobi_svd(R, max_sweeps: int = 30):
    """One-sided Jacobi SVD R = Us diag(D) Vs^T -> (D, Us, Vs, sweeps, status)."""
    R = _fortran(R)
    n = R.shape[0]
    D = np.zeros(n)
    Us = np.zeros((n, n), order="F")
    Vs = np.zeros((n, n), order="F")
    sw = ctypes.c_int(0)
    rc = _load().oracle_jacobi_svd(n, _ptr(R), max(n, 1), _ptr(D), _ptr(Us), max(n, 1), _ptr(Vs),
                                   max(n, 1), max_sweeps, ctypes.byref(sw))
    return D, Us, Vs, sw.value, rc


def randutv(A, b: int, q: int, seed: int, want_uv: bool = True, stop_after: int = -1,
            max_sweeps: int = 30):
    """Blocked randUTV A = U T V^T (Sec. 3.2) -> (U, T, V, status).

    U and V are None when ``want_uv`` is False ("no orthonormal matrices").
    """
    A = _fortran(A)
    m, n = A.shape
    T = np.zeros((m, n), order="F")
    U = np.zeros((m, m), order="F") if want_uv else None
    V = np.zeros((n, n), order="F") if want_uv else None
    rc = _load().oracle_randutv(m, n, _ptr(A), max(m, 1), b, q, seed, _ptr(U), _ptr(T), _ptr(V),
                                stop_after, max_sweeps)
    if rc < 0:
        raise ValueError("oracle_randutv: invalid arguments")
    return U, T, V, rc


def randutv_qrfirst(A, b: int, q: int, seed: int, want_uv: bool = True, stop_after: int = -1,
                    max_sweeps: int = 30):
    """randUTV with a Householder QR first (Sec. 5.1, tall inputs): A = Q_A [R; 0],
    R = U_R T_R V^T, U = Q_A diag(U_R, I) -> (U, T, V, status)."""
    A = _fortran(A)
    m, n = A.shape
    T = np.zeros((m, n), order="F")
    U = np.zeros((m, m), order="F") if want_uv else None
    V = np.zeros((n, n), order="F") if want_uv else None
    rc = _load().oracle_randutv_qrfirst(m, n, _ptr(A), max(m, 1), b, q, seed, _ptr(U), _ptr(T), _ptr(V),
                                        stop_after, max_sweeps)
    if rc < 0:
        raise ValueError("oracle_randutv_qrfirst: invalid arguments")
    return U, T, V, rc

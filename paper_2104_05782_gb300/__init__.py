"""GB300-native blocked randUTV (A = U T V^T), Python binding of librandutv.so.

The functions below carry the names of the C ABI in ``include/randutv.h`` and
only marshal arguments: every step of the factorization runs in the library's
CUDA kernels.  PyTorch is used for device memory and streams only.  There is no
CPU fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librandutv.so")

RANDUTV_OK = 0
RANDUTV_EINVAL = 1
RANDUTV_ENOMEM = 2
RANDUTV_ENONFINITE = 3
RANDUTV_ENOCONV = 4
RANDUTV_ETIMEOUT = 5
RANDUTV_ECUDA = 6
RANDUTV_ENOTIMPL = 7

RANDUTV_FP64 = 0
RANDUTV_SKETCH_BF16 = 1
RANDUTV_SKETCH_FP16_SCALED = 2
RANDUTV_SKETCH_FP32 = 3

_lib = None
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p


class TraceClass(ctypes.Structure):
    """randutv_trace_class of the C ABI."""
    _fields_ = [("name", ctypes.c_char * 32), ("scopes", ctypes.c_int64), ("kernels", ctypes.c_int64),
                ("ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class RandUTVError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s: status %d (%s)" % (what or "randutv", status, status_string(status)))


def load():
    """Load librandutv.so (built by ``paper_2104_05782_gb300.build``); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librandutv.so is not built (%s); run __graft_entry__.build() or "
                           "python -m paper_2104_05782_gb300.build" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    lib.randutv_status_string.argtypes = [ctypes.c_int]
    lib.randutv_status_string.restype = ctypes.c_char_p
    lib.randutv_factor.argtypes = [_i64, _i64, _vp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                   _vp, _vp, _vp]
    lib.randutv_factor.restype = ctypes.c_int
    lib.randutv_factor_ex.argtypes = [_i64, _i64, _vp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                      _vp, _vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_size_t, _i64, _vp]
    lib.randutv_factor_ex.restype = ctypes.c_int
    lib.randutv_workspace_size.argtypes = [_i64, _i64, ctypes.c_int, ctypes.c_int]
    lib.randutv_workspace_size.restype = ctypes.c_size_t
    lib.randutv_factor_host.argtypes = [_i64, _i64, _vp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                        _vp, _vp, _vp, ctypes.c_int]
    lib.randutv_factor_host.restype = ctypes.c_int
    lib.randutv_trace_enable.argtypes = [ctypes.c_int]
    lib.randutv_trace_enable.restype = ctypes.c_int
    lib.randutv_trace_read.argtypes = [ctypes.POINTER(TraceClass), ctypes.c_int]
    lib.randutv_trace_read.restype = ctypes.c_int
    lib.randutv_trace_reset.argtypes = []
    lib.randutv_trace_reset.restype = None
    lib.randutv_launch_count.argtypes = []
    lib.randutv_launch_count.restype = ctypes.c_longlong
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().randutv_status_string(int(status)).decode()


def _ptr(x):
    """Device/host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("expected a tensor, array, int address or None, got %r" % type(x))


def _stream_handle(stream):
    if stream is None or isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- C ABI mirrors
def randutv_factor(m, n, A, lda, b, q, seed, U, T, V) -> int:
    """randutv_factor of the C ABI (device pointers / CUDA tensors); returns the status."""
    return load().randutv_factor(m, n, _ptr(A), lda, b, q, seed, _ptr(U), _ptr(T), _ptr(V))


def randutv_factor_ex(m, n, A, lda, b, q, seed, U, T, V, prec=RANDUTV_FP64, stream=None,
                      workspace=None, ws_bytes=0, stop_after=-1, info=None) -> int:
    """randutv_factor_ex of the C ABI; returns the status."""
    return load().randutv_factor_ex(m, n, _ptr(A), lda, b, q, seed, _ptr(U), _ptr(T), _ptr(V), prec,
                                    _stream_handle(stream), _ptr(workspace), ws_bytes, stop_after, _ptr(info))


def randutv_workspace_size(m, n, b, prec=RANDUTV_FP64) -> int:
    return int(load().randutv_workspace_size(m, n, b, prec))


def randutv_factor_host(m, n, A, lda, b, q, seed, U, T, V, prec=RANDUTV_FP64) -> int:
    """randutv_factor_host of the C ABI: host (numpy, Fortran-order) buffers."""
    return load().randutv_factor_host(m, n, _ptr(A), lda, b, q, seed, _ptr(U), _ptr(T), _ptr(V), prec)


def randutv_trace_enable(on: bool) -> int:
    return int(load().randutv_trace_enable(1 if on else 0))


def randutv_trace_reset() -> None:
    load().randutv_trace_reset()


def randutv_launch_count() -> int:
    return int(load().randutv_launch_count())


def randutv_trace_read(max_classes: int = 64) -> dict:
    """Per-class totals {name: {scopes, kernels, ms, flops, bytes}} (synchronises the events)."""
    buf = (TraceClass * max_classes)()
    n = load().randutv_trace_read(buf, max_classes)
    out = {}
    for i in range(min(n, max_classes)):
        c = buf[i]
        out[c.name.decode()] = {"scopes": c.scopes, "kernels": c.kernels, "ms": c.ms, "flops": c.flops,
                                "bytes": c.bytes}
    return out


# ---------------------------------------------------------------- conveniences
def colmajor_empty(rows, cols, device="cuda"):
    """Uninitialised FP64 column-major (rows x cols) CUDA tensor (a transposed view)."""
    import torch

    return torch.empty((cols, rows), dtype=torch.float64, device=device).t()


def is_colmajor(x) -> bool:
    rows, cols = x.shape
    return x.stride(0) == 1 and (x.stride(1) == rows or cols <= 1) or (rows <= 1 and x.stride(1) >= 1)


def factor(A, b: int, q: int, seed: int = 0, want_uv: bool = True, prec: int = RANDUTV_FP64,
           stream=None, stop_after: int = -1, check: bool = True):
    """Factor a column-major FP64 CUDA tensor A (m x n) -> (U, T, V) column-major tensors.

    U and V are None when ``want_uv`` is False.
    """
    m, n = A.shape
    if not is_colmajor(A):
        raise ValueError("A must be column-major (e.g. a transposed contiguous tensor)")
    T = colmajor_empty(m, n, A.device)
    U = colmajor_empty(m, m, A.device) if want_uv else None
    V = colmajor_empty(n, n, A.device) if want_uv else None
    lda = A.stride(1) if n > 1 else max(m, 1)
    st = randutv_factor_ex(m, n, A, max(lda, m, 1), b, q, seed, U, T, V, prec, stream, None, 0, stop_after, None)
    if check and st != RANDUTV_OK:
        raise RandUTVError(st, "randutv_factor_ex")
    return U, T, V

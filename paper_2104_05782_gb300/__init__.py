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
RANDUTV_FP64_EMULATED = 4
RANDUTV_EMULATED_SKETCH_BF16 = 5

_lib = None
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p


class TraceClass(ctypes.Structure):
    """randutv_trace_class of the C ABI."""
    _fields_ = [("name", ctypes.c_char * 32), ("scopes", ctypes.c_int64), ("kernels", ctypes.c_int64),
                ("ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class Options(ctypes.Structure):
    """randutv_options of the C ABI."""
    _fields_ = [("prec", ctypes.c_int), ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t), ("stop_after", ctypes.c_int64), ("rank_tol", ctypes.c_double),
                ("start_col", ctypes.c_int64), ("qr_first", ctypes.c_int), ("cols_done", ctypes.c_int64),
                ("rank", ctypes.c_int64)]


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
    pa = ctypes.POINTER(ctypes.c_int64)
    pp = ctypes.POINTER(ctypes.c_void_p)
    lib.randutv_batched.argtypes = [ctypes.c_int, pa, pa, pp, pa, pp, pp, pp, ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), _vp]
    lib.randutv_batched.restype = ctypes.c_int
    lib.randutv_batched_plan_create.argtypes = [ctypes.c_int, pa, pa, pp, pa, pp, pp, pp,
                                                ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.c_int,
                                                ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    lib.randutv_batched_plan_create.restype = ctypes.c_int
    lib.randutv_batched_plan_run.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), _vp]
    lib.randutv_batched_plan_run.restype = ctypes.c_int
    lib.randutv_batched_plan_destroy.argtypes = [_vp]
    lib.randutv_batched_plan_destroy.restype = None
    lib.randutv_batched_autotune.argtypes = [ctypes.c_int, pa, pa, pp, pa, pp, pp, pp,
                                             ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_char_p, ctypes.c_size_t, _vp]
    lib.randutv_batched_autotune.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.randutv_learnq_model_floats.argtypes = []
    lib.randutv_learnq_model_floats.restype = ctypes.c_int
    lib.randutv_factor_learnedq.argtypes = [_i64, _i64, _vp, _i64, ctypes.c_int, fp, ctypes.c_uint64, _vp, _vp, _vp,
                                            ip]
    lib.randutv_factor_learnedq.restype = ctypes.c_int
    lib.randutv_factor_learnedq_ex.argtypes = [_i64, _i64, _vp, _i64, ctypes.c_int, fp, ctypes.c_uint64, _vp, _vp,
                                               _vp, ip, ctypes.c_int, _vp]
    lib.randutv_factor_learnedq_ex.restype = ctypes.c_int
    lib.randutv_learnq_trace.argtypes = [_i64, _i64, _vp, _i64, ctypes.c_int, ctypes.c_uint64, _vp, fp, ip,
                                         ctypes.POINTER(ctypes.c_double), _i64, ctypes.POINTER(ctypes.c_int64)]
    lib.randutv_learnq_trace.restype = ctypes.c_int
    lib.randutv_learnq_trace_ex.argtypes = [_i64, _i64, _vp, _i64, ctypes.c_int, ctypes.c_uint64, _vp, fp, ip,
                                            ctypes.POINTER(ctypes.c_double), _i64, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.c_int, _i64]
    lib.randutv_learnq_trace_ex.restype = ctypes.c_int
    lib.randutv_learnq_train.argtypes = [fp, ip, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float, fp, fp]
    lib.randutv_learnq_train.restype = ctypes.c_int
    lib.randutv_learnq_grad.argtypes = [fp, ip, ctypes.c_int, fp, fp, fp]
    lib.randutv_learnq_grad.restype = ctypes.c_int
    lib.randutv_learnq_predict.argtypes = [fp, fp, ctypes.c_int, fp]
    lib.randutv_learnq_predict.restype = ctypes.c_int
    op = ctypes.POINTER(Options)
    lib.randutv_options_init.argtypes = [op]
    lib.randutv_options_init.restype = None
    lib.randutv_workspace_size_opt.argtypes = [_i64, _i64, ctypes.c_int, op]
    lib.randutv_workspace_size_opt.restype = ctypes.c_size_t
    lib.randutv_factor_opt.argtypes = [_i64, _i64, _vp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                       _vp, _vp, _vp, op]
    lib.randutv_factor_opt.restype = ctypes.c_int
    lib.randutv_set_limits.argtypes = [_i64, ctypes.c_int]
    lib.randutv_set_limits.restype = None
    lib.randutv_svd_small_noalloc.argtypes = [ctypes.c_int, _vp, _i64, _vp, _vp, _vp, _vp]
    lib.randutv_svd_small_noalloc.restype = ctypes.c_int
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


def randutv_options(prec=RANDUTV_FP64, stream=None, workspace=None, ws_bytes=0, stop_after=-1, rank_tol=0.0,
                    start_col=0, qr_first=False) -> Options:
    """A randutv_options filled by randutv_options_init, then with these fields."""
    o = Options()
    load().randutv_options_init(ctypes.byref(o))
    o.prec = prec
    o.stream = _stream_handle(stream)
    o.workspace = _ptr(workspace)
    o.ws_bytes = ws_bytes
    o.stop_after = stop_after
    o.rank_tol = rank_tol
    o.start_col = start_col
    o.qr_first = 1 if qr_first else 0
    return o


def randutv_factor_opt(m, n, A, lda, b, q, seed, U, T, V, opt=None) -> int:
    """randutv_factor_opt of the C ABI; opt (an Options or None) receives cols_done and rank."""
    return load().randutv_factor_opt(m, n, _ptr(A), lda, b, q, seed, _ptr(U), _ptr(T), _ptr(V),
                                     ctypes.byref(opt) if opt is not None else None)


def randutv_workspace_size_opt(m, n, b, opt=None) -> int:
    return int(load().randutv_workspace_size_opt(m, n, b, ctypes.byref(opt) if opt is not None else None))


def randutv_set_limits(wait_polls: int, max_sweeps: int) -> None:
    """randutv_set_limits of the C ABI (<= 0 restores a default)."""
    load().randutv_set_limits(int(wait_polls), int(max_sweeps))


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


def _batch_arrays(m, n, A, lda, U, T, V, seed):
    count = len(m)
    i64 = lambda xs: (ctypes.c_int64 * count)(*[int(x) for x in xs])
    ptrs = lambda xs: None if xs is None else (ctypes.c_void_p * count)(*[_ptr(x) for x in xs])
    seeds = (ctypes.c_uint64 * count)(*[int(x) for x in (seed if seed is not None else [0] * count)])
    return count, i64(m), i64(n), ptrs(A), i64(lda), ptrs(U), ptrs(T), ptrs(V), seeds


def randutv_batched(m, n, A, lda, U, T, V, seed, q, prec=RANDUTV_FP64, autotune_table=None, status=None,
                    stream=None) -> int:
    """randutv_batched of the C ABI; per-matrix lists of sizes and device buffers."""
    count, cm, cn, cA, cl, cU, cT, cV, cs = _batch_arrays(m, n, A, lda, U, T, V, seed)
    st = (ctypes.c_int * count)() if status is not None else None
    tab = autotune_table.encode() if isinstance(autotune_table, str) else autotune_table
    r = load().randutv_batched(count, cm, cn, cA, cl, cU, cT, cV, cs, q, prec, tab, st, _stream_handle(stream))
    if status is not None:
        status[:] = list(st)
    return r


def randutv_batched_autotune(m, n, A, lda, U, T, V, seed, q, prec=RANDUTV_FP64, stream=None):
    """randutv_batched_autotune of the C ABI -> (status, table text)."""
    count, cm, cn, cA, cl, cU, cT, cV, cs = _batch_arrays(m, n, A, lda, U, T, V, seed)
    buf = ctypes.create_string_buffer(8192)
    r = load().randutv_batched_autotune(count, cm, cn, cA, cl, cU, cT, cV, cs, q, prec, buf, 8192,
                                        _stream_handle(stream))
    return r, buf.value.decode()


class BatchPlan:
    """randutv_batched_plan_create / _run / _destroy: a batch held on the device as a CUDA graph."""

    def __init__(self, m, n, A, lda, U, T, V, seed, q, prec=RANDUTV_FP64, autotune_table=None):
        count, cm, cn, cA, cl, cU, cT, cV, cs = _batch_arrays(m, n, A, lda, U, T, V, seed)
        self.count = count
        self._keep = (A, U, T, V)
        tab = autotune_table.encode() if isinstance(autotune_table, str) else autotune_table
        h = ctypes.c_void_p()
        r = load().randutv_batched_plan_create(count, cm, cn, cA, cl, cU, cT, cV, cs, q, prec, tab, ctypes.byref(h))
        if r != RANDUTV_OK:
            raise RandUTVError(r, "randutv_batched_plan_create")
        self.handle = h

    def run(self, stream=None):
        """Replay the batch; returns (worst status, per-matrix statuses)."""
        st = (ctypes.c_int * self.count)()
        r = load().randutv_batched_plan_run(self.handle, st, _stream_handle(stream))
        return r, list(st)

    def close(self):
        if getattr(self, "handle", None):
            load().randutv_batched_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def randutv_svd_small_noalloc(w, R, ldr, D, Us, Vs, stream=None) -> int:
    """randutv_svd_small_noalloc of the C ABI (device buffers; allocates nothing)."""
    return load().randutv_svd_small_noalloc(w, _ptr(R), ldr, _ptr(D), _ptr(Us), _ptr(Vs), _stream_handle(stream))


# ---------------------------------------------------------------- learned q
def _f32(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _i32(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def randutv_learnq_model_floats() -> int:
    return int(load().randutv_learnq_model_floats())


def randutv_factor_learnedq(m, n, A, lda, b, model, seed, U, T, V, q_used=None, prec=RANDUTV_FP64, stream=None):
    """randutv_factor_learnedq_ex of the C ABI; model: float32 array or None; returns (status, q_used list)."""
    import numpy as np
    nb = -(-n // b) if n > 0 else 0
    qu, qp = _i32(np.zeros(max(nb, 1), dtype=np.int32))
    mp = None
    if model is not None:
        mk, mp = _f32(model)
    r = load().randutv_factor_learnedq_ex(m, n, _ptr(A), lda, b, mp, seed, _ptr(U), _ptr(T), _ptr(V), qp, prec,
                                          _stream_handle(stream))
    return r, list(qu[:nb])


def randutv_learnq_trace(m, n, A, lda, b, seed, T, max_blocks=None, candidates=False, prec=None, stride=1):
    """randutv_learnq_trace (or, with prec / stride, randutv_learnq_trace_ex) of the C ABI
    -> (status, features (k x 16), labels (k,), candidates (k x 4 x b) or None)."""
    import numpy as np
    mb = max_blocks if max_blocks is not None else max(-(-n // b), 1)
    f, fp = _f32(np.zeros((mb, 16), dtype=np.float32))
    y, yp = _i32(np.zeros(mb, dtype=np.int32))
    cand = np.zeros((mb, 4, b), dtype=np.float64) if candidates else None
    cp = cand.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if candidates else None
    cnt = ctypes.c_int64(0)
    if prec is None and stride == 1:
        r = load().randutv_learnq_trace(m, n, _ptr(A), lda, b, seed, _ptr(T), fp, yp, cp, mb, ctypes.byref(cnt))
    else:
        r = load().randutv_learnq_trace_ex(m, n, _ptr(A), lda, b, seed, _ptr(T), fp, yp, cp, mb, ctypes.byref(cnt),
                                           RANDUTV_FP64 if prec is None else prec, stride)
    k = cnt.value
    return r, f[:k].copy(), y[:k].copy(), (cand[:k].copy() if candidates else None)


def randutv_learnq_train(X, y, model, epochs, lr=1e-3, wd=0.0):
    """randutv_learnq_train of the C ABI -> (status, trained model, loss history)."""
    import numpy as np
    X, xp = _f32(X)
    y, yp = _i32(y)
    mk, mp = _f32(np.array(model, dtype=np.float32))
    hist, hp = _f32(np.zeros(max(epochs, 1), dtype=np.float32))
    r = load().randutv_learnq_train(xp, yp, len(y), epochs, lr, wd, mp, hp)
    return r, mk, hist[:epochs]


def randutv_learnq_grad(X, y, model):
    """randutv_learnq_grad of the C ABI -> (status, gradient, loss)."""
    import numpy as np
    X, xp = _f32(X)
    y, yp = _i32(y)
    mk, mp = _f32(model)
    g, gp = _f32(np.zeros(len(mk), dtype=np.float32))
    loss = ctypes.c_float(0.0)
    r = load().randutv_learnq_grad(xp, yp, len(y), mp, gp, ctypes.byref(loss))
    return r, g, float(loss.value)


def randutv_learnq_predict(model, X):
    """randutv_learnq_predict of the C ABI -> (status, probabilities N x 4)."""
    import numpy as np
    X, xp = _f32(X)
    mk, mp = _f32(model)
    pr, pp = _f32(np.zeros((X.shape[0], 4), dtype=np.float32))
    r = load().randutv_learnq_predict(mp, xp, X.shape[0], pp)
    return r, pr


QNET_PATH = os.path.join(_HERE, "qnet.f32")


def load_qnet(path: str = QNET_PATH):
    """Trained learned-q network (float32 parameters) shipped with the package, or None."""
    import numpy as np
    if not os.path.exists(path):
        return None
    return np.fromfile(path, dtype=np.float32)


# ---------------------------------------------------------------- conveniences
def colmajor_empty(rows, cols, device="cuda"):
    """Uninitialised FP64 column-major (rows x cols) CUDA tensor (a transposed view)."""
    import torch

    return torch.empty((cols, rows), dtype=torch.float64, device=device).t()


def is_colmajor(x) -> bool:
    rows, cols = x.shape
    if x.numel() == 0:
        return True
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


def factor_opt(A, b: int, q: int, seed: int = 0, want_uv: bool = True, prec: int = RANDUTV_FP64, stream=None,
               stop_after: int = -1, rank_tol: float = 0.0, qr_first: bool = False, check: bool = True):
    """randutv_factor_opt on a column-major FP64 CUDA tensor -> (U, T, V, cols_done, rank)."""
    m, n = A.shape
    if not is_colmajor(A):
        raise ValueError("A must be column-major (e.g. a transposed contiguous tensor)")
    T = colmajor_empty(m, n, A.device)
    U = colmajor_empty(m, m, A.device) if want_uv else None
    V = colmajor_empty(n, n, A.device) if want_uv else None
    lda = A.stride(1) if n > 1 else max(m, 1)
    o = randutv_options(prec=prec, stream=stream, stop_after=stop_after, rank_tol=rank_tol, qr_first=qr_first)
    st = randutv_factor_opt(m, n, A, max(lda, m, 1), b, q, seed, U, T, V, o)
    if check and st != RANDUTV_OK:
        raise RandUTVError(st, "randutv_factor_opt")
    return U, T, V, int(o.cols_done), int(o.rank)


def resume(U, T, V, b: int, q: int, seed: int, start_col: int, prec: int = RANDUTV_FP64, stream=None,
           stop_after: int = -1, rank_tol: float = 0.0, check: bool = True):
    """Continue the partial factorization held in (U, T, V) (column-major CUDA
    tensors, updated in place) from column start_col -> (cols_done, rank)."""
    m, n = T.shape
    o = randutv_options(prec=prec, stream=stream, stop_after=stop_after, rank_tol=rank_tol, start_col=start_col)
    st = randutv_factor_opt(m, n, None, max(m, 1), b, q, seed, U, T, V, o)
    if check and st != RANDUTV_OK:
        raise RandUTVError(st, "randutv_factor_opt (resume)")
    return int(o.cols_done), int(o.rank)

"""Benchmark of the GB300 randUTV library on the paper-shaped 16000 x 16000 workload.

One step = one complete factorization A = U T V^T (every block step: sketch,
QR of the sketch, right WY update, panel QR, left WY update, b x b SVD) of a
16000 x 16000 FP64 matrix with the gap spectrum, b = 128, q = 2, U and V formed.
The default path computes every FP64 product emulated on the BF16 tensor
cores (RANDUTV_FP64_EMULATED); one plain-FP64 (DMMA) factorization of the same
matrix is timed beside it for the ratio (`vs_plain_fp64`).
value = whole-job effective TFLOP/s from the fixed randUTV flop count F (below),
summed over ranks (one independent factorization per GPU: replicas, weak
scaling).  Prints ONE JSON line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--n 16000] [--b 128] [--q 2] [--prec emul|emul_bf16|fp64|bf16|fp16]
                    [--workload single|batched] [--no-e2e] [--no-cpu] [--no-compare]

--impl reference times the CPU oracle (the plain FP64 randUTV used as the
parity reference) on the host cores, each step a bounded sample of the same
workload (the same spectrum, b and q at n = 1536).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "randUTV s/factorization & TFLOP/s at n=16000: mixed/learned-q vs FP64, % peak"
# digit products per emulated FP64 product (8 digits, the pairs with s + t <= 7, 0-based)
SIDE_STREAM_CLASSES = ("gemm_accumulate_merge", "gemm_svdapply")  # product classes run on the side stream
OZ_PAIRS = 36
DTYPES = {"fp64": "f64", "bf16": "f64+bf16-sketch", "fp16": "f64+fp16-sketch",
          "emul": "f64 (products emulated on bf16 tensor cores)",
          "emul_bf16": "f64 (products emulated on bf16 tensor cores)+bf16-sketch"}


E2E_STEPS = 2   # timed end-to-end calls after one untimed call

def measured_peak(key: str, fallback: float) -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return fallback


# ncu: 222.2 MB of DRAM traffic for the 4.295 GFLOP rank-128 update launch (4096^2)
GEMM_F64_DRAM_BYTES_PER_FLOP = 222.2e6 / (2.0 * 4096 * 4096 * 128)
# ncu: 531 MB of DRAM traffic for the three emulated products of the 4096^2
# right update (8.72 GFLOP of FP64-equivalent work)
OZ_DRAM_BYTES_PER_FP64_FLOP = 531.0e6 / 8.72e9


def randutv_flops(m: int, n: int, b: int, q: int, uv: bool = True) -> float:
    """Fixed leading-order flop count F of blocked randUTV (the paper gives none).

    Summed over the sketch steps i (n' = n - i b > b), with m' = m - i b:
      2(1+2q) m' n' b    sketch and power iteration (Sec. 3.2.1)
      4 m n' b           right WY update of T(:, J2), all m rows (Sec. 5.4)
      4 m' (n'-b) b      left WY update of T22(:, b+1:) (Sec. 3.2.2)
      4 n n' b, 4 m m' b right updates of V and U (when formed)
      2 (m'+n') b^2      the two Householder panels
    The final block (n' <= b) adds 2 m' n'^2 (+ 4 m m' n' for U).
    """
    F = 0.0
    i = 0
    while True:
        mp, np_ = m - i * b, n - i * b
        if np_ <= 0:
            break
        if np_ <= b:
            F += 2.0 * mp * np_ * np_ + (4.0 * m * mp * np_ if uv else 0.0)
            break
        F += 2.0 * (1 + 2 * q) * mp * np_ * b + 4.0 * m * np_ * b + 4.0 * mp * (np_ - b) * b
        if uv:
            F += 4.0 * n * np_ * b + 4.0 * m * mp * b
        F += 2.0 * (mp + np_) * b * b
        i += 1
    return F


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, flag in zip(names, parts[4:8]):
                if flag.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(n: int, b: int, q: int, kind: str, reps: int = 1):
    """Time the CPU oracle on one n x n sample of the workload -> (TFLOP/s, seconds, threads)."""
    import oracle
    import synthetic

    A = synthetic.test_matrix(n, n, kind, 1, 2)
    oracle.build()
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.randutv(A, b, q, 0)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return randutv_flops(n, n, b, q) / best / 1e12, best, oracle.num_threads()


def blas_randutv(A, b: int, q: int, seed: int, gaussian, want_uv: bool = True):
    """Blocked randUTV on the host's BLAS and LAPACK: the CPU comparison run.

    It follows the steps of Sec. 3.2 in the Householder form the GPU library
    uses, on one node: the same Gaussian draws (``gaussian(seed, step, rows,
    cols)``), Householder QRs with LAPACK's sign rule (dgeqrf through numpy)
    and their compact WY factor (Sec. 2.3), right WY updates over all m rows,
    left WY updates, and the b x b SVD (LAPACK dgesdd) with the canonical sign
    (the entry of largest modulus of each right singular vector positive).
    Everything goes through numpy, so one BLAS thread pool serves every call
    and the products use every core.  Returns (U, T, V); U and V are None when
    want_uv is False.
    """
    import numpy as np

    def fmm(X, Y):  # X @ Y in column-major order, so updates of T, U, V run contiguously
        return (Y.T @ X.T).T

    def hqr(X):  # Householder QR -> (W unit lower, Tf upper with Q = I - W Tf W^T, R)
        h, tau = np.linalg.qr(X, mode="raw")
        f = h.T
        k = X.shape[1]
        W = np.tril(f, -1)[:, :k] + np.eye(X.shape[0], k)
        Gm = fmm(W.T, W)
        Tf = np.zeros((k, k))
        for j in range(k):
            Tf[:j, j] = -tau[j] * (Tf[:j, :j] @ Gm[:j, j])
            Tf[j, j] = tau[j]
        return np.asfortranarray(W), Tf, np.triu(f[:k, :k])

    m, n = A.shape
    T = np.array(A, dtype=np.float64, order="F")
    U = np.eye(m, order="F") if want_uv else None
    V = np.eye(n, order="F") if want_uv else None
    k0, step = 0, 0
    while k0 < n:
        mp, np_ = m - k0, n - k0
        if np_ > b:   # sketch step (Sec. 3.2.1) and right update with V_alpha
            w = b
            T22 = T[k0:, k0:]
            Y = fmm(T22.T, gaussian(seed, step, mp, b))
            for _ in range(q):
                Y = fmm(T22.T, fmm(T22, Y))
            W, Tf, _ = hqr(Y)
            T[:, k0:] -= fmm(fmm(fmm(T[:, k0:], W), Tf), W.T)
            if want_uv:
                V[:, k0:] -= fmm(fmm(fmm(V[:, k0:], W), Tf), W.T)
        else:         # final block: no sketch
            w = np_
        # panel QR (Sec. 3.2.2), left update of T22 and right update of U
        W, Tf, R = hqr(T[k0:, k0:k0 + w])
        if np_ > w:
            C = T[k0:, k0 + w:]
            C -= fmm(W, fmm(Tf.T, fmm(W.T, C)))
        if want_uv:
            U[:, k0:] -= fmm(fmm(fmm(U[:, k0:], W), Tf), W.T)
        # b x b SVD (Sec. 3.2.3), canonical sign, and its application
        Us, D, VsT = np.linalg.svd(R)
        Vs = VsT.T
        piv = np.argmax(np.abs(Vs), axis=0)
        sgn = np.where(Vs[piv, np.arange(w)] < 0.0, -1.0, 1.0)
        Us, Vs = Us * sgn, Vs * sgn
        if k0 > 0:
            T[:k0, k0:k0 + w] = fmm(T[:k0, k0:k0 + w], Vs)
        if np_ > w:
            T[k0:k0 + w, k0 + w:] = fmm(Us.T, T[k0:k0 + w, k0 + w:])
        T[k0:, k0:k0 + w] = 0.0
        T[k0:k0 + w, k0:k0 + w] = np.diag(D)
        if want_uv:
            V[:, k0:k0 + w] = fmm(V[:, k0:k0 + w], Vs)
            U[:, k0:k0 + w] = fmm(U[:, k0:k0 + w], Us)
        k0 += w
        step += 1
    return U, T, V


def cpu_blas_sample(n: int, b: int, q: int, kind: str):
    """Time blas_randutv on one n x n sample of the workload -> (TFLOP/s, seconds, cores)."""
    import oracle
    import synthetic

    A = synthetic.test_matrix(n, n, kind, 1, 2)
    oracle.build()
    t0 = time.perf_counter()
    blas_randutv(A, b, q, 0, oracle.gaussian)
    dt = time.perf_counter() - t0
    return randutv_flops(n, n, b, q) / dt / 1e12, dt, len(os.sched_getaffinity(0))


# The BLAS-based CPU comparison at the full size takes minutes, so it is
# measured once (python bench.py --cpu-blas-full) and recorded here.
CPU_BLAS_FULL_RECORD = os.path.join(ROOT, "cpu_blas_full_size.json")


def run_cpu_blas_full(args):
    """One blas_randutv factorization of the full-size workload on the host
    cores; the matrix is built on the GPU with the bench's own recipe and copied
    to the host.  Writes CPU_BLAS_FULL_RECORD and prints it."""
    import datetime

    import numpy as np
    import torch

    import oracle
    import synthetic

    n = args.n
    m = args.m if args.m > 0 else n
    A, _ = synthetic.test_matrix_device(m, n, args.spectrum, 1, 2, device=torch.device("cuda", 0))
    Ah = np.asfortranarray(A.cpu().numpy())
    del A
    oracle.build()
    t0 = time.perf_counter()
    blas_randutv(Ah, args.b, args.q, 0, oracle.gaussian)
    dt = time.perf_counter() - t0
    rec = {"value": randutv_flops(m, n, args.b, args.q) / dt / 1e12, "unit": "TFLOP/s", "seconds": dt,
           "cores": len(os.sched_getaffinity(0)),
           "kind": "blocked randUTV on numpy's BLAS/LAPACK (bench.blas_randutv)",
           "sample": "one %dx%d %s-spectrum factorization (b=%d, q=%d, U and V formed): the full workload size"
                     % (m, n, args.spectrum, args.b, args.q),
           "command": "python bench.py --cpu-blas-full --n %d --b %d --q %d --spectrum %s"
                      % (n, args.b, args.q, args.spectrum),
           "measured_utc": datetime.datetime.utcnow().strftime("%Y-%m-%dT%H:%M:%SZ")}
    with open(CPU_BLAS_FULL_RECORD, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec), flush=True)


def cpu_blas_full_record(m: int, n: int, b: int, q: int, spectrum: str):
    """The recorded full-size BLAS CPU run for this workload, or None."""
    try:
        with open(CPU_BLAS_FULL_RECORD) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    want = "one %dx%d %s-spectrum factorization (b=%d, q=%d" % (m, n, spectrum, b, q)
    if not rec.get("sample", "").startswith(want):
        return None
    rec["source"] = "recorded by a separate run of its command (minutes of CPU time), not measured in this run"
    return rec


def diag_quality(d, sigma, b: int) -> dict:
    """How closely |T_ii| tracks the prescribed singular values sigma_i.

    The median of r = |T_ii| / sigma_i alone can land in a run of repeated
    sigma (the gap spectrum's sigma = 1 cluster, found exactly), so the
    spread |r - 1| is reported beside it.
    """
    import numpy as np

    r = np.asarray(d, dtype=np.float64) / np.asarray(sigma, dtype=np.float64)
    dev = np.abs(r - 1.0)
    return {"Tii_over_sigma_median": float(np.median(r)),
            "Tii_over_sigma_median_abs_dev": float(np.median(dev)),
            "Tii_within_5pct_of_sigma": float((dev <= 0.05).mean()),
            "Tii_over_sigma_first_block_max_dev": float(dev[:b].max())}


# The CPU oracle arm (--impl reference) times a bounded sample of the workload
# per step: the same spectrum, b and q at this size.
REF_SAMPLE_N = 1536


def diag_vs_plain(d_run, d_64, sigma) -> dict:
    """Index-by-index comparison of two diagonals of T for the same matrix and seed.

    r_i = |T_ii| / sigma_i of the timed run against the plain FP64 run.  An
    index passes when r_i is within 5% of the FP64 ratio, or closer to 1 than
    it.  Only sigma_i above the FP64 noise floor 1e3 2^-53 sigma_1 count (below
    it both diagonals are rounding).  Indices that fail are listed (up to 20).
    """
    import numpy as np

    d_run = np.asarray(d_run, dtype=np.float64)
    d_64 = np.asarray(d_64, dtype=np.float64)
    sg = np.asarray(sigma, dtype=np.float64) if sigma is not None else d_64
    keep = sg > 1e3 * 2.0 ** -53 * sg[0]
    idx = np.nonzero(keep)[0]
    r_run, r_64 = d_run[keep] / sg[keep], d_64[keep] / sg[keep]
    dev = np.abs(r_run / r_64 - 1.0)
    ok = (dev <= 0.05) | (np.abs(np.log(r_run)) <= np.abs(np.log(r_64)))
    bad = idx[~ok]
    return {"indices_compared": int(keep.sum()), "noise_floor": "sigma_i > 1e3 2^-53 sigma_1",
            "max_dev": float(dev.max()) if dev.size else None,
            "median_dev": float(np.median(dev)) if dev.size else None,
            "frac_within_5pct": float((dev <= 0.05).mean()) if dev.size else None,
            "frac_within_5pct_or_closer_to_sigma": float(ok.mean()) if dev.size else None,
            "failing_indices": [{"i": int(i), "sigma": float(sg[i]), "Tii": float(d_run[i]),
                                 "Tii_fp64": float(d_64[i])} for i in bad[:20]],
            "failing_count": int(bad.size)}


def workload_config(args, m: int, n: int, F: float, world: int) -> dict:
    """The `config` object of both arms: the single-matrix workload timed.

    Both arms print the same object; `reference_sample` states the size the
    CPU oracle arm actually factors per step."""
    return {"workload": "randUTV %s %dx%d, %s spectrum, b=%d, %s, U and V formed%s" %
                        (args.prec.upper(), m, n, args.spectrum, args.b,
                         "learned q (fallback q=%d)" % args.q if args.learnedq else "q=%d" % args.q,
                         ", Householder QR first" if getattr(args, "qr_first", False) else ""),
            "m": m, "n": n, "b": args.b, "q": args.q, "spectrum": args.spectrum, "precision": args.prec,
            "flops_per_factorization": F,
            "l2": "inputs larger than L2 (A, T, U, V are %.2f GB each at m = n)" % (8e-9 * m * n),
            "parallelism": "replicas x%d" % world,
            "reference_sample": "the CPU oracle arm factors a %dx%d sample of this workload (same spectrum, b, q) "
                                "per step, not the full size" % (REF_SAMPLE_N, REF_SAMPLE_N)}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import oracle
    import synthetic

    n_s = REF_SAMPLE_N
    A = synthetic.test_matrix(n_s, n_s, args.spectrum, 1, 2)
    oracle.build()
    for _ in range(args.warmup):
        oracle.randutv(A, args.b, args.q, 0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.randutv(A, args.b, args.q, 0)
    dt = (time.perf_counter() - t0) / args.steps
    F = randutv_flops(n_s, n_s, args.b, args.q)
    val = F / dt / 1e12
    sample = "oracle (plain C, OpenMP, FP64) on a %dx%d %s-spectrum matrix, b=%d, q=%d, U and V formed; " \
             "one factorization per step" % (n_s, n_s, args.spectrum, args.b, args.q)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, args.m if args.m > 0 else args.n, args.n,
                                  randutv_flops(args.m if args.m > 0 else args.n, args.n, args.b, args.q), world),
        "sample": {"m": n_s, "n": n_s, "b": args.b, "q": args.q, "spectrum": args.spectrum,
                   "flops_per_factorization": F},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def measure_fp64_peak(torch, dev) -> float:
    """cuBLAS DGEMM 8192^3 throughput (TFLOP/s), the FP64 tensor denominator."""
    n = 8192
    a = torch.randn(n, n, device=dev, dtype=torch.float64)
    bm = torch.randn(n, n, device=dev, dtype=torch.float64)
    c = a @ bm
    torch.cuda.synchronize()
    best = None
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ bm
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, bm, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def run_gb300(args, rank: int, world: int, local_rank: int):
    import torch

    import paper_2104_05782_gb300 as rutv
    import synthetic
    from paper_2104_05782_gb300 import build as rbuild

    rbuild.build()
    rutv.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    n = args.n
    m = args.m if args.m > 0 else n
    b, q = args.b, args.q
    prec = {"fp64": rutv.RANDUTV_FP64, "bf16": rutv.RANDUTV_SKETCH_BF16,
            "fp16": rutv.RANDUTV_SKETCH_FP16_SCALED, "emul": rutv.RANDUTV_FP64_EMULATED,
            "emul_bf16": rutv.RANDUTV_EMULATED_SKETCH_BF16}[args.prec]
    F = randutv_flops(m, n, b, q)
    A, sigma = synthetic.test_matrix_device(m, n, args.spectrum, 1 + 2 * rank, 2 + 2 * rank, device=dev)
    torch.cuda.synchronize()
    fp64_peak = measure_fp64_peak(torch, dev)

    T = rutv.colmajor_empty(m, n, dev)
    U = rutv.colmajor_empty(m, m, dev)
    V = rutv.colmajor_empty(n, n, dev)
    stream = torch.cuda.current_stream(dev)
    opt = None
    if args.qr_first:
        opt = rutv.randutv_options(prec=prec, stream=stream, qr_first=True)
        ws_bytes = rutv.randutv_workspace_size_opt(m, n, b, opt)
    else:
        ws_bytes = rutv.randutv_workspace_size(m, n, b, prec)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
    if opt is not None:
        opt.workspace, opt.ws_bytes = ws.data_ptr(), ws_bytes

    qnet = rutv.load_qnet() if args.learnedq else None
    q_used = []

    def step():
        if args.learnedq:
            st, qu = rutv.randutv_factor_learnedq(m, n, A, m, b, qnet, 0, U, T, V, prec=prec, stream=stream)
            q_used[:] = qu
        elif opt is not None:
            st = rutv.randutv_factor_opt(m, n, A, m, b, q, 0, U, T, V, opt)
        else:
            st = rutv.randutv_factor_ex(m, n, A, m, b, q, 0, U, T, V, prec, stream, ws, ws_bytes, -1, None)
        if st != rutv.RANDUTV_OK:
            raise rutv.RandUTVError(st, "randutv_factor")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else local_rank)
    sampler.start()
    rutv.randutv_trace_reset()
    rutv.randutv_trace_enable(True)
    launches0 = rutv.randutv_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    launches = rutv.randutv_launch_count() - launches0
    rutv.randutv_trace_enable(False)
    trace = rutv.randutv_trace_read()
    clocks = sampler.stop()
    if dist:
        t = torch.tensor([elapsed_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / args.steps
    value = world * F / (ms_per_step * 1e-3) / 1e12

    # quality of this run (not timed): diagonal of T against the prescribed spectrum
    d = torch.diagonal(T).abs().cpu().numpy()
    d_primary = d.copy()
    quality = None
    if sigma is not None:
        quality = diag_quality(d, sigma, b)

    # dominant kernel: the FP64 products (class names "gemm_*") on the main
    # stream.  The side stream's products (the small-SVD application and the
    # merges of the U/V groups) run concurrently with main-stream products, so
    # their event times include time the two streams share: they are left out
    # (about 1% of the product flops).
    main = {k: v for k, v in trace.items() if k.startswith("gemm") and k not in SIDE_STREAM_CLASSES}
    g_ms = sum(v["ms"] for v in main.values())
    g_fl = sum(v["flops"] for v in main.values())
    g_launch = sum(v["scopes"] for v in main.values())
    tot_ms = sum(v["ms"] for v in trace.values())
    if args.prec in ("emul", "emul_bf16"):
        # k_oz_gemm executes OZ_PAIRS BF16 digit products per FP64 product
        # (plus its digit split); its roofline is that BF16 tensor work against
        # the measured BF16 peak
        bf_fl = OZ_PAIRS * g_fl
        achieved = bf_fl / (g_ms * 1e-3) / 1e12 if g_ms > 0 else None
        bf16_peak = measured_peak("bf16_tflops", 1917.9)
        roofline = {
            "kernel": "k_oz_gemm (FP64 product emulated by %d BF16 digit products on tcgen05, "
                      "with its digit split)" % OZ_PAIRS,
            "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": (achieved / bf16_peak) if achieved else None,
            "traffic": OZ_DRAM_BYTES_PER_FP64_FLOP * g_fl / max(g_launch, 1),
            "traffic_source": "ncu dram__bytes_read+write of k_oz_gemm on the 4096^2 right update (0.061 B per "
                              "FP64-equivalent flop), scaled by the average work per launch",
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured",
            "fp64_equivalent_tflops": g_fl / (g_ms * 1e-3) / 1e12 if g_ms > 0 else None,
            "launches": g_launch, "share_of_traced_time": g_ms / tot_ms if tot_ms else None,
            "share_of_step_time": g_ms / (args.steps * ms_per_step) if ms_per_step else None,
            "avg_flops_per_launch": bf_fl / max(g_launch, 1), "avg_ms_per_launch": g_ms / max(g_launch, 1),
        }
    else:
        achieved = g_fl / (g_ms * 1e-3) / 1e12 if g_ms > 0 else None
        roofline = {
            "kernel": "k_gemm_f64 (FP64 mma.sync m8n8k4, with its split-K reduce)",
            "bound": "tensor", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": (achieved / fp64_peak) if achieved else None,
            # DRAM bytes per flop of one ncu-captured launch of this kernel (the
            # 4096^2 rank-128 update) times the average flops of a launch here
            "traffic": GEMM_F64_DRAM_BYTES_PER_FLOP * g_fl / max(g_launch, 1),
            "traffic_source": "ncu dram__bytes_read+write of k_gemm_f64 on the 4096^2 case (0.0518 B/flop), "
                              "scaled by the average flops per launch",
            "peak_source": "cuBLAS DGEMM 8192^3 measured in this run (MEASURED_PEAKS.json has no FP64 entry)",
            "launches": g_launch, "share_of_traced_time": g_ms / tot_ms if tot_ms else None,
            "share_of_step_time": g_ms / (args.steps * ms_per_step) if ms_per_step else None,
            "avg_flops_per_launch": g_fl / max(g_launch, 1),
            "avg_ms_per_launch": g_ms / max(g_launch, 1),
        }
    breakdown = {k: {"ms": round(v["ms"] / args.steps, 3), "launches": v["kernels"] // args.steps}
                 for k, v in sorted(trace.items(), key=lambda kv: -kv[1]["ms"])}

    # quality against a reference precision (same matrix, same seed)
    ref_quality = None
    if args.ref_prec or args.learnedq:
        import numpy as np
        rp = {"": prec, "fp64": rutv.RANDUTV_FP64, "emul": rutv.RANDUTV_FP64_EMULATED}[args.ref_prec]
        d_run = torch.diagonal(T).abs().cpu().numpy()
        wsr_bytes = rutv.randutv_workspace_size(m, n, b, rp)
        wsr = torch.empty(max(wsr_bytes, 1), dtype=torch.uint8, device=dev)
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        r0.record(stream)
        st = rutv.randutv_factor_ex(m, n, A, m, b, q, 0, U, T, V, rp, stream, wsr, wsr_bytes, -1, None)
        r1.record(stream)
        torch.cuda.synchronize()
        if st != rutv.RANDUTV_OK:
            raise rutv.RandUTVError(st, "randutv_factor_ex (reference)")
        d_ref = torch.diagonal(T).abs().cpu().numpy()
        del wsr
        keep = (sigma > 1e3 * 2.0 ** -53 * sigma[0]) if sigma is not None else (d_ref > 1e3 * 2.0 ** -53 * d_ref[0])
        sg = sigma if sigma is not None else d_ref
        r_run, r_ref = d_run[keep] / sg[keep], d_ref[keep] / sg[keep]
        dev_ = np.abs(r_run / r_ref - 1.0)
        ok = (dev_ <= 0.05) | (np.abs(np.log(r_run)) <= np.abs(np.log(r_ref)))
        ref_quality = {"reference": ("fixed q=%d, " % q if args.learnedq else "") +
                       {"": args.prec, "fp64": "fp64", "emul": "emul"}[args.ref_prec],
                       "reference_s_per_factorization": r0.elapsed_time(r1) / 1e3,
                       "Tii_ratio_max_dev": float(dev_.max()), "Tii_ratio_median_dev": float(np.median(dev_)),
                       "frac_within_5pct_or_better": float(ok.mean())}
        if args.learnedq:
            ref_quality["q_used"] = [int(x) for x in q_used]
            ref_quality["power_iterations"] = int(sum(x for x in q_used if x >= 0))
            ref_quality["power_iterations_fixed_q"] = int(q * sum(1 for x in q_used if x >= 0))

    # the plain FP64 path (DMMA products) on the same matrix, once, for the time ratio
    compare = None
    if not args.no_compare and args.prec != "fp64":
        ws64_bytes = rutv.randutv_workspace_size(m, n, b, rutv.RANDUTV_FP64)
        ws64 = torch.empty(max(ws64_bytes, 1), dtype=torch.uint8, device=dev)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        c0.record(stream)
        st = rutv.randutv_factor_ex(m, n, A, m, b, q, 0, U, T, V, rutv.RANDUTV_FP64, stream, ws64, ws64_bytes, -1,
                                    None)
        c1.record(stream)
        torch.cuda.synchronize()
        if st != rutv.RANDUTV_OK:
            raise rutv.RandUTVError(st, "randutv_factor_ex (FP64)")
        t64 = c0.elapsed_time(c1) / 1e3
        compare = {"path": "plain FP64 (DMMA products), same matrix, one timed run after the primary runs",
                   "s_per_factorization": t64, "tflops": F / t64 / 1e12,
                   "speedup_of_primary": t64 / (ms_per_step / 1e3),
                   "Tii_vs_plain_fp64": diag_vs_plain(d_primary, torch.diagonal(T).abs().cpu().numpy(), sigma)}
        del ws64

    # QR first: the same precision without the QR, once, on the same matrix
    vs_direct = None
    if args.qr_first:
        wsd_bytes = rutv.randutv_workspace_size(m, n, b, prec)
        wsd = torch.empty(max(wsd_bytes, 1), dtype=torch.uint8, device=dev)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        c0.record(stream)
        st = rutv.randutv_factor_ex(m, n, A, m, b, q, 0, U, T, V, prec, stream, wsd, wsd_bytes, -1, None)
        c1.record(stream)
        torch.cuda.synchronize()
        if st != rutv.RANDUTV_OK:
            raise rutv.RandUTVError(st, "randutv_factor_ex (without the QR)")
        td = c0.elapsed_time(c1) / 1e3
        vs_direct = {"path": "the same precision without the QR first, one timed run",
                     "s_per_factorization": td, "speedup_of_qr_first": td / (ms_per_step / 1e3)}
        del wsd

    # end to end through the C ABI on HOST buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e and not args.qr_first:
        Ah = A.t().contiguous().cpu().pin_memory()   # row-major A^T == column-major A
        Th = torch.empty((n, m), dtype=torch.float64).pin_memory()
        Uh = torch.empty((m, m), dtype=torch.float64).pin_memory()
        Vh = torch.empty((n, n), dtype=torch.float64).pin_memory()
        del T, U, V, ws
        torch.cuda.empty_cache()
        if dist:
            dist.barrier()
        # one untimed call (the library's device buffers are allocated once and
        # cached), then E2E_STEPS timed calls, each with both copies inside
        st = rutv.randutv_factor_host(m, n, Ah, m, b, q, 0, Uh, Th, Vh, prec)
        if st != rutv.RANDUTV_OK:
            raise rutv.RandUTVError(st, "randutv_factor_host")
        t0 = time.perf_counter()
        for _ in range(E2E_STEPS):
            st = rutv.randutv_factor_host(m, n, Ah, m, b, q, 0, Uh, Th, Vh, prec)
            if st != rutv.RANDUTV_OK:
                raise rutv.RandUTVError(st, "randutv_factor_host")
        t_e2e = (time.perf_counter() - t0) / E2E_STEPS
        if dist:
            t = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        e2e = {"value": world * F / t_e2e / 1e12, "unit": "TFLOP/s", "s_per_factorization": t_e2e,
               "h2d_bytes_per_step": 8 * m * n, "d2h_bytes_per_step": 8 * (m * n + m * m + n * n),
               "steps": E2E_STEPS, "warmup": 1,
               "api": "randutv_factor_host (pinned host buffers; H2D of A and D2H of U, T, V inside every timed call)"}

    cpu = cpu_blas = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n_s = 2048
        val, secs, cores = cpu_oracle_sample(n_s, b, q, args.spectrum)
        cpu = {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
               "sample": "one %dx%d %s-spectrum factorization (b=%d, q=%d, U and V formed), %.1f s; "
                         "TFLOP/s from the same flop formula" % (n_s, n_s, args.spectrum, b, q, secs)}
        # the same method on the host's BLAS and LAPACK (a comparison run, not the checker)
        n_b = 4096
        try:
            bval, bsecs, bcores = cpu_blas_sample(n_b, b, q, args.spectrum)
            cpu_blas = {"value": bval, "unit": "TFLOP/s", "cores": bcores,
                        "kind": "blocked randUTV on numpy's BLAS/LAPACK (bench.blas_randutv)",
                        "sample": "one %dx%d %s-spectrum factorization (b=%d, q=%d, U and V formed), %.1f s"
                                  % (n_b, n_b, args.spectrum, b, q, bsecs)}
        except Exception as exc:  # report, never lose the bench line over the comparison run
            cpu_blas = {"error": "%s: %s" % (type(exc).__name__, exc)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "s_per_factorization": ms_per_step / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.prec], "data": "synthetic",
            "config": workload_config(args, m, n, F, world),
            "fp64_peak_tflops": fp64_peak,
            "pct_of_fp64_peak": 100.0 * (value / world) / fp64_peak,
            "vs_plain_fp64": compare,
            "vs_without_qr_first": vs_direct,
            "quality_vs_reference": ref_quality,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "cpu_baseline_blas": cpu_blas,
            "cpu_baseline_blas_full_size": cpu_blas_full_record(m, n, b, q, args.spectrum),
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "breakdown_ms_per_step": breakdown,
            "quality": quality,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def batched_shapes(count: int, seed: int = 0):
    """4096-matrix workload: n = round(exp(U[ln 32, ln 512])), 25% tall (m = 2n)."""
    import numpy as np
    g = np.random.default_rng(seed)
    n = np.rint(np.exp(g.uniform(np.log(32.0), np.log(512.0), count))).astype(int)
    tall = g.uniform(size=count) < 0.25
    m = np.where(tall, 2 * n, n)
    return [int(x) for x in m], [int(x) for x in n]


def run_batched(args, rank: int, world: int, local_rank: int):
    """One step = one replay of the whole batch (CUDA graph of one persistent launch)."""
    import torch

    import paper_2104_05782_gb300 as rutv
    import synthetic
    from paper_2104_05782_gb300 import build as rbuild

    rbuild.build()
    rutv.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2104_05782_gb300 import shard

    q = args.q
    ms_all, ns_all = batched_shapes(args.count)
    # the fixed batch is split over the ranks, longest-processing-time first
    mine = shard.lpt_partition([randutv_flops(a, b_, 32, q) for a, b_ in zip(ms_all, ns_all)], world)[rank]
    ms = [ms_all[k] for k in mine]
    ns = [ns_all[k] for k in mine]
    count = len(mine)
    A, T, U, V = [], [], [], []
    for j, k in enumerate(mine):
        a, _ = synthetic.test_matrix_device(ms[j], ns[j], "geometric8", 7 * k + 1, 7 * k + 2, device=dev)
        A.append(a)
        T.append(rutv.colmajor_empty(ms[j], ns[j], dev))
        U.append(rutv.colmajor_empty(ms[j], ms[j], dev))
        V.append(rutv.colmajor_empty(ns[j], ns[j], dev))
    seeds = list(mine)
    # the batched kernel runs FP64 products (DMMA) or, with --prec fp32, an FP32 sketch
    prec = rutv.RANDUTV_SKETCH_FP32 if args.prec == "fp32" else rutv.RANDUTV_FP64
    t0 = time.perf_counter()
    r, table = rutv.randutv_batched_autotune(ms, ns, A, ms, U, T, V, seeds, q, prec)
    t_tune = time.perf_counter() - t0
    if r != 0:
        raise rutv.RandUTVError(r, "randutv_batched_autotune")
    plan = rutv.BatchPlan(ms, ns, A, ms, U, T, V, seeds, q, prec, table)
    b_of = {}
    for line in table.strip().splitlines():
        f = line.split()
        if f[0] == "threads":
            continue
        lo, hi, tall, b = map(int, f[:4])
        b_of[(lo, hi, tall)] = b
    F = 0.0
    for k in range(count):
        b = next(bb for (lo, hi, tl), bb in b_of.items() if lo <= ns[k] <= hi and tl == (1 if ms[k] > ns[k] else 0))
        F += randutv_flops(ms[k], ns[k], b, q)
    for _ in range(args.warmup):
        plan.run()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    l0 = rutv.randutv_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    worst = 0
    for _ in range(args.steps):
        r, st = plan.run()
        worst = max(worst, r)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_step = e0.elapsed_time(e1) / args.steps
    launches = rutv.randutv_launch_count() - l0
    clocks = sampler.stop()
    if dist:
        t = torch.tensor([ms_step], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
        f = torch.tensor([F], device=dev, dtype=torch.float64)
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
        F = float(f.item())
    plan.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": F / (ms_step * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "s_per_batch": ms_step / 1e3,
            "higher_is_better": True, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "f64+fp32-sketch" if args.prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "batched randUTV, %d matrices, n log-uniform in [32, 512], 25%% with m = 2n, "
                                   "sigma_i = 10^(-8(i-1)/(n-1)), q=%d, U and V formed" % (args.count, q),
                       "count": args.count, "q": q, "parallelism": "LPT shard over %d ranks" % world, "autotune_table": table, "autotune_seconds": t_tune,
                       "flops_per_batch": F},
            "status_worst": worst, "gpu_launches": launches, "clocks": clocks}), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=16000)
    p.add_argument("--m", type=int, default=0, help="rows (default: n, square)")
    p.add_argument("--ref-prec", default="", choices=["", "fp64", "emul"],
                   help="also factor with this precision and report T_ii/sigma_i against it")
    p.add_argument("--learnedq", action="store_true",
                   help="primary path picks q per block with the shipped network (fixed q=2 timed beside it)")
    p.add_argument("--qr-first", action="store_true",
                   help="Householder QR of A first, then randUTV of its R (tall inputs); one timed "
                        "factorization of the default path on the same matrix is reported beside it")
    p.add_argument("--b", type=int, default=128)
    p.add_argument("--q", type=int, default=2)
    p.add_argument("--spectrum", default="gap")
    p.add_argument("--prec", default="emul", choices=["fp64", "bf16", "fp16", "fp32", "emul", "emul_bf16"])
    p.add_argument("--no-compare", action="store_true", help="skip the timed plain-FP64 (DMMA) factorization")
    p.add_argument("--workload", default="single", choices=["single", "batched"])
    p.add_argument("--count", type=int, default=4096)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-blas-full", action="store_true",
                   help="only time the BLAS-based CPU randUTV once at the full size and record it")
    args = p.parse_args()
    if args.workload == "single" and args.prec == "fp32":
        p.error("--prec fp32 (the FP32 sketch) applies to --workload batched only")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.cpu_blas_full:
        run_cpu_blas_full(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args, rank, world, local_rank)
    else:
        run_gb300(args, rank, world, local_rank)


if __name__ == "__main__":
    main()

"""Train the learned-q network on traces generated by the method itself (GPU).

1. Draws `--count` matrices with n log-uniform in [--nmin, --nmax] and a spectrum
   cycling through geometric (1 -> 1e-10), algebraic (1/i), gap (1 then 1e-3 ->
   1e-12), dense N(0,1), and two numerically low-rank ones (10^(-i/32) and
   10^(-i/128) down to 1e-15), where fewer power iterations suffice; training
   seeds 0..count-1 (held-out evaluation uses seeds from 10^6).
2. For each, randutv_learnq_trace_ex factors it along the q = 2 trajectory (T
   only, products emulated on the BF16 tensor cores) and records, at step 0 and
   every --stride-th step, the 16 features and the label: the smallest q whose
   block diagonal sigma(T22 Q1(q)) stays within 5% of q = 2's.
3. Trains the 16-64-64-4 network with randutv_learnq_train (full-batch Adam on
   the GPU, the library's own kernels), inputs standardised by the training
   mean / std, and writes the parameters to paper_2104_05782_gb300/qnet.f32
   plus a summary to qnet.json.

    python -m paper_2104_05782_gb300.learnq_train [--count 1000] [--nmin 1000] [--nmax 8000] [--stride 4]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def initial_parameters(seed, mu, sd):
    """He-initialised weights, zero biases, and the input standardisation (mu, sd)."""
    g = np.random.default_rng(seed)
    parts = [g.standard_normal(16 * 64) * math.sqrt(2.0 / 16), np.zeros(64),
             g.standard_normal(64 * 64) * math.sqrt(2.0 / 64), np.zeros(64),
             g.standard_normal(64 * 4) * math.sqrt(1.0 / 64), np.zeros(4), mu, sd]
    return np.concatenate(parts).astype(np.float32)


def main():
    import torch

    import paper_2104_05782_gb300 as rutv
    import synthetic
    from paper_2104_05782_gb300 import build

    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=1000)
    ap.add_argument("--stride", type=int, default=4)
    ap.add_argument("--nmin", type=int, default=1000)
    ap.add_argument("--nmax", type=int, default=8000)
    ap.add_argument("--b", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=os.path.join(HERE, "qnet.f32"))
    args = ap.parse_args()
    build.build()
    rutv.load()
    kinds = ["geometric10", "algebraic", "gap", "normal", "exp32", "exp128"]
    rng = np.random.default_rng(12345)
    feats, labels, sizes = [], [], []
    t0 = time.time()
    for k in range(args.count):
        n = int(round(math.exp(rng.uniform(math.log(args.nmin), math.log(args.nmax)))))
        kind = kinds[k % len(kinds)]
        A, _ = synthetic.test_matrix_device(n, n, kind, k, 10 ** 5 + k)
        T = rutv.colmajor_empty(n, n)
        r, F, y, _ = rutv.randutv_learnq_trace(n, n, A, n, args.b, k, T, prec=rutv.RANDUTV_FP64_EMULATED,
                                               stride=args.stride)
        if r != 0:
            raise rutv.RandUTVError(r, "randutv_learnq_trace")
        feats.append(F)
        labels.append(y)
        sizes.append(n)
        del A, T
        torch.cuda.empty_cache()
    X = np.concatenate(feats).astype(np.float32)
    y = np.concatenate(labels).astype(np.int32)
    t_trace = time.time() - t0
    mu = X.mean(axis=0)
    sd = X.std(axis=0) + 1e-3
    p0 = initial_parameters(0, mu, sd)
    r, p, hist = rutv.randutv_learnq_train(X, y, p0, args.epochs, lr=args.lr, wd=1e-4)
    if r != 0:
        raise rutv.RandUTVError(r, "randutv_learnq_train")
    _, pr = rutv.randutv_learnq_predict(p, X)
    acc = float(np.mean(np.argmax(pr, axis=1) == y))
    p.tofile(args.out)
    summary = {"matrices": args.count, "spectra": kinds, "stride": args.stride,
               "n_range": [args.nmin, args.nmax], "n_drawn": sizes, "b": args.b,
               "samples": int(len(y)), "label_counts": [int(np.sum(y == q)) for q in range(4)],
               "epochs": args.epochs, "final_loss": float(hist[-1]), "initial_loss": float(hist[0]),
               "train_accuracy": acc, "trace_seconds": t_trace}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()

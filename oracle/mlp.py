"""FP64 reference of the learned-q network (TEST INFRASTRUCTURE ONLY).

Plain numpy: forward pass, mean cross-entropy and its gradient by the chain
rule, for the 16 -> 64 -> 64 -> 4 GELU network whose parameters are stored as
W1[16][64] b1[64] W2[64][64] b2[64] W3[64][4] b3[4] mu[16] sd[16] (row-major,
inputs standardised as (x - mu) / sd).  Pinned by finite differences and by a
closed-form case in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import math

import numpy as np

NI, NH, NO = 16, 64, 4
SIZES = [("W1", NI * NH), ("b1", NH), ("W2", NH * NH), ("b2", NH), ("W3", NH * NO), ("b3", NO), ("mu", NI),
         ("sd", NI)]
NPARAM = sum(s for _, s in SIZES)
NTRAIN = NPARAM - 2 * NI

_erf = np.vectorize(math.erf)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, size in SIZES:
        out[name] = p[o:o + size]
        o += size
    out["W1"] = out["W1"].reshape(NI, NH)
    out["W2"] = out["W2"].reshape(NH, NH)
    out["W3"] = out["W3"].reshape(NH, NO)
    return out


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_prime(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(p, X):
    """-> (logits, cache) for X (N x 16)."""
    w = unpack(p)
    sd = np.where(w["sd"] > 0, w["sd"], 1.0)
    x = (np.asarray(X, dtype=np.float64) - w["mu"]) / sd
    z1 = x @ w["W1"] + w["b1"]
    h1 = gelu(z1)
    z2 = h1 @ w["W2"] + w["b2"]
    h2 = gelu(z2)
    logits = h2 @ w["W3"] + w["b3"]
    return logits, (x, z1, h1, z2, h2)


def softmax(logits):
    e = np.exp(logits - logits.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def loss(p, X, y):
    logits, _ = forward(p, X)
    P = softmax(logits)
    return float(-np.mean(np.log(P[np.arange(len(y)), y])))


def grad(p, X, y):
    """Gradient of the mean cross-entropy w.r.t. every parameter (mu, sd -> 0)."""
    w = unpack(p)
    logits, (x, z1, h1, z2, h2) = forward(p, X)
    N = len(y)
    d3 = softmax(logits)
    d3[np.arange(N), y] -= 1.0
    d3 /= N
    gW3 = h2.T @ d3
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ w["W3"].T) * gelu_prime(z2)
    gW2 = h1.T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ w["W2"].T) * gelu_prime(z1)
    gW1 = x.T @ d1
    gb1 = d1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, np.zeros(2 * NI)])


def init(seed: int = 0, mu=None, sd=None):
    """He-style random initial parameters with the given input standardisation."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal(NI * NH) * math.sqrt(2.0 / NI), np.zeros(NH),
             rng.standard_normal(NH * NH) * math.sqrt(2.0 / NH), np.zeros(NH),
             rng.standard_normal(NH * NO) * math.sqrt(1.0 / NH), np.zeros(NO),
             np.zeros(NI) if mu is None else np.asarray(mu, dtype=np.float64),
             np.ones(NI) if sd is None else np.asarray(sd, dtype=np.float64)]
    return np.concatenate(parts)

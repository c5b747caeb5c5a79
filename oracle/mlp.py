"""ORACLE -- test infrastructure only: the rank predictor's network in plain
FP64 numpy, written from its definition (it shares no code with the CUDA
library).  Only tests/ use it.

Network (the learned part of assembly; the paper has none): standardised
features x = (f - mu) / sd, h1 = relu(W1 x + b1) (64), h2 = relu(W2 h1 + b2)
(64), z = W3 h2 + b3 (6 classes), p = softmax(z); loss = mean over samples
of -log p[y].  The library's forward pass uses the weights rounded to FP16;
`round_fp16=True` applies the same rounding (round to nearest even) before
the FP64 arithmetic here.

Flat parameter layout: W1 (64 x 10, row-major), b1, W2 (64 x 64), b2,
W3 (6 x 64), b3; then mu (10) and sd (10).
"""
from __future__ import annotations

import numpy as np

NF, NH, NC = 10, 64, 6
SIZES = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NC, NH)), ("b3", (NC,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta: np.ndarray, round_fp16: bool = False) -> dict:
    """Split a flat vector (NPARAM weights, optionally + mu + sd) into arrays (FP64)."""
    theta = np.asarray(theta)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        w = theta[o:o + k].astype(np.float32)
        if round_fp16:
            w = w.astype(np.float16)
        out[name] = w.astype(np.float64).reshape(shape)
        o += k
    if theta.size >= NPARAM + 2 * NF:
        out["mu"] = theta[NPARAM:NPARAM + NF].astype(np.float64)
        out["sd"] = theta[NPARAM + NF:NPARAM + 2 * NF].astype(np.float64)
    else:
        out["mu"] = np.zeros(NF)
        out["sd"] = np.ones(NF)
    return out


def forward(P: dict, F: np.ndarray) -> dict:
    """All intermediate values for features F (n x NF)."""
    x = (np.asarray(F, dtype=np.float64) - P["mu"]) / P["sd"]
    a1 = x @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ P["W3"].T + P["b3"]
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    p = e / e.sum(axis=1, keepdims=True)
    return {"x": x, "a1": a1, "h1": h1, "a2": a2, "h2": h2, "p": p}


def loss(P: dict, F: np.ndarray, y: np.ndarray) -> float:
    p = forward(P, F)["p"]
    return float(-np.mean(np.log(p[np.arange(len(y)), y])))


def backward(P: dict, F: np.ndarray, y: np.ndarray) -> tuple[float, np.ndarray]:
    """Mean loss and its gradient with respect to the flat weights (NPARAM),
    by the chain rule through softmax cross-entropy and the two ReLU layers."""
    v = forward(P, F)
    n = len(y)
    onehot = np.zeros_like(v["p"])
    onehot[np.arange(n), y] = 1.0
    dz = (v["p"] - onehot) / n                 # d loss / d z
    dW3 = dz.T @ v["h2"]
    db3 = dz.sum(axis=0)
    da2 = (dz @ P["W3"]) * (v["a2"] > 0)       # through h2 = relu(a2)
    dW2 = da2.T @ v["h1"]
    db2 = da2.sum(axis=0)
    da1 = (da2 @ P["W2"]) * (v["a1"] > 0)
    dW1 = da1.T @ v["x"]
    db1 = da1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    L = float(-np.mean(np.log(v["p"][np.arange(n), y])))
    return L, g


def flat(P: dict) -> np.ndarray:
    return np.concatenate([P[name].ravel() for name, _ in SIZES])


def with_flat(P: dict, w: np.ndarray) -> dict:
    """P with its weights replaced by the flat FP64 vector w (no rounding)."""
    Q = dict(P)
    o = 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        Q[name] = np.asarray(w[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return Q

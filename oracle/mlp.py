"""FP64 CPU reference of the conditioning-set proposal network (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by the tests and the smoke check to pin the GPU
forward/backward kernels; the product path never imports it.

The paper has no learned component; this network is the proposal of the
spec design: a member score s(u, v, k) for every candidate k of an
ordered pair (u, v) at stage l, so that the enumeration of Algorithms 1/2 can
try the likeliest separating sets first.  Plain definitions:

    h1 = relu(W1 x + b1)        W1: 128 x 16
    h2 = relu(W2 h1 + b2)       W2: 128 x 128
    s  = w3 . h2 + b3
    loss = mean_r [ softplus(s_r) - y_r s_r ]        (binary cross-entropy on sigmoid(s))

Parameters are one flat vector in the order W1 (row-major), b1, W2 (row-major),
b2, w3, b3 -- 18817 values.
"""
from __future__ import annotations

import numpy as np

NF, NH = 16, 128
SIZES = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(theta, X, h1_store=None):
    """Scores s (rows,) and the activations (h1, h2, pre-activations).
    h1_store: optional map applied to h1 before the second layer reads it (the
    precision a network stores its hidden activations in; identity if None)."""
    P = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    if h1_store is not None:
        h1 = np.asarray(h1_store(h1), dtype=np.float64)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    s = h2 @ P["w3"] + P["b3"][0]
    return s, (a1, h1, a2, h2)


def softplus(s):
    return np.logaddexp(0.0, s)


def loss(theta, X, y, h1_store=None):
    s, _ = forward(theta, X, h1_store)
    return float(np.mean(softplus(s) - np.asarray(y, dtype=np.float64) * s))


def grad(theta, X, y, h1_store=None, dh_store=None) -> np.ndarray:
    """Gradient of loss() by the chain rule written out layer by layer (h1_store as
    in forward(): the second layer and its weight gradient use the stored h1).
    dh_store: optional map applied to the back-propagated signals dL/da2 and
    dL/da1 (after the ReLU masks) before anything reads them -- the precision a
    network stores them in for its gradient products (identity if None)."""
    P = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    s, (a1, h1, a2, h2) = forward(theta, X, h1_store)
    B = X.shape[0]
    ds = (1.0 / (1.0 + np.exp(-s)) - y) / B            # d loss / d s
    g = {}
    g["w3"] = h2.T @ ds
    g["b3"] = np.array([ds.sum()])
    dh2 = np.outer(ds, P["w3"]) * (a2 > 0)
    if dh_store is not None:
        dh2 = np.asarray(dh_store(dh2), dtype=np.float64)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ P["W2"]) * (a1 > 0)
    if dh_store is not None:
        dh1 = np.asarray(dh_store(dh1), dtype=np.float64)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(0)
    return pack(g)


def init(seed: int) -> np.ndarray:
    """He-uniform initial parameters drawn from a seeded generator (input side)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = {
        "W1": rng.uniform(-1, 1, (NH, NF)) * np.sqrt(6.0 / NF),
        "b1": np.zeros(NH),
        "W2": rng.uniform(-1, 1, (NH, NH)) * np.sqrt(6.0 / NH),
        "b2": np.zeros(NH),
        "w3": rng.uniform(-1, 1, NH) * np.sqrt(6.0 / NH),
        "b3": np.zeros(1),
    }
    return pack(parts)

"""Surrogate model of the tuning search, in FP64 -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the product never does.

The paper tunes its hyper-parameters with an external AutoML search (Sec. 4.4);
the GPU library replaces most of the full runs of that search with a small
regression network trained on the scores that full runs produce. This module
states that network plainly:

* the model: 30 inputs -> 256 ReLU -> 256 ReLU -> 1 linear output;
* its inputs are standardised per feature, x' = (x - mean) / std;
* the loss of a batch is the mean squared error, (1/B) sum_r (y_r - t_r)^2;
* the gradient is backpropagation written out layer by layer;
* the optimiser is Adam (Kingma and Ba, 2015) with bias correction.

The GPU keeps FP32 master weights and runs the products with their bfloat16
roundings (``bf16_round``) and FP32 accumulation; the parity tests feed this
module the same rounded weights.

Parameter layout (flat, FP32 on the GPU): W1 [30][256], b1 [256],
W2 [256][256], b2 [256], w3 [256], b3 [1] -- 73,985 values; W[i][j] is the
weight from input i to unit j.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 30, 256
LAYOUT = (("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("w3", (N_HID,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in LAYOUT)


def unpack(theta: np.ndarray) -> dict:
    """Views of the flat parameter vector, by name."""
    theta = np.asarray(theta)
    out, o = {}, 0
    for name, shape in LAYOUT:
        size = int(np.prod(shape))
        out[name] = theta[o:o + size].reshape(shape)
        o += size
    assert o == theta.size
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).ravel() for name, _ in LAYOUT])


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16 (8 significant bits), to nearest with ties
    to even, returned as FP64. The bfloat16 of an FP32 value is its upper 16
    bits after adding half a unit of the dropped part (plus one when the kept
    part is odd, so that exact halves go to the even neighbour)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def standardize(X: np.ndarray, mean: np.ndarray, std: np.ndarray) -> np.ndarray:
    return (np.asarray(X, np.float64) - mean) / std


def feature_scaling(X: np.ndarray):
    """Per-feature mean and population standard deviation of the training rows
    (a standard deviation below 1e-6 is replaced by 1: constant features pass
    through centred)."""
    X = np.asarray(X, np.float64)
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    return mean, np.where(std < 1e-6, 1.0, std)


def forward(theta: np.ndarray, X: np.ndarray):
    """y = w3 . relu(W2^T relu(W1^T x + b1) + b2) + b3 for every row x of X
    (already standardised). Returns y [B] and the activations for backprop."""
    p = unpack(theta)
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(theta: np.ndarray, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(theta, X)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Gradient of ``loss`` by the chain rule, output layer first."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    B = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, np.float64)) / B          # dL/dy
    g = {"b3": np.array([dy.sum()]), "w3": h2.T @ dy}
    dz2 = np.outer(dy, p["w3"]) * (z2 > 0)                   # through the second ReLU
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * (z1 > 0)                       # through the first ReLU
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return pack(g)


def adam_step(theta, m, v, g, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1): m and v are the running first and
    second moments, corrected by 1 - beta^step before the update."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v

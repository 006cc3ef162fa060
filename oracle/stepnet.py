"""FP64 oracle of the step network (TEST INFRASTRUCTURE ONLY; see
oracle/__init__.py): features, forward pass, mean-squared-error gradient and
the learned step, written out plainly in numpy.

Layout of the flat FP32 parameters: W1[8][64], b1[64], W2[64][64], b2[64],
w3[64], b3.  The GPU path runs the forward pass with BF16 copies of the
weights; `bf16` rounds FP32 values to BF16 (nearest, ties to even) so that
the oracle can use exactly the same weight values.
"""
from __future__ import annotations

import math

import numpy as np

IN, HID = 8, 64
N_PARAMS = IN * HID + HID + HID * HID + HID + HID + 1
MU = 398600.4418
RE = 6378.137


def bf16(x) -> np.ndarray:
    """Round FP32 values to BF16 (round to nearest, ties to even); returned
    as float64 holding the BF16 values exactly."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, round_weights: bool = True):
    p = np.asarray(params, np.float32).reshape(-1)
    assert p.size == N_PARAMS
    o = 0
    W1 = p[o:o + IN * HID].reshape(IN, HID); o += IN * HID
    b1 = p[o:o + HID]; o += HID
    W2 = p[o:o + HID * HID].reshape(HID, HID); o += HID * HID
    b2 = p[o:o + HID]; o += HID
    w3 = p[o:o + HID]; o += HID
    b3 = p[o]
    f = bf16 if round_weights else (lambda v: np.asarray(v, np.float64))
    return (f(W1), b1.astype(np.float64), f(W2), b2.astype(np.float64), f(w3),
            np.float64(b3))


def forward(params, X, round_weights: bool = True):
    """y = w3 . relu(W2^T relu(W1^T x + b1) + b2) + b3, in FP64."""
    W1, b1, W2, b2, w3, b3 = unpack(params, round_weights)
    X = np.asarray(X, np.float64)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ w3 + b3


def loss_and_grad(params, X, T, round_weights: bool = True):
    """Mean squared error over the samples and its gradient with respect to
    the flat parameters (by the chain rule, layer by layer)."""
    W1, b1, W2, b2, w3, b3 = unpack(params, round_weights)
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    n = len(X)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    r = y - T
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    d2 = np.outer(dy, w3) * (a2 > 0)
    g_W2 = h1.T @ d2
    g_b2 = d2.sum(0)
    d1 = (d2 @ W2.T) * (a1 > 0)
    g_W1 = X.T @ d1
    g_b1 = d1.sum(0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


def features(els) -> np.ndarray:
    """The eight per-object features, FP64 (see the library's definition)."""
    E = np.asarray(els, np.float64)
    a, e, inc = E[:, 0], E[:, 1], E[:, 2]
    hp = np.maximum(a * (1 - e) - RE, 1.0)
    ha = np.maximum(a * (1 + e) - RE, 1.0)
    P = 2 * math.pi * np.sqrt(a ** 3 / MU)
    s = np.sort(a)
    dens = np.searchsorted(s, a + 50.0, side="right") - np.searchsorted(s, a - 50.0, side="left") - 1
    return np.stack([np.log(a / RE), e, np.sin(inc), np.cos(inc), np.log(hp / 100.0),
                     np.log(ha / 100.0), np.log(P / 3600.0), np.log1p(np.maximum(dens, 0))], 1)


def learned_step_seconds(els, y) -> np.ndarray:
    """exp(y) clamped to [P/400, P/50]."""
    a = np.asarray(els, np.float64)[:, 0]
    P = 2 * math.pi * np.sqrt(a ** 3 / MU)
    return np.clip(np.exp(np.asarray(y, np.float64)), P / 400.0, P / 50.0)

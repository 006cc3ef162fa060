"""Learned per-object time steps: training data from the method's own sweeps,
a fitted cost model, and training with the library's step-network kernels.

Sweep: screen a population with every object on the period-fraction step
P/f for each f in MULTIPLIERS, recording per object its box count and the
overlapping box pairs it takes part in, and the screen's GPU time.  Cost
model: screen time ~ c_box * boxes + c_hit * box pairs, fitted by least
squares over the sweep.  Target of object i: log of P_i / f*, f* the
multiplier minimising c_box * boxes_i(f) + c_hit * pairs_i(f) / 2 (a pair's
cost is shared by its two objects).  All screening and training run in
libscd; this module only orchestrates them.
"""
from __future__ import annotations

import math

import numpy as np

from . import _binding as B

MULTIPLIERS = (50.0, 71.0, 100.0, 141.0, 200.0, 283.0, 400.0)
MU = 398600.4418


class StepNet:
    """A step network living on the GPU (see scd_stepnet_* in include/scd.h)."""

    def __init__(self, seed: int = 1, stream=None):
        import torch
        B.use_torch_allocator()
        self._stream = stream or torch.cuda.current_stream()
        self.handle = B.scd_stepnet_create(int(self._stream.cuda_stream), seed)

    @property
    def params(self) -> np.ndarray:
        return B.scd_stepnet_get_params(self.handle)

    @params.setter
    def params(self, p):
        B.scd_stepnet_set_params(self.handle, p)

    def forward(self, x):
        import torch
        x = x.contiguous()
        y = torch.empty(len(x), dtype=torch.float32, device=x.device)
        B.scd_stepnet_forward(self.handle, x.data_ptr(), len(x), y.data_ptr())
        return y

    def grad(self, x, t):
        import torch
        g = torch.zeros(B.SCD_STEPNET_PARAMS, dtype=torch.float32, device=x.device)
        loss = B.scd_stepnet_grad(self.handle, x.contiguous().data_ptr(),
                                  t.contiguous().data_ptr(), len(x), g.data_ptr())
        return loss, g

    def train_step(self, x, t, lr: float, weight_decay: float = 0.0) -> float:
        return B.scd_stepnet_train_step(self.handle, x.data_ptr(), t.data_ptr(), len(x), lr,
                                        weight_decay)

    def save(self, path: str):
        B.scd_stepnet_save(self.handle, path)

    def load(self, path: str):
        B.scd_stepnet_load(self.handle, path)

    def policy(self):
        return B.make_step_policy(B.SCD_STEP_LEARNED, stepnet=self.handle)

    def close(self):
        if getattr(self, "handle", None):
            B.scd_stepnet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def features(elements):
    """Per-object features (n x 8 float32, on the GPU)."""
    import torch
    d_el = torch.as_tensor(np.ascontiguousarray(elements, np.float64), device="cuda")
    f = torch.empty((len(elements), B.SCD_STEPNET_IN), dtype=torch.float32, device="cuda")
    B.scd_stepnet_features(d_el.data_ptr(), len(elements), f.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    return f


def sweep(elements, horizon_s: float, tick_s: float = 1.0, multipliers=MULTIPLIERS,
          mode: int = B.SCD_BOX_SPEED, count: str = "cells"):
    """Screen the population once per multiplier.  Returns a dict of arrays:
    boxes [F, n], pairs [F, n] (per object: its overlapping box pairs when
    count == "cells", its merged candidate pairs when count == "runs"; the
    latter stays within the record limits at long horizons), ms [F],
    total_boxes [F], total_pairs [F]."""
    import torch

    from . import Scene
    n = len(elements)
    F = len(multipliers)
    boxes = np.zeros((F, n))
    pairs = np.zeros((F, n))
    ms = np.zeros(F)
    T = int(round(horizon_s / tick_s))
    st = torch.cuda.current_stream()
    for q, f in enumerate(multipliers):
        sc = Scene(elements, horizon_s, tick_s,
                   B.make_step_policy(B.SCD_STEP_PERIOD_FRACTION, period_fraction=f), mode=mode)
        sc.build_boxes()
        sc.find_pairs_device()  # sizes the buffers
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sc.build_boxes()
        sc.find_pairs_device()
        e1.record(st)
        e1.synchronize()
        ms[q] = e0.elapsed_time(e1)
        k = sc.steps().cpu().numpy().astype(np.int64)
        boxes[q] = (T + k) // k
        if count == "runs":
            ptr, m = B.scd_find_pairs_device(sc.handle)
        else:
            ptr, m = B.scd_find_raw_cells_device(sc.handle)
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        B.scd_count_pairs_per_object(ptr, m, n, cnt.data_ptr(), st.cuda_stream)
        pairs[q] = cnt.cpu().numpy()
        sc.close()
    return {"multipliers": np.array(multipliers), "boxes": boxes, "pairs": pairs, "ms": ms,
            "total_boxes": boxes.sum(1), "total_pairs": pairs.sum(1) / 2.0}


def fit_cost_model(sw):
    """Least-squares c_box, c_hit >= 0 with ms ~ c_box * boxes + c_hit * pairs."""
    A = np.stack([sw["total_boxes"], sw["total_pairs"]], 1)
    c, *_ = np.linalg.lstsq(A, sw["ms"], rcond=None)
    if c[0] < 0 or c[1] < 0:  # fall back to one-term fits
        c = np.array([max(0.0, float(np.dot(A[:, 0], sw["ms"]) / np.dot(A[:, 0], A[:, 0]))),
                      max(0.0, float(np.dot(A[:, 1], sw["ms"]) / np.dot(A[:, 1], A[:, 1])))])
    return float(c[0]), float(c[1])


def object_cost(sw, c_box, c_hit):
    """[F, n] modelled cost of each object at each multiplier."""
    return c_box * sw["boxes"] + 0.5 * c_hit * sw["pairs"]


def targets(elements, sw, c_box, c_hit):
    """log of each object's best step [s] over the sweep's multipliers."""
    cost = object_cost(sw, c_box, c_hit)
    best = sw["multipliers"][np.argmin(cost, 0)]
    a = np.asarray(elements)[:, 0]
    P = 2 * math.pi * np.sqrt(a ** 3 / MU)
    return np.log(P / best)


def train(net: StepNet, X, Y, epochs: int = 40, batch: int = 4096, lr: float = 2e-3,
          weight_decay: float = 1e-4, seed: int = 0):
    """Minibatch AdamW on the GPU over host arrays X [n, 8], Y [n]: each
    epoch uploads one seeded shuffle and steps through contiguous slices.
    Returns the loss of every step."""
    import torch
    rng = np.random.default_rng(seed)
    X = np.ascontiguousarray(X, np.float32)
    Y = np.ascontiguousarray(Y, np.float32)
    n = len(X)
    losses = []
    for ep in range(epochs):
        perm = rng.permutation(n)
        dx = torch.as_tensor(X[perm], device="cuda")
        dy = torch.as_tensor(Y[perm], device="cuda")
        for s in range(0, n, batch):
            e = min(n, s + batch)
            losses.append(net.train_step(dx[s:e], dy[s:e], lr, weight_decay))
    return np.array(losses)

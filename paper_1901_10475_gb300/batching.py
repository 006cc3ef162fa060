"""Grouping independent scenes into batches for one GPU.

Every batch becomes one BatchScene: one box build, one sort, one tree and one
persistent traversal over all of its scenes, so a batch's scenes all finish
when the batch does.  A batch holds scenes whose estimated box counts add up
to at most a budget (a scene above the budget alone), which bounds the
batch's device memory.  The batches run one after the other; taking the
scenes shortest first (the classic rule that minimises the mean completion
time of jobs on one server) lets the small scenes finish early instead of
waiting behind large ones, without changing the total work.  Host-side
planning only: the screening itself is the library's.
"""
from __future__ import annotations

import math

import numpy as np

MU_KM3_S2 = 398600.4418


def estimated_boxes(elements, horizon_s: float, tick_s: float = 1.0,
                    period_fraction: float = 100.0) -> float:
    """Boxes of a scene under the period-fraction step rule: per object
    ceil((T + 1) / k) segments of k = max(1, floor(P / (fraction tick))) ticks,
    P = 2 pi sqrt(a^3 / mu) (elements: rows whose first column is a [km])."""
    a = np.asarray(elements, dtype=np.float64)[:, 0]
    T = int(math.floor(horizon_s / tick_s))
    k = np.maximum(np.floor(2.0 * math.pi * np.sqrt(a ** 3 / MU_KM3_S2) / (period_fraction * tick_s)), 1.0)
    return float(np.sum(np.ceil((T + 1) / k)))


def plan_batches(costs, budget: float, order: str = "shortest_first") -> list[list[int]]:
    """Scene indices grouped into batches, in the order they should run.

    costs: per scene an estimate of its work (e.g. estimated_boxes).
    budget: the most cost one batch may hold (a scene above it runs alone).
    order: "shortest_first" (scenes by increasing cost, ties by index) or
    "arrival" (the given order).  Scenes are packed greedily in that order:
    a batch closes when the next scene would take it over the budget."""
    costs = [float(c) for c in costs]
    if budget <= 0:
        raise ValueError("budget must be positive")
    if order == "shortest_first":
        seq = sorted(range(len(costs)), key=lambda s: (costs[s], s))
    elif order == "arrival":
        seq = list(range(len(costs)))
    else:
        raise ValueError(f"unknown order {order!r}")
    groups: list[list[int]] = []
    cur: list[int] = []
    cur_cost = 0.0
    for s in seq:
        if cur and cur_cost + costs[s] > budget:
            groups.append(cur)
            cur, cur_cost = [], 0.0
        cur.append(s)
        cur_cost += costs[s]
    if cur:
        groups.append(cur)
    return groups

"""The batch planner (host logic): every scene in exactly one batch, no
batch over the budget unless it holds a single larger scene, shortest
first, and the arrival order as a plain greedy packing."""
import math

import numpy as np
import pytest

from paper_1901_10475_gb300 import batching


def test_estimated_boxes_matches_the_step_rule():
    # a = 7000 km: P = 2 pi sqrt(a^3 / mu) = 5828.5 s, k = floor(P / 100) = 58
    els = np.array([[7000.0, 0, 0, 0, 0, 0, 1.0], [42164.0, 0, 0, 0, 0, 0, 1.0]])
    P1 = 2 * math.pi * math.sqrt(7000.0 ** 3 / batching.MU_KM3_S2)
    P2 = 2 * math.pi * math.sqrt(42164.0 ** 3 / batching.MU_KM3_S2)
    k1, k2 = math.floor(P1 / 100), math.floor(P2 / 100)
    assert k1 == 58
    want = math.ceil(3601 / k1) + math.ceil(3601 / k2)
    assert batching.estimated_boxes(els, 3600.0) == want


@pytest.mark.parametrize("order", ["shortest_first", "arrival"])
def test_plan_covers_every_scene_within_budget(order):
    rng = np.random.default_rng(3)
    costs = np.exp(rng.uniform(math.log(1e3), math.log(1e8), 64))
    groups = batching.plan_batches(costs, 4e7, order)
    flat = [s for g in groups for s in g]
    assert sorted(flat) == list(range(64))
    for g in groups:
        assert len(g) == 1 or sum(costs[s] for s in g) <= 4e7
    if order == "shortest_first":
        assert [costs[s] for s in flat] == sorted(costs)
    else:
        assert flat == list(range(64))


def test_arrival_order_is_the_greedy_packing():
    costs = [5, 3, 4, 9, 1, 1, 7]
    assert batching.plan_batches(costs, 10, "arrival") == [[0, 1], [2], [3, 4], [5, 6]]
    assert batching.plan_batches(costs, 10, "shortest_first") == [[4, 5, 1, 2], [0], [6], [3]]
    with pytest.raises(ValueError):
        batching.plan_batches(costs, 0)
    with pytest.raises(ValueError):
        batching.plan_batches(costs, 10, "longest_first")


def test_estimated_boxes_equals_the_oracle_segments():
    # the planner's box estimate is the screen's segment count under P/100
    # steps: per object ceil((T + 1) / k_i), k_i from the oracle's step rule
    import oracle as O
    import population as P
    els = P.catalog_mixture(1000, seed=17)
    for horizon in (3600.0, 86400.0):
        T = int(horizon)
        k = O.step_ticks(els, 1, 1.0, frac=100.0)
        want = int(np.sum((T + 1 + k - 1) // k))
        assert batching.estimated_boxes(els, horizon) == want

"""The find sequence replayed as one captured CUDA graph gives exactly the
eagerly launched result, for the plain screen, the decompositions and a
batch of scenes, on repeated replays and after the inputs change size."""
import numpy as np
import pytest
import torch

import oracle as O
import population as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scd():
    import paper_1901_10475_gb300 as m
    torch.cuda.set_device(0)
    return m


def _same(a, b):
    return np.array_equal(np.asarray(a).view(np.int32), np.asarray(b).view(np.int32))


@pytest.mark.parametrize("decomp", [None, (2, 0, 16), (1, 8, 0)])
def test_graph_replay_equals_eager(scd, decomp):
    els = P.catalog_mixture(n=900, seed=81, radius_km=25.0)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    eager = scd.Scene(els, 20000.0, 1.0, pol).build_boxes()
    want = eager.find_pairs(decomp)
    eager.close()
    g = scd.Scene(els, 20000.0, 1.0, pol, tuning=dict(use_graph=1)).build_boxes()
    for it in range(4):  # first call runs eagerly and captures; then replays
        g.build_boxes()
        got = g.find_pairs(decomp)
        assert _same(got, want), (len(got), len(want))
        # (the host-output call may have run twice to size its buffer)
        assert g.metrics()["graph"] in ((1, 2) if it == 0 else (2,))
    m = g.metrics()
    assert m["pairs"] == len(want)
    g.close()


def test_graph_recaptures_when_sizes_change(scd):
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    a = P.catalog_mixture(n=500, seed=82, radius_km=25.0)
    b = P.catalog_mixture(n=500, seed=83, radius_km=60.0)  # more pairs, other box count
    g = scd.Scene(a, 10000.0, 1.0, pol, tuning=dict(use_graph=1)).build_boxes()
    for els in (a, a, b, b, a):
        g.set_elements(els)
        g.build_boxes()
        got = g.find_pairs()
        lo, hi, obj = (x.cpu().numpy() for x in g.boxes())
        want = O.canonicalize(O.raw_cells_sweep(lo, hi, obj.view(np.uint32)))
        assert _same(got, want)
    g.close()


def test_graph_batch_of_scenes(scd):
    scenes = [P.catalog_mixture(n=m, seed=600 + k, radius_km=25.0, crossing_frac=0.0)
              for k, m in enumerate([60, 300, 150])]
    hz = [3600.0, 7200.0, 5400.0]
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    e = scd.BatchScene(scenes, hz, 1.0, pol).build_boxes()
    want = e.find_pairs_per_scene()
    e.close()
    g = scd.BatchScene(scenes, hz, 1.0, pol, tuning=dict(use_graph=1)).build_boxes()
    for _ in range(3):
        g.build_boxes()
        got = g.find_pairs_per_scene()
        assert all(_same(x, y) for x, y in zip(got, want))
    g.close()

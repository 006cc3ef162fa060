"""A batch of independent scenes (own sizes, horizons) screened in one
persistent traversal: every scene's list equals the oracle's for that scene
alone, and no pair joins objects of different scenes."""
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


def test_batch_of_uneven_scenes_matches_each_scene_alone(scd):
    sizes = [40, 400, 7, 250, 1, 120]
    horizons = [3600.0, 7200.0, 600.0, 5400.0, 1200.0, 10800.0]
    scenes = [P.catalog_mixture(n=m, seed=500 + k, radius_km=25.0, crossing_frac=0.0)
              for k, m in enumerate(sizes)]
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    b = scd.BatchScene(scenes, horizons, 1.0, pol).build_boxes()
    per = b.find_pairs_per_scene()
    total = 0
    for k, els in enumerate(scenes):
        kk = O.step_ticks(els, O.STEP_PERIOD_FRACTION, 1.0, frac=100.0)
        T = int(horizons[k])
        lo, hi, obj = O.boxes(els, T, 1.0, kk)
        want = O.canonicalize(O.raw_cells_sweep(lo, hi, obj))
        got = per[k]
        total += len(got)
        assert len(got) == len(want), (k, len(got), len(want))
        assert np.array_equal(got.view(np.int32), want.view(np.int32)), k
        # each scene alone through the single-scene path gives the same list
        one = scd.Scene(els, horizons[k], 1.0, pol).build_boxes()
        assert np.array_equal(one.find_pairs().view(np.int32), got.view(np.int32)), k
        one.close()
    assert total > 50
    b.close()


def test_batch_argument_checks(scd):
    pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    els = [P.uniform_leo(5, seed=1), P.uniform_leo(6, seed=2)]
    with pytest.raises(scd.ScdError):
        scd.BatchScene(els, [600.0, 600.5], 1.0, pol)
    b = scd.BatchScene(els, [600.0, 300.0], 1.0, pol).build_boxes()
    with pytest.raises(scd.ScdError):
        b.find_pairs((scd.SCD_DECOMP_SLAB_OCT, 0, 4))
    b.close()

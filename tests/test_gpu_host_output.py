"""The canonical list delivered into host memory (scd_find_pairs) is the
device list (scd_find_pairs_device) element for element, whichever way it
travels: streamed bucket by bucket into pinned memory while later buckets
are still being sorted, into pageable memory, or after a first call whose
buffer was too small (which writes nothing)."""
import numpy as np
import pytest
import torch

import population as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scd():
    import paper_1901_10475_gb300 as m
    torch.cuda.set_device(0)
    return m


def _device_list(scd, sc):
    return sc.find_pairs_device().cpu().numpy().view(scd.PAIR_DTYPE).reshape(-1)


# catalog mixtures, and small crowded shells whose keys leave 8 (12 objects)
# or 6 (8 objects) bits for the pair's objects: the latter is copied whole
@pytest.mark.parametrize("n,horizon_s,mode", [(3000, 21600.0, 0), (3000, 21600.0, 1),
                                              (200, 3000.0, 0), (12, 3000.0, 0), (8, 3000.0, 0)])
def test_host_list_equals_device_list(scd, n, horizon_s, mode):
    els = (P.catalog_mixture(n=n, seed=41) if n >= 100
           else P.uniform_leo(n, seed=5, radius_km=400.0))
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc = scd.Scene(els, horizon_s, 1.0, pol, mode=mode).build_boxes()
    want = _device_list(scd, sc)
    assert len(want) > 0
    pinned = torch.empty(len(want) * 16, dtype=torch.uint8).pin_memory()
    out = pinned.numpy().view(scd.PAIR_DTYPE)
    out[:] = 0
    assert scd.scd_find_pairs_into(sc.handle, out) == len(want)
    assert np.array_equal(out, want)
    # a larger pinned buffer: only the first n entries are written
    big = torch.full(((len(want) + 5) * 4,), -7, dtype=torch.int32).pin_memory()
    bo = big.numpy().view(scd.PAIR_DTYPE)
    assert scd.scd_find_pairs_into(sc.handle, bo) == len(want)
    assert np.array_equal(bo[:len(want)], want)
    assert (bo[len(want):].view(np.int32) == -7).all()
    # pageable memory, and the binding's grow-and-retry call
    page = np.zeros(len(want), scd.PAIR_DTYPE)
    assert scd.scd_find_pairs_into(sc.handle, page) == len(want)
    assert np.array_equal(page, want)
    assert np.array_equal(sc.find_pairs(), want)
    sc.close()


def test_too_small_writes_nothing(scd):
    els = P.catalog_mixture(n=1000, seed=42)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc = scd.Scene(els, 7200.0, 1.0, pol).build_boxes()
    n = len(_device_list(scd, sc))
    small = np.full(n - 1, 0, scd.PAIR_DTYPE)
    small.view(np.int32)[:] = -3
    with pytest.raises(scd.ScdError) as e:
        scd.scd_find_pairs_into(sc.handle, small)
    assert e.value.status == scd.SCD_ERR_BUFFER_TOO_SMALL
    assert (small.view(np.int32) == -3).all()
    sc.close()


def test_no_pairs(scd):
    els = np.array([[7000.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0],
                    [42164.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    sc = scd.Scene(els, 3600.0, 1.0, pol).build_boxes()
    out = np.zeros(4, scd.PAIR_DTYPE)
    assert scd.scd_find_pairs_into(sc.handle, out) == 0
    sc.close()

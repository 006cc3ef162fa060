"""The autotuner (paper_1901_10475_gb300.autotune) on a small scene: its
search returns one of the tunings it timed, that tuning's screen equals the
oracle's pair list on the same FP32 boxes, and its JSON cache stores the
choice under the (GPU, workload hash, log2 of the box count) key and hands
it back on the next call without timing anything."""
import json

import numpy as np
import pytest
import torch

import oracle as O
import population as P

pytestmark = pytest.mark.gpu

HORIZON_S = 7200.0


@pytest.fixture(scope="module")
def scene():
    import paper_1901_10475_gb300 as scd
    torch.cuda.set_device(0)
    els = P.catalog_mixture(n=300, seed=P.SEED_BASE + 77)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc = scd.Scene(els, HORIZON_S, 1.0, pol)
    sc.build_boxes()
    yield scd, els, sc
    sc.close()


def _oracle_list(sc):
    lo, hi, obj = (x.cpu().numpy() for x in sc.boxes())
    return O.canonicalize(O.raw_cells_sweep(lo, hi, obj.view(np.uint32)))


def test_tune_returns_a_timed_candidate_whose_screen_is_the_oracles(scene):
    from paper_1901_10475_gb300 import autotune
    scd, els, sc = scene
    best, results = autotune.tune(sc, reps=1)
    timed = [t for t, _ in results]
    assert len(timed) >= 10 and all(ms > 0 for _, ms in results)
    assert best in timed
    assert min(results, key=lambda r: r[1])[0] == best
    # the tuning is in force on the scene; its screen equals the oracle's
    sc.set_tuning(best)
    sc.build_boxes()
    got = sc.find_pairs()
    want = _oracle_list(sc)
    assert len(got) == len(want) > 0
    assert (got.view(np.int32).reshape(-1, 4) == want.view(np.int32).reshape(-1, 4)).all()


def test_load_or_tune_caches_under_its_key(scene, tmp_path, monkeypatch):
    from paper_1901_10475_gb300 import autotune
    scd, els, sc = scene
    nbox = sc.metrics()["boxes"]
    key = autotune.workload_key(els, HORIZON_S, 1.0, "P/100", nbox)
    gpu, digest, log2n = key.split("|")
    assert gpu == torch.cuda.get_device_name()
    assert log2n == f"log2N={int(np.log2(nbox))}" and len(digest) == 16
    # a different population or horizon gives a different key
    assert autotune.workload_key(els[:-1], HORIZON_S, 1.0, "P/100", nbox) != key
    assert autotune.workload_key(els, HORIZON_S + 60, 1.0, "P/100", nbox) != key
    cache = tmp_path / "tune.json"
    t1, r1 = autotune.load_or_tune(sc, key, cache_path=str(cache), reps=1)
    assert r1 is not None and t1 in [t for t, _ in r1]
    stored = json.loads(cache.read_text())
    assert list(stored) == [key] and stored[key]["tuning"] == t1
    assert stored[key]["ms"] == pytest.approx(min(ms for _, ms in r1))
    # the second call reads the cache: nothing is timed
    timed = []
    monkeypatch.setattr(autotune, "_time_screen", lambda *a, **k: timed.append(1) or 1.0)
    t2, r2 = autotune.load_or_tune(sc, key, cache_path=str(cache), reps=1)
    assert r2 is None and t2 == t1 and timed == []
    # and the cached tuning is the one in force
    cur = sc.tuning()
    assert all(cur[f] == pytest.approx(v) for f, v in t1.items())

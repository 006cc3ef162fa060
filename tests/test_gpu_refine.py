"""Parity of the CUDA adaptive refinement (scd_refine_witnesses, through the
C ABI) with the oracle (its rounds starting from the scene's period-bounded
first intervals, as the CUDA rounds do): the witness list is exact (Alg 1's test decides every
tick candidate), so it must equal the oracle's refinement and Alg 1 witness
for witness, in Alg 1's order.  The rounds' interval counts come from
overlap tests of FP32 boxes whose centres agree with the oracle's to 1e-7 km,
so they may differ where two boxes touch; they must agree within 2%.  Both
box modes; the 24 h catalog subset against the narrow phase."""
import math

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


def _scene(scd, els, horizon_s, mode=0):
    step = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    return scd.Scene(els, horizon_s, 1.0, step=step, mode=mode).build_boxes()


def _f(sc):
    """the scene's refinement start fraction (the oracle takes the same)"""
    return float(sc.tuning()["refine_start"])


def _tuples(w):
    return [(int(a), int(b), int(c)) for a, b, c in w.tolist()]


@pytest.mark.parametrize("seed", [300, 302, 310, 311])
def test_small_large_radii_equal_alg1_and_oracle(scd, seed):
    els = P.uniform_leo(10, seed=seed, radius_km=400.0)
    T = 300
    sc = _scene(scd, els, float(T))
    w, rb = sc.refine_witnesses()
    ref = O.alg1_witnesses(els, T, 1.0)
    assert _tuples(w) == _tuples(ref)
    ow, orb, _ = O.refine_discrete(els, T, 1.0, O.BOX_SPEED, start_fraction=_f(sc))
    assert len(rb) <= math.ceil(math.log2(T + 1)) + 2
    assert abs(int(rb.sum()) - int(orb.sum())) <= 0.02 * orb.sum()
    sc.close()


def test_uniform_512_six_thousand_seconds(scd):
    # the small workload's population (n = 512, 6000 s), with one pair of
    # identical elements that collide at every tick
    els = P.uniform_leo(512)
    els[511] = els[7]
    sc = _scene(scd, els, 6000.0)
    w, rb = sc.refine_witnesses()
    ow, orb, _ = O.refine_discrete(els, 6000, 1.0, O.BOX_SPEED, start_fraction=_f(sc))
    assert _tuples(w) == _tuples(ow)
    mine = w[(w["i"] == 7) & (w["j"] == 511)]
    assert mine["t"].tolist() == list(range(6001))
    assert len(rb) == len(orb)
    assert abs(int(rb.sum()) - int(orb.sum())) <= 0.02 * orb.sum()
    # an INTERVAL-mode scene refines with INTERVAL boxes (Sec. 4.5): the
    # same witnesses (both exact), the oracle's rounds with its INTERVAL boxes
    sc2 = _scene(scd, els, 6000.0, mode=1)
    w2, rb2 = sc2.refine_witnesses()
    ow2, orb2, _ = O.refine_discrete(els, 6000, 1.0, O.BOX_INTERVAL, start_fraction=_f(sc2))
    assert _tuples(w2) == _tuples(w) == _tuples(ow2)
    assert len(rb2) == len(orb2)
    assert abs(int(rb2.sum()) - int(orb2.sum())) <= 0.02 * orb2.sum()
    # tighter boxes: fewer intervals in all
    assert rb2.sum() < rb.sum()
    sc.close()
    sc2.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_catalog_subset_full_day(scd, mode):
    """The refinement at the catalog workload's horizon: 2000 objects of the
    mixture (with seeded crossing pairs) over 24 h at 1 s ticks.  Its
    witnesses equal the narrow phase's over the fixed-step screen's
    candidates (P/100 steps), and every seeded crossing is among them."""
    els, cr = P.catalog_mixture(n=2000, seed=23, crossing_frac=0.004, horizon_s=86400.0,
                                return_crossings=True)
    T = 86400
    sc = _scene(scd, els, float(T), mode=mode)
    w, rb = sc.refine_witnesses()
    assert len(rb) <= math.ceil(math.log2(T + 1)) + 2
    got = set(_tuples(w))
    for (b, c, tc) in cr:
        assert (b, c, tc) in got
    step = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc2 = scd.Scene(els, float(T), 1.0, step=step, mode=mode).build_boxes()
    first, count, earliest = sc2.narrow_phase(sc2.find_pairs_device())
    assert int(count.cpu().numpy().astype(np.int64).sum()) == len(w)
    assert earliest == (tuple(_tuples(w[:1])[0]) if len(w) else None)
    print(f"24 h, 2000 objects, mode {mode}: {len(w)} witnesses, {len(rb)} rounds, "
          f"{int(rb.sum())} intervals, peak {int(rb.max())}")
    sc.close()
    sc2.close()


def test_catalog_mixture_crossings(scd):
    els, cr = P.catalog_mixture(n=2000, seed=21, crossing_frac=0.004, horizon_s=1800.0,
                                return_crossings=True)
    T = 1800
    sc = _scene(scd, els, float(T))
    w, rb = sc.refine_witnesses()
    ref = O.alg1_sweep(els, 0, T, 1.0)
    assert sorted(_tuples(w)) == sorted((int(a), int(b), int(c)) for a, b, c, _ in ref.tolist())
    got = set(_tuples(w))
    for (b, c, tc) in cr:
        assert (b, c, tc) in got
    # the same witnesses as the narrow phase over the fixed-step screen's
    # candidates (P/100 steps): both are exact
    step = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc2 = scd.Scene(els, float(T), 1.0, step=step).build_boxes()
    first, count, earliest = sc2.narrow_phase(sc2.find_pairs_device())
    assert int(count.cpu().numpy().astype(np.int64).sum()) == len(w)
    assert earliest == (tuple(_tuples(w[:1])[0]) if len(w) else None)
    sc.close()
    sc2.close()


@pytest.mark.parametrize("frac", [0.0, 32.0, 1024.0])
def test_start_fraction_follows_the_tuning(scd, frac):
    """Another start fraction on a scene whose rounds were captured with the
    default: the first round holds exactly the oracle's first intervals for
    that fraction, and the witnesses stay Alg 1's."""
    els = P.uniform_leo(10, seed=311, radius_km=400.0)
    T = 300
    sc = _scene(scd, els, float(T))
    sc.refine_witnesses()
    sc.refine_witnesses()
    sc.set_tuning(dict(sc.tuning(), refine_start=frac))
    w, rb = sc.refine_witnesses()
    ow, orb, _ = O.refine_discrete(els, T, 1.0, O.BOX_SPEED, start_fraction=frac)
    assert _tuples(w) == _tuples(ow) == _tuples(O.alg1_witnesses(els, T, 1.0))
    assert rb[0] == orb[0]
    assert abs(int(rb.sum()) - int(orb.sum())) <= 0.02 * orb.sum()
    with pytest.raises(scd.ScdError):
        sc.set_tuning(dict(sc.tuning(), refine_start=-1.0))
    sc.close()


def test_far_apart_orbits_and_errors(scd):
    els = np.array([[7000.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0],
                    [42164.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    step = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    sc = scd.Scene(els, 86400.0, 1.0, step=step)
    with pytest.raises(scd.ScdError) as e:
        sc.refine_witnesses()  # boxes not built yet
    assert e.value.status == scd.SCD_ERR_STATE
    sc.build_boxes()
    w, rb = sc.refine_witnesses()
    _, orb, _ = O.refine_discrete(els, 86400, 1.0, O.BOX_SPEED, start_fraction=_f(sc))
    assert len(w) == 0 and rb.tolist() == orb.tolist()
    sc.close()
    # a buffer too small reports the count needed and writes nothing
    els = P.uniform_leo(4, seed=5)
    els[2] = els[0]
    sc = _scene(scd, els, 50.0)
    import ctypes
    n = ctypes.c_int64(0)
    out = np.zeros(4, scd.WITNESS_DTYPE)
    rc = scd._binding.lib().scd_refine_witnesses(sc.handle, out.ctypes.data, 4, ctypes.byref(n),
                                                 None, None)
    assert rc == scd.SCD_ERR_BUFFER_TOO_SMALL and n.value == 51
    assert not out.view(np.int32).any()
    sc.close()


def _crossing_between_ticks(tc=100.5, a=7000.0, r=1.0):
    # two circular orbits in perpendicular planes, both at (a, 0, 0) at tc,
    # about 3.8 km apart (infinity norm) at the ticks either side
    n = math.sqrt(O.MU / a ** 3)
    return np.array([[a, 0.0, 0.0, 0.0, 0.0, -n * tc, r],
                     [a, 0.0, math.pi / 2, 0.0, 0.0, -n * tc, r]])


def test_continuous_finds_crossing_between_ticks(scd):
    els = _crossing_between_ticks()
    sc = _scene(scd, els, 200.0)
    assert len(sc.refine_witnesses()[0]) == 0  # the discrete problem tunnels
    spans, rb = sc.refine_continuous(0.1)
    ospans, orb = O.refine_continuous(els, 200.0, 0.1, O.BOX_SPEED)
    assert spans.tolist() == ospans.tolist()
    assert rb.tolist() == orb.tolist()
    assert np.any((spans["t0"] <= 100.5) & (100.5 <= spans["t1"]))
    sc.close()


@pytest.mark.parametrize("seed", [300, 310])
def test_continuous_equals_oracle_and_covers_alg1(scd, seed):
    els = P.uniform_leo(10, seed=seed, radius_km=400.0)
    T = 300
    sc = _scene(scd, els, float(T))
    spans, rb = sc.refine_continuous(0.5)
    ospans, orb = O.refine_continuous(els, float(T), 0.5, O.BOX_SPEED)
    # spans are exact multiples of the finest interval; boxes that merely
    # touch may decide differently between the two FP32 roundings
    g = set(spans.tolist())
    o = set(ospans.tolist())
    assert len(g ^ o) <= 0.01 * len(o)
    assert len(rb) == len(orb)
    for i, j, t in O.alg1_witnesses(els, T, 1.0).tolist():
        m = spans[(spans["i"] == i) & (spans["j"] == j)]
        assert np.any((m["t0"] <= t) & (t <= m["t1"])), (i, j, t)
    with pytest.raises(scd.ScdError):
        sc.refine_continuous(0.0)
    sc.close()


def _round_intervals(lo, hi, obj):
    return sorted(zip(obj.astype(np.int64).tolist(), lo[:, 3].astype(np.int64).tolist(),
                      hi[:, 3].astype(np.int64).tolist()))


@pytest.mark.parametrize("mode", [0, 1])
def test_every_round_follows_from_its_own_boxes(scd, mode):
    """Exact per-round parity: each round's intervals are exactly the
    oracle's round rule applied to the GPU's own FP32 boxes of the round
    before (every pair of other objects' boxes tested), and every box is the
    oracle's box of its interval within one FP32 ulp (512 objects, 6000 s,
    with a pair of identical elements)."""
    els = P.uniform_leo(512)
    els[511] = els[7]
    sc = _scene(scd, els, 6000.0, mode=mode)
    tr = scd.scd_refine_trace(sc.handle)
    w, rb = sc.refine_witnesses()
    assert [len(o) for _, _, o in tr] == rb.tolist()
    # the first round: every object's ticks cut by its own start length
    first = []
    for i in range(len(els)):
        L = O.refine_start_ticks(els[i], 6000, 1.0, _f(sc))
        first += [(i, a, min(a + L - 1, 6000)) for a in range(0, 6001, L)]
    assert _round_intervals(*tr[0]) == sorted(first)
    g = np.random.default_rng(mode)
    for r, (lo, hi, obj) in enumerate(tr):
        want = O.refine_round(lo, hi, obj, False)
        if r + 1 < len(tr):
            assert _round_intervals(*tr[r + 1]) == sorted(map(tuple, want.tolist())), r
        else:
            assert len(want) == 0
        for q in g.choice(len(obj), min(200, len(obj)), replace=False):
            ol, oh, _, _ = O.box(els[obj[q]], mode, int(lo[q, 3]), int(hi[q, 3]), 1.0)
            assert np.all(np.abs(lo[q].view(np.int32) - ol.view(np.int32)) <= 1)
            assert np.all(np.abs(hi[q].view(np.int32) - oh.view(np.int32)) <= 1)
    sc.close()


def test_every_continuous_round_follows_from_its_own_boxes(scd):
    els = P.uniform_leo(10, seed=310, radius_km=400.0)
    sc = _scene(scd, els, 300.0)
    tr = scd.scd_refine_trace(sc.handle, 0.5)
    spans, rb = sc.refine_continuous(0.5)
    assert [len(o) for _, _, o in tr] == rb.tolist()
    for r in range(len(tr) - 1):
        want = O.refine_round(*tr[r], True)
        assert _round_intervals(*tr[r + 1]) == sorted(map(tuple, want.tolist())), r
    # the spans are the meeting pairs of the last round's own boxes
    lo, hi, obj = tr[-1]
    unit = 300.0 / 2 ** (len(tr) - 1)
    cells = O.raw_cells_bruteforce(lo, hi, obj)
    want = sorted({(int(c["i"]), int(c["j"]), c["tlo"] * unit, c["thi"] * unit) for c in cells})
    assert sorted(map(tuple, spans.tolist())) == want
    sc.close()


def test_repeated_calls_replay_the_same_rounds(scd):
    """The second and later calls on a scene replay its captured rounds: the
    same witnesses and round sizes; after new elements (same count) the
    results are those of a fresh scene; the continuous variant in between
    (another shape of rounds) changes nothing."""
    els = P.uniform_leo(512)
    els[511] = els[7]
    sc = _scene(scd, els, 6000.0)
    w1, rb1 = sc.refine_witnesses()
    for _ in range(3):
        w, rb = sc.refine_witnesses()
        assert _tuples(w) == _tuples(w1) and rb.tolist() == rb1.tolist()
    spans, _ = sc.refine_continuous(1.0)
    w, rb = sc.refine_witnesses()
    assert _tuples(w) == _tuples(w1) and rb.tolist() == rb1.tolist()
    els2 = P.uniform_leo(512, seed=77)
    els2[100] = els2[200]
    sc.set_elements(els2)
    sc.build_boxes()
    w2, rb2 = sc.refine_witnesses()
    fresh = _scene(scd, els2, 6000.0)
    w3, rb3 = fresh.refine_witnesses()
    assert _tuples(w2) == _tuples(w3) and rb2.tolist() == rb3.tolist()
    assert len(w2) > 0
    sc.close()
    fresh.close()

"""Pins of the oracle's pair sets: the closed 4D overlap set (Defs 2, 8),
its canonical merged form, and coverage of every true collision found by the
paper's brute force Alg 1 (soundness, Sec. 7.2)."""
import os

import numpy as np
import pytest

import oracle as O
import population as P

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _cells(rows):
    return np.array([tuple(int(x) for x in r) for r in rows], dtype=O.CELL_DTYPE)


def test_merge_golden():
    raw, want = [], []
    with open(os.path.join(GOLD, "merge_example.txt")) as f:
        for line in f:
            s = line.split()
            if not s or s[0].startswith("#"):
                continue
            (raw if s[0] == "raw" else want).append(s[1:])
    got = O.canonicalize(_cells(raw))
    assert got.tolist() == _cells(want).tolist()


def _random_boxes(g, N, nobj, span=100.0, size=10.0, T=200):
    lo = np.zeros((N, 4), np.float32)
    hi = np.zeros((N, 4), np.float32)
    c = g.uniform(-span, span, (N, 3)).astype(np.float32)
    w = g.uniform(0, size, (N, 3)).astype(np.float32)
    # quantise so that exact touching (lo_a == hi_b) happens often
    c = np.round(c)
    w = np.round(w)
    lo[:, :3] = c - w
    hi[:, :3] = c + w
    t0 = g.integers(0, T, N)
    t1 = t0 + g.integers(0, 20, N)
    lo[:, 3] = t0
    hi[:, 3] = t1
    obj = g.integers(0, nobj, N).astype(np.uint32)
    return lo, hi, obj


@pytest.mark.parametrize("seed", range(6))
def test_sweep_equals_bruteforce_and_python_loop(seed):
    g = np.random.default_rng(seed)
    lo, hi, obj = _random_boxes(g, 300, 40)
    a = O.raw_cells_bruteforce(lo, hi, obj)
    b = O.raw_cells_sweep(lo, hi, obj)
    key = lambda c: sorted(map(tuple, c.tolist()))
    assert key(a) == key(b)
    # a third, pure-Python definition of the same set
    ref = []
    for x in range(len(obj)):
        for y in range(x + 1, len(obj)):
            if obj[x] == obj[y]:
                continue
            if all(lo[x, k] <= hi[y, k] and lo[y, k] <= hi[x, k] for k in range(4)):
                i, j = sorted((int(obj[x]), int(obj[y])))
                ref.append((i, j, int(max(lo[x, 3], lo[y, 3])), int(min(hi[x, 3], hi[y, 3]))))
    assert key(a) == sorted(ref)
    assert len(a) > 0


def test_selected_is_restriction():
    g = np.random.default_rng(11)
    lo, hi, obj = _random_boxes(g, 400, 50)
    full = O.raw_cells_bruteforce(lo, hi, obj)
    sel = np.zeros(50, np.uint8)
    sel[[3, 7, 19, 44]] = 1
    part = O.raw_cells_selected(lo, hi, obj, sel)
    keep = [c for c in map(tuple, full.tolist()) if sel[c[0]] or sel[c[1]]]
    assert sorted(map(tuple, part.tolist())) == sorted(keep)


def test_touching_boxes_count_and_same_object_never():
    lo = np.array([[0, 0, 0, 0], [1, 0, 0, 5], [0, 0, 0, 0]], np.float32)
    hi = np.array([[1, 1, 1, 5], [2, 1, 1, 9], [1, 1, 1, 5]], np.float32)
    obj = np.array([0, 1, 0], np.uint32)
    got = O.raw_cells_bruteforce(lo, hi, obj).tolist()
    assert sorted(got) == [(0, 1, 5, 5), (0, 1, 5, 5)]


def test_identical_elements_collide_over_whole_horizon():
    # the docked-spacecraft case of Sec. 6.2: identical elements
    els = P.uniform_leo(6, seed=3)
    els[4] = els[1]
    k = np.array([10, 7, 13, 10, 7, 10], np.int64)
    cells = O.screen(els, 600, 1.0, k)
    mine = cells[(cells["i"] == 1) & (cells["j"] == 4)]
    assert mine.tolist() == [(1, 4, 0, 600)]


def test_crossing_pair_is_reported_at_its_tick():
    els, cr = P.catalog_mixture(n=2000, seed=21, crossing_frac=0.004, horizon_s=3000.0,
                                return_crossings=True)
    sub = sorted({x for c in cr for x in c[:2]})
    e2 = els[sub]
    k = O.step_ticks(e2, O.STEP_PERIOD_FRACTION, 1.0, frac=100.0)
    cells = O.screen(e2, 3000, 1.0, k)
    for (b, c, tc) in cr:
        i, j = sub.index(b), sub.index(c)
        m = cells[(cells["i"] == i) & (cells["j"] == j)]
        assert np.any((m["tlo"] <= tc) & (tc <= m["thi"]))
        # and at t_c the two objects really meet (Alg 1's test)
        assert np.abs(O.position(e2[i], tc) - O.position(e2[j], tc)).max() < 1e-6


def test_geo_and_leo_never_pair():
    els = np.array([[42164.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.5],
                    [6778.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.5]])
    k = np.array([100, 50], np.int64)
    assert len(O.screen(els, 86400, 1.0, k)) == 0


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_screen_covers_every_alg1_witness(mode, seed):
    """Soundness: each true collision (i, j, t) of Alg 1 lies inside a
    reported (i, j, [tlo, thi])."""
    g = np.random.default_rng(seed)
    els = P.uniform_leo(24, seed=100 + seed, radius_km=300.0)
    T = 400
    wit = O.alg1_witnesses(els, T, 1.0)
    assert len(wit) > 0
    k = g.integers(1, 40, len(els)).astype(np.int64)
    cells = O.screen(els, T, 1.0, k, mode)
    for w in wit.tolist():
        m = cells[(cells["i"] == w[0]) & (cells["j"] == w[1])]
        assert np.any((m["tlo"] <= w[2]) & (w[2] <= m["thi"])), w


def test_one_tick_segments_equal_alg1_exactly():
    """With a step of one tick every box is a single instant (Property 1), so
    the pair set is Alg 1's witness set up to the epsilon margin and FP32
    rounding; with well-separated distances it is exactly that set."""
    els = P.uniform_leo(16, seed=5, radius_km=400.0)
    T = 120
    wit = O.alg1_witnesses(els, T, 1.0)
    k = np.ones(len(els), np.int64)
    lo, hi, obj = O.boxes(els, T, 1.0, k)
    raw = O.raw_cells_sweep(lo, hi, obj)
    got = sorted((c[0], c[1], c[2]) for c in raw.tolist())
    assert all(c[2] == c[3] for c in raw.tolist())
    assert got == sorted(map(tuple, wit.tolist()))


@pytest.mark.parametrize("seed", [0, 1])
def test_alg1_sweep_equals_alg1(seed):
    """The x-swept Alg 1 finds exactly the all-pairs Alg 1 witnesses, and each
    witness's distance is the Euclidean distance of the two positions."""
    els = P.uniform_leo(60, seed=seed, radius_km=250.0)
    a = O.alg1_witnesses(els, 300, 1.0)
    b = O.alg1_sweep(els, 0, 300, 1.0)
    key = lambda w: sorted(zip(w["i"].tolist(), w["j"].tolist(), w["t"].tolist()))
    assert len(a) > 20 and key(a) == key(b)
    for w in b[:10]:
        pi = O.position(els[w["i"]], float(w["t"]))
        pj = O.position(els[w["j"]], float(w["t"]))
        assert w["dist"] == pytest.approx(np.linalg.norm(pi - pj), abs=1e-9)


def test_close_approaches_find_the_seeded_crossings():
    """Crossing pairs seeded at a known tick come within a few km then; the
    pooled close-approach search returns them, and only distances < d."""
    els = P.catalog_mixture(n=400, seed=9, crossing_frac=0.05)
    got = O.close_approaches(els, 1200, 1.0, 5.0, processes=2)
    assert len(got) > 0 and (got["dist"] < 5.0).all()
    one = O.alg1_sweep(els, 0, 1200, 1.0)
    want = one[one["dist"] < 5.0]
    key = lambda w: sorted(zip(w["i"].tolist(), w["j"].tolist(), w["t"].tolist()))
    assert key(got) == key(want)


def _keys(c):
    return sorted(zip(c["i"].tolist(), c["j"].tolist(), c["tlo"].tolist(), c["thi"].tolist()))


@pytest.mark.parametrize("seed,radius", [(4, 60.0), (5, 250.0), (6, 10.0)])
def test_aabb_tree_equals_bruteforce(seed, radius):
    """The paper's incrementally built AABB tree (Sec. 3.2) finds exactly the
    brute-force set of overlapping box pairs, from sparse to crowded."""
    els = P.uniform_leo(120, seed=seed, radius_km=radius)
    k = O.step_ticks(els, O.STEP_FIXED, 1.0, fixed_ticks=10)
    lo, hi, obj = O.boxes(els, 1200, 1.0, k)
    a = O.raw_cells_bruteforce(lo, hi, obj)
    b = O.raw_cells_tree(lo, hi, obj)
    assert len(a) > 0 and _keys(a) == _keys(b)


def test_aabb_tree_equals_sweep_on_the_small_workload():
    """n = 512, 6000 s, fixed 10 s steps: 307,712 boxes."""
    els = P.uniform_leo(512)
    k = O.step_ticks(els, O.STEP_FIXED, 1.0, fixed_ticks=10)
    lo, hi, obj = O.boxes(els, 6000, 1.0, k)
    assert _keys(O.raw_cells_tree(lo, hi, obj)) == _keys(O.raw_cells_sweep(lo, hi, obj))


def test_time_windows_partition_the_screen():
    """The CPU baseline's sample unit: the boxes whose segments start in a
    window [t0, t1) are exactly those of the whole screen starting there, and
    the sweep's pairs found from boxes starting in [t0, t1) (with the boxes
    starting before t1 + the longest box as candidates), over a partition of
    the horizon into windows, are exactly the whole screen's pairs."""
    els = P.catalog_mixture(n=150, seed=P.SEED_BASE + 41)
    T = 1500
    k = O.step_ticks(els, O.STEP_PERIOD_FRACTION, 1.0, frac=100.0)
    lo, hi, obj = O.boxes(els, T, 1.0, k, O.BOX_SPEED)
    want = O.raw_cells_sweep(lo, hi, obj)
    assert len(want) > 100
    # the boxes of a window: the whole set's boxes with tlo in [t0, t1)
    wl, wh, wo = O.boxes_starting(els, T, 1.0, k, 300, 700, O.BOX_SPEED)
    sel = (lo[:, 3] >= 300) & (lo[:, 3] < 700)
    assert np.array_equal(wl, lo[sel]) and np.array_equal(wh, hi[sel])
    assert np.array_equal(wo, obj[sel])
    longest = int(np.max(k))
    got = []
    edges = [0, 137, 400, 401, 950, 1500 + 1]
    for t0, t1 in zip(edges[:-1], edges[1:]):
        bl, bh, bo = O.boxes_starting(els, T, 1.0, k, t0, t1 + longest, O.BOX_SPEED)
        c = O.raw_cells_sweep_before(bl, bh, bo, t1)
        # a pair's cell starts where its later box starts: not before t0
        assert (c["tlo"] >= t0).all()
        got.append(c)
    got = np.concatenate(got)
    key = lambda c: np.sort(c, order=["i", "j", "tlo", "thi"]).tolist()
    assert key(got) == key(want)

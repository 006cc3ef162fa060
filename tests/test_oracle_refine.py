"""Pins of the oracle's adaptive refinement: the interval doubling and
halving of Alg 5 and Alg 6 taken top-down in bulk-synchronous rounds, and
its continuous-time variant (Sec. 4.6).

The discrete form must find exactly Alg 1's witnesses (soundness of the
interval occupancy regions, Property 1 at single ticks), its earliest must
be Alg 3's first witness, far-apart objects must need a number of boxes that
does not depend on the time step (the paper's case for growing intervals),
and the rounds are bounded by the halvings of [0, T].  The continuous form
must cover every discrete witness, find a crossing that falls between two
ticks (the tunnelling Alg 1 misses), and nest as eps shrinks."""
import math

import numpy as np
import pytest

import oracle as O
import population as P


def _key(w):
    return sorted(map(tuple, np.asarray(w).tolist()))


@pytest.mark.parametrize("start", [0.0, 64.0, 256.0])
@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
@pytest.mark.parametrize("seed", [300, 302, 310, 311])
def test_discrete_refinement_equals_alg1(mode, seed, start):
    els = P.uniform_leo(10, seed=seed, radius_km=400.0)
    T = 300
    w, rb, ntc = O.refine_discrete(els, T, 1.0, mode, start)
    ref = O.alg1_witnesses(els, T, 1.0)
    assert _key(w) == _key(ref)
    assert ntc >= len(w)
    # Alg 1's order, and the earliest is Alg 1's return value
    assert w.tolist() == ref.tolist()
    # every round halves the long intervals: at most ceil(log2(T+1)) + 2 rounds
    assert len(rb) <= math.ceil(math.log2(T + 1)) + 2
    if len(ref):
        rc, w3, _ = O.alg3(els, T, 1.0, mode, int(ref["t"][0]))
        assert rc == 1 and w3[2] == int(w["t"][0])


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
def test_far_apart_objects_cost_the_same_at_any_time_step(mode):
    # a LEO and a GEO orbit never meet; their boxes separate once the
    # intervals are a fraction of an orbit long, so the rounds and boxes do
    # not depend on the time step: 100x finer ticks, the same work (where a
    # fixed-step method does 100x more)
    els = np.array([[7000.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0],
                    [42164.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    runs = [O.refine_discrete(els, T, tick, mode) for tick, T in ((1.0, 86400), (0.01, 8640000))]
    for w, rb, ntc in runs:
        assert len(w) == 0 and ntc == 0
        assert rb.sum() <= 100
    assert runs[0][1].tolist() == runs[1][1].tolist()


def test_refinement_uses_far_fewer_boxes_than_single_ticks():
    # a sparse population: most objects are proven free over long intervals
    els = P.uniform_leo(40, seed=5, radius_km=2.5)
    T = 3000
    w, rb, _ = O.refine_discrete(els, T, 1.0, O.BOX_INTERVAL)
    assert _key(w) == _key(O.alg1_witnesses(els, T, 1.0))
    assert rb.sum() < 0.1 * len(els) * (T + 1)


def test_identical_elements_witness_every_tick():
    els = P.uniform_leo(4, seed=5)
    els[2] = els[0]
    T = 120
    w, rb, _ = O.refine_discrete(els, T, 1.0, O.BOX_SPEED)
    mine = w[(w["i"] == 0) & (w["j"] == 2)]
    assert mine["t"].tolist() == list(range(T + 1))


def _crossing_between_ticks(tc=100.5, a=7000.0, r=1.0):
    """Two circular orbits of radius a in perpendicular planes through the x
    axis, both at (a, 0, 0) at time tc: distance 0 there, but at the ticks
    either side (0.5 s away) the infinity-norm distance is a sin(n / 2),
    about 3.8 km, above r_i + r_j = 2 km."""
    n = math.sqrt(O.MU / a ** 3)
    M0 = -n * tc
    return np.array([[a, 0.0, 0.0, 0.0, 0.0, M0, r],
                     [a, 0.0, math.pi / 2, 0.0, 0.0, M0, r]])


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
def test_continuous_finds_the_crossing_alg1_tunnels_through(mode):
    els = _crossing_between_ticks()
    T = 200
    assert len(O.alg1_witnesses(els, T, 1.0)) == 0  # tunnelling at 1 s ticks
    assert len(O.refine_discrete(els, T, 1.0, mode)[0]) == 0
    spans, rb = O.refine_continuous(els, float(T), 0.1, mode)
    assert len(spans) > 0
    assert np.all(spans["t1"] - spans["t0"] <= 0.1 + 1e-12)
    assert np.any((spans["t0"] <= 100.5) & (100.5 <= spans["t1"]))
    # every span lies near the crossing: the boxes shrink with the interval
    assert spans["t0"].min() > 95.0 and spans["t1"].max() < 106.0


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
@pytest.mark.parametrize("seed", [300, 310])
def test_continuous_covers_every_discrete_witness(mode, seed):
    els = P.uniform_leo(10, seed=seed, radius_km=400.0)
    T = 300
    spans, _ = O.refine_continuous(els, float(T), 0.5, mode)
    for i, j, t in O.alg1_witnesses(els, T, 1.0).tolist():
        m = spans[(spans["i"] == i) & (spans["j"] == j)]
        assert np.any((m["t0"] <= t) & (t <= m["t1"])), (i, j, t)


def test_continuous_spans_nest_as_eps_shrinks():
    els = P.uniform_leo(10, seed=300, radius_km=400.0)
    coarse, _ = O.refine_continuous(els, 300.0, 2.0, O.BOX_INTERVAL)
    fine, _ = O.refine_continuous(els, 300.0, 0.5, O.BOX_INTERVAL)
    assert 0 < len(coarse) <= len(fine)
    for i, j, t0, t1 in fine.tolist():
        m = coarse[(coarse["i"] == i) & (coarse["j"] == j)]
        assert np.any((m["t0"] <= t0) & (t1 <= m["t1"]))


def test_continuous_robustly_safe_system_is_proven_safe():
    els = np.array([[7000.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0],
                    [42164.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    spans, rb = O.refine_continuous(els, 86400.0, 0.01, O.BOX_INTERVAL)
    assert len(spans) == 0 and rb.sum() <= 100


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
def test_round_step_reproduces_the_refinement(mode):
    """The round step applied to given boxes (used to check each GPU round
    on the GPU's own boxes): iterated from [0, T] on the oracle's boxes it
    gives the oracle refinement's intervals per round exactly, in both the
    discrete and the continuous rule."""
    els = P.uniform_leo(10, seed=310, radius_km=400.0)
    T = 300

    def run(cont, levels=None):
        cur = np.array([[i, 0, 1 if cont else T] for i in range(len(els))], np.int64)
        sizes = []
        r = 0
        while len(cur) and (levels is None or r <= levels):
            sizes.append(len(cur))
            unit = T / 2 ** r if cont else 1.0
            lo = np.zeros((len(cur), 4), np.float32)
            hi = np.zeros((len(cur), 4), np.float32)
            for q, (o, t0, t1) in enumerate(cur):
                lo[q], hi[q], _, _ = O.box(els[o], mode, int(t0), int(t1), unit)
            if cont and r == levels:
                break
            cur = O.refine_round(lo, hi, cur[:, 0], cont)
            r += 1
        return sizes

    _, orb, _ = O.refine_discrete(els, T, 1.0, mode)
    assert run(False) == orb.tolist()
    _, crb = O.refine_continuous(els, float(T), 0.5, mode)
    L = len(crb) - 1
    assert run(True, L) == crb.tolist()


def test_start_lengths_from_the_period():
    """The first-interval length for start fraction f: the largest power of
    two of ticks not above P / (f tick) (P = 2 pi sqrt(a^3 / mu)), at least
    one tick, the whole horizon when longer or f = 0; worked by hand for a
    LEO and a GEO orbit."""
    leo = [7000.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]   # P = 5828.5 s, P / 64 = 91.1
    geo = [42164.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]  # P = 86164 s, P / 64 = 1346.3
    assert O.refine_start_ticks(leo, 86400, 1.0, 64) == 64
    assert O.refine_start_ticks(geo, 86400, 1.0, 64) == 1024
    assert O.refine_start_ticks(leo, 86400, 0.5, 64) == 128    # P / 32 = 182.1
    assert O.refine_start_ticks(leo, 86400, 200.0, 64) == 1    # P / 12800 < 1
    assert O.refine_start_ticks(leo, 50, 1.0, 64) == 51        # longer than [0, 50]
    assert O.refine_start_ticks(leo, 86400, 1.0, 256) == 16    # P / 256 = 22.8
    assert O.refine_start_ticks(geo, 86400, 1.0, 128) == 512   # P / 128 = 673.2
    assert O.refine_start_ticks(leo, 86400, 1.0, 0) == 86401   # the whole horizon
    assert O.refine_start_ticks(leo, 86400, 1.0, 1e-30) == 86401
    # the first round: ceil(3001 / 64) + ceil(3001 / 1024) intervals
    _, rb, _ = O.refine_discrete(np.array([leo, geo]), 3000, 1.0, O.BOX_SPEED, 64.0)
    assert rb[0] == 47 + 3
    # and ceil(3001 / 16) + ceil(3001 / 256)
    _, rb, _ = O.refine_discrete(np.array([leo, geo]), 3000, 1.0, O.BOX_SPEED, 256.0)
    assert rb[0] == 188 + 12


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
def test_both_starts_give_the_same_witnesses_on_a_crowded_shell(mode):
    els = P.uniform_leo(24, seed=101, radius_km=300.0)
    T = 400
    w0, rb0, _ = O.refine_discrete(els, T, 1.0, mode, 0.0)
    w1, rb1, _ = O.refine_discrete(els, T, 1.0, mode, 64.0)
    assert w0.tolist() == w1.tolist() == O.alg1_witnesses(els, T, 1.0).tolist()
    assert len(w1) > 0
    # starting from intervals of 64 ticks skips the rounds in which nearly
    # every box meets every other
    assert len(rb1) < len(rb0)


@pytest.mark.parametrize("frac", [0.0, 16.0, 64.0, 256.0])
def test_rounds_within_the_budget_of_the_longest_first_interval(frac):
    """The rounds end within 2 + ceil(log2(L_max)) rounds, L_max the longest
    first interval: the halvings down to single ticks, one round to decide
    them and one for single ticks that wait for a longer interval (the GPU
    queues exactly that many rounds)."""
    els = P.uniform_leo(24, seed=101, radius_km=300.0)
    els[5] = els[3]  # a pair that meets at every tick
    T = 400
    _, rb, _ = O.refine_discrete(els, T, 1.0, O.BOX_SPEED, frac)
    lmax = max(O.refine_start_ticks(e, T, 1.0, frac) for e in els)
    budget = 2 + math.ceil(math.log2(lmax))
    assert 0 < len(rb) <= budget
    # the identical pair keeps single ticks alive to the last halving
    assert len(rb) >= 1 + math.ceil(math.log2(lmax))

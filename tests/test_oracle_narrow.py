"""Pins of the oracle's narrow phase: the collision witnesses (Def 4) inside a
screen's candidate list.  Because every true collision lies in some candidate
(soundness of the interval occupancy boxes, Sec. 7.2), the witnesses found
inside the candidates must be exactly the witnesses of the brute force Alg 1,
and the earliest of them must be Alg 1's answer (the first witness in tick,
then i, then j order) and the serial Alg 3's first witness tick (Def 5)."""
import numpy as np
import pytest

import oracle as O
import population as P


def _key(w):
    return sorted(map(tuple, np.asarray(w).tolist()))


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
@pytest.mark.parametrize("seed,kfix", [(300, 1), (302, 7), (310, 30), (310, 13), (300, 61)])
def test_witnesses_inside_candidates_equal_alg1(mode, seed, kfix):
    # large radii so that ten LEO objects collide within 300 ticks
    els = P.uniform_leo(10, seed=seed, radius_km=400.0)
    T = 300
    k = np.full(len(els), kfix, np.int64)
    cand = O.screen(els, T, 1.0, k, mode)
    first, count, margin, wit = O.narrow_phase(els, cand, 1.0)
    ref = O.alg1_witnesses(els, T, 1.0)
    assert len(ref) > 0, "the case must contain collisions"
    assert _key(wit) == _key(ref)
    # per-candidate summaries agree with the witness list
    assert int(count.sum()) == len(wit)
    for q, c in enumerate(cand.tolist()):
        mine = wit[(wit["i"] == c[0]) & (wit["j"] == c[1]) & (wit["t"] >= c[2]) & (wit["t"] <= c[3])]
        assert count[q] == len(mine)
        assert first[q] == (int(mine["t"].min()) if len(mine) else -1)
    # Def 5: the earliest witness is Alg 1's return value and Alg 3's tick
    e = O.earliest_witness(wit)
    assert e == (int(ref["i"][0]), int(ref["j"][0]), int(ref["t"][0]))
    rc, w3, _ = O.alg3(els, T, 1.0, mode, int(ref["t"][0]))
    assert rc == 1 and w3[2] == e[2]


def test_no_collision_gives_none():
    els = np.array([[7000.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0],
                    [7100.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    # a hand-made candidate over the whole horizon: the orbits stay 100 km apart
    cand = np.array([(0, 1, 0, 500)], dtype=O.CELL_DTYPE)
    first, count, margin, wit = O.narrow_phase(els, cand, 1.0)
    assert first.tolist() == [-1] and count.tolist() == [0] and len(wit) == 0
    assert O.earliest_witness(wit) is None
    # coplanar equatorial circular orbits: the Euclidean gap is never below
    # the radial 100 km and z is always 0, so the infinity norm stays at or
    # above 100 / sqrt(2); at t = 0 it is exactly 100 km (both on the x axis)
    assert 100.0 / np.sqrt(2.0) - 2.0 <= margin[0] <= 100.0 - 2.0 + 1e-9


def test_identical_elements_witness_every_tick():
    els = P.uniform_leo(4, seed=5)
    els[2] = els[0]
    cand = np.array([(0, 2, 17, 140), (0, 2, 300, 300)], dtype=O.CELL_DTYPE)
    first, count, margin, wit = O.narrow_phase(els, cand, 1.0)
    assert first.tolist() == [17, 300]
    assert count.tolist() == [124, 1]
    assert [t for (_, _, t) in wit.tolist()] == list(range(17, 141)) + [300]
    assert margin.tolist() == [2 * 2.5, 2 * 2.5]


def test_radius_boundary_decides_in_the_infinity_norm():
    # two objects on one circular equatorial orbit at angles -45 deg +- d/2
    # at t = 0: their difference points along the diagonal of x and y, so
    # the infinity-norm gap is sqrt(2) a sin(d/2), a factor sqrt(2) below the
    # Euclidean chord 2 a sin(d/2).  Radii just above / below half the
    # infinity-norm gap decide the tick (a Euclidean test would reject both).
    a, d = 7000.0, 0.01
    gap = np.sqrt(2.0) * a * np.sin(d / 2)
    for R_half, expect in [(gap / 2 + 1e-3, 1), (gap / 2 - 1e-3, 0)]:
        els = np.array([[a, 0.0, 0.0, 0.0, 0.0, -np.pi / 4 + d / 2, R_half],
                        [a, 0.0, 0.0, 0.0, 0.0, -np.pi / 4 - d / 2, R_half]])
        cand = np.array([(0, 1, 0, 0)], dtype=O.CELL_DTYPE)
        first, count, margin, _ = O.narrow_phase(els, cand, 1.0)
        assert count.tolist() == [expect]
        assert first.tolist() == [0 if expect else -1]
        assert margin[0] == pytest.approx(2e-3, abs=1e-6)


def test_crossing_pairs_have_a_witness_at_their_tick():
    els, cr = P.catalog_mixture(n=2000, seed=21, crossing_frac=0.004, horizon_s=3000.0,
                                return_crossings=True)
    sub = sorted({x for c in cr for x in c[:2]})
    e2 = els[sub]
    k = O.step_ticks(e2, O.STEP_PERIOD_FRACTION, 1.0, frac=100.0)
    cand = O.screen(e2, 3000, 1.0, k)
    first, count, _, wit = O.narrow_phase(e2, cand, 1.0)
    got = set(map(tuple, wit.tolist()))
    for (b, c, tc) in cr:
        assert (sub.index(b), sub.index(c), tc) in got


def test_bad_candidate_is_refused():
    els = P.uniform_leo(3, seed=1)
    with pytest.raises(ValueError):
        O.narrow_phase(els, np.array([(0, 3, 0, 1)], dtype=O.CELL_DTYPE), 1.0)
    with pytest.raises(ValueError):
        O.narrow_phase(els, np.array([(0, 1, 5, 4)], dtype=O.CELL_DTYPE), 1.0)


def test_relative_motion_bound_holds():
    """The skip rule of the GPU narrow phase rests on two-body facts (reading
    18): over s seconds the infinity-norm distance d of two objects falls by
    at most min(V s, w s + A s^2 / 2), V the sum of the perigee speeds, w the
    infinity norm of the relative velocity at the start, A the sum of the
    perigee gravities mu / rp^2.  Checked on the oracle's positions for
    random pairs of the catalog mixture, co-orbital pairs included."""
    g = np.random.default_rng(17)
    els = P.catalog_mixture(n=400, seed=33, crossing_frac=0.0)
    co = els[:40].copy()
    co[:, 5] += g.uniform(-0.02, 0.02, 40)  # same orbits, nearby phases
    els = np.concatenate([els, co])
    n = len(els)
    tight = 0.0
    for _ in range(3000):
        i, j = g.choice(n, 2, replace=False)
        if _ < 600:
            j = 400 + (i % 40)
            i = i % 40
        t = g.uniform(0, 86400.0)
        s = g.uniform(0.5, 3000.0)
        d0 = np.abs(O.position(els[i], t) - O.position(els[j], t)).max()
        d1 = np.abs(O.position(els[i], t + s) - O.position(els[j], t + s)).max()
        w = np.abs(O.velocity_fd(els[i], t) - O.velocity_fd(els[j], t)).max()
        V = O.max_speed(els[i]) + O.max_speed(els[j])
        A = sum(O.MU / (e[0] * (1 - e[1])) ** 2 for e in (els[i], els[j]))
        fall = min(V * s, w * s + A * s * s / 2)
        assert d1 >= d0 - fall - 1e-6
        tight = max(tight, (d0 - d1) / fall)
    assert tight > 0.9  # the bound is nearly met on some of these pairs

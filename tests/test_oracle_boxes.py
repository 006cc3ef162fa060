"""Pins of the oracle's interval occupancy regions (Def 7, Properties 1-2,
Def 8) and of its interval arithmetic (Sec. 4.5)."""
import math
import os

import numpy as np
import pytest

import oracle as O
import population as P

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_interval_examples_of_sec_4_5():
    rows = {r[0]: [float(x) for x in r[1:]] for r in _golden("interval_examples.txt")}
    xl, xh, yl, yh, ol, oh = rows["two_x_plus_y"]
    got = O.iv_add(O.iv_scale(2.0, [xl, xh]), [yl, yh])
    assert list(got) == [ol, oh]
    xl, xh, _, _, ol, oh = rows["x_times_x"]
    assert list(O.iv_mul([xl, xh], [xl, xh])) == [ol, oh]


@pytest.mark.parametrize("seed", range(5))
def test_cos_sin_ranges_are_exact(seed):
    g = np.random.default_rng(seed)
    for _ in range(200):
        x0 = g.uniform(-20, 20)
        x1 = x0 + g.choice([g.uniform(0, 0.3), g.uniform(0, 4), g.uniform(0, 8)])
        xs = np.concatenate([np.linspace(x0, x1, 4001), [x0, x1]])
        # add every extremum inside the interval to the samples
        k0, k1 = math.ceil(x0 / (math.pi / 2)), math.floor(x1 / (math.pi / 2))
        xs = np.concatenate([xs, np.arange(k0, k1 + 1) * (math.pi / 2)])
        for fn, ref in [(O.iv_cos, np.cos), (O.iv_sin, np.sin)]:
            lo, hi = fn([x0, x1])
            v = ref(xs)  # numpy's vector sin/cos may differ from libm by a few ulp
            assert lo <= v.min() + 1e-14 and hi >= v.max() - 1e-14
            assert lo >= v.min() - 1e-12 and hi <= v.max() + 1e-12
    assert list(O.iv_cos([math.pi / 3, 2 * math.pi / 3])) == pytest.approx([-0.5, 0.5], abs=1e-15)
    assert list(O.iv_cos([0.0, math.pi])) == [-1.0, 1.0]


def _contains(lo, hi, p, t):
    return bool(np.all(lo[:3] <= p) and np.all(p <= hi[:3]) and lo[3] <= t <= hi[3])


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
def test_boxes_contain_dense_samples_sound(mode):
    """Def 7: the box covers the occupancy at every time of its interval.
    Positions here come from RK4 integration of Eq. 1, an independent path."""
    els = P.catalog_mixture(n=200, seed=7, crossing_frac=0.0)
    g = np.random.default_rng(1)
    for i in g.choice(200, 25, replace=False):
        e0 = els[i]
        k = int(O.step_ticks(e0, O.STEP_PERIOD_FRACTION, 1.0, frac=50.0)[0])
        t0 = int(g.integers(0, 20000))
        lo, hi, _, _ = O.box(e0, mode, t0, t0 + k - 1, 1.0)
        r = e0[6]
        for t in np.linspace(t0, t0 + k - 1, 64):
            nu = O.nu_rk4(e0, t, 0.05)
            p = O.position_from_nu(e0, nu)
            # the whole occupancy cube of half-width r lies inside
            assert _contains(lo, hi, p - r + 1e-7, t) and _contains(lo, hi, p + r - 1e-7, t)


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
def test_property_1_single_instant_is_exact(mode):
    els = P.catalog_mixture(n=50, seed=3, crossing_frac=0.0)
    for e0 in els:
        for t in [0, 17, 5000]:
            lo, hi, _, _ = O.box(e0, mode, t, t, 1.0)
            p = O.position(e0, float(t))
            r = e0[6] + 1e-6
            # exactly the cube around pos(t), up to FP32 outward rounding
            ulp = np.spacing(np.float32(np.abs(p).max() + r))
            assert np.all(lo[:3] <= p - r) and np.all(hi[:3] >= p + r)
            assert np.all(lo[:3] >= p - r - 2 * ulp) and np.all(hi[:3] <= p + r + 2 * ulp)
            assert lo[3] == t and hi[3] == t


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
def test_property_2_monotone_in_interval(mode):
    els = P.catalog_mixture(n=60, seed=5, crossing_frac=0.0)
    g = np.random.default_rng(2)
    for e0 in els:
        t0 = int(g.integers(0, 50000))
        L = int(g.integers(1, 2000))
        lo, hi, _, _ = O.box(e0, mode, t0, t0 + L, 1.0)
        for _ in range(5):
            a = int(g.integers(t0, t0 + L + 1))
            b = int(g.integers(a, t0 + L + 1))
            lo2, hi2, _, _ = O.box(e0, mode, a, b, 1.0)
            assert np.all(lo2 >= lo) and np.all(hi2 <= hi)


def test_speed_box_half_width_and_outward_rounding():
    e0 = np.array([7000.0, 0.01, 0.5, 0.1, 0.2, 0.3, 2.5])
    lo, hi, c, hw = O.box(e0, O.BOX_SPEED, 100, 159, 1.0)
    assert hw == pytest.approx(2.5 + O.max_speed(e0) * 59.0 / 2 + 1e-6, rel=1e-15)
    assert c == pytest.approx(O.position(e0, 129.5), abs=0)
    assert np.all(lo[:3].astype(np.float64) <= c - hw)
    assert np.all(hi[:3].astype(np.float64) >= c + hw)
    # rounding is outward by at most one FP32 ulp
    assert np.all(np.nextafter(lo[:3], np.float32(np.inf)).astype(np.float64) > c - hw)
    assert np.all(np.nextafter(hi[:3], np.float32(-np.inf)).astype(np.float64) < c + hw)


def test_segments_partition_the_horizon():
    els = P.uniform_leo(8)
    k = np.array([1, 2, 3, 7, 10, 6001, 6000, 5999], dtype=np.int64)
    lo, hi, obj = O.boxes(els, 6000, 1.0, k, O.BOX_SPEED)
    for i in range(8):
        t = np.stack([lo[obj == i, 3], hi[obj == i, 3]], 1).astype(np.int64)
        assert t[0, 0] == 0 and t[-1, 1] == 6000
        assert np.all(t[1:, 0] == t[:-1, 1] + 1)
        assert np.all(t[:-1, 1] - t[:-1, 0] + 1 == k[i])

"""The seeded input generators against the recipe they state: class counts
and element ranges of the catalog mixture, the radius, the seeding, the
crossing pairs (checked through the oracle's positions: both objects of a
pair at the same place at their seeded tick, apart a few seconds earlier),
the dense shells' weight, the uniform LEO shell and the scene batch."""
import math

import numpy as np
import pytest

import oracle as O
import population as P

RE = P.RE
DEG = math.pi / 180.0


def _classes(el):
    """Row masks by the generator's class ranges (the crossing pairs are LEO)."""
    alt = el[:, 0] - RE
    hp = el[:, 0] * (1.0 - el[:, 1]) - RE
    leo = (alt >= 300.0) & (alt <= 2000.0) & (el[:, 1] <= 0.02)
    meo = (alt >= 19000.0) & (alt <= 24000.0) & (el[:, 1] <= 0.01)
    geo = (alt >= 35736.0) & (alt <= 35836.0) & (el[:, 1] <= 0.001)
    heo = (el[:, 1] >= 0.5) & (el[:, 1] <= 0.75) & (hp >= 200.0) & (hp <= 1000.0)
    return leo, meo, geo, heo


def test_catalog_mixture_classes_and_ranges():
    n = 16848
    el = P.catalog_mixture(n)
    assert el.shape == (n, 7)
    leo, meo, geo, heo = _classes(el)
    # every object in exactly one class, in the stated shares
    assert np.all(leo.astype(int) + meo + geo + heo == 1)
    assert leo.sum() == round(0.72 * n) and meo.sum() == round(0.08 * n)
    assert geo.sum() == round(0.10 * n)
    assert heo.sum() == n - leo.sum() - meo.sum() - geo.sum()
    # the classes lie in consecutive index blocks: LEO, MEO, GEO, HEO
    assert np.all(np.diff(np.argmax(np.stack([leo, meo, geo, heo]), axis=0)) >= 0)
    inc = el[:, 2] / DEG
    assert np.all((inc[meo] >= 50.0) & (inc[meo] <= 65.0))
    assert np.all(inc[geo] <= 5.0)
    assert np.all((inc[heo] >= 55.0) & (inc[heo] <= 65.0))
    # LEO inclinations in the three clusters, except the turned crossing copies
    _, cr = P.catalog_mixture(n, return_crossings=True)
    turned = np.zeros(n, bool)
    turned[[c for p in cr for c in p[:2]]] = True
    li = inc[leo & ~turned]
    in_cluster = (li <= 2.0) | ((li >= 50.6) & (li <= 52.6)) | ((li >= 65.0) & (li <= 100.0))
    assert np.all(in_cluster)
    for lo, hi in ((0.0, 2.0), (50.6, 52.6), (65.0, 100.0)):
        share = np.mean((li >= lo) & (li <= hi))
        assert abs(share - 1.0 / 3.0) < 0.02, (lo, hi, share)
    # angles in [0, 2 pi), radius 2.5 km everywhere
    assert np.all((el[:, 3:6] >= 0.0) & (el[:, 3:6] < 2.0 * math.pi))
    assert np.all(el[:, 6] == 2.5)


def test_seeding():
    a = P.catalog_mixture(2000, seed=7)
    assert np.array_equal(a, P.catalog_mixture(2000, seed=7))
    assert not np.array_equal(a, P.catalog_mixture(2000, seed=8))
    # the workloads' seeds: SEED_BASE + workload id, Philox
    assert P.SEED_BASE == 190110475
    g1, g2 = P.rng(P.SEED_BASE), np.random.Generator(np.random.Philox(P.SEED_BASE))
    assert np.array_equal(g1.uniform(size=8), g2.uniform(size=8))
    assert np.array_equal(P.uniform_leo(), P.uniform_leo(512, seed=P.SEED_BASE + 1))


@pytest.mark.parametrize("n,frac,horizon", [(16848, 0.001, 86400.0), (2000, 0.004, 1800.0)])
def test_crossing_pairs_meet_at_their_tick(n, frac, horizon):
    el, cr = P.catalog_mixture(n, crossing_frac=frac, horizon_s=horizon, return_crossings=True)
    assert len(cr) == round(frac * n / 2.0)
    seen = set()
    for b, c, tc in cr:
        assert b < c and b not in seen and c not in seen
        seen.update((b, c))
        assert 0 <= tc <= round(horizon)
        # the same circular orbit, planes turned 30-150 deg about the line of nodes
        assert el[b, 1] == el[c, 1] == 0.0
        assert np.array_equal(el[b, [0, 3, 4, 5, 6]], el[c, [0, 3, 4, 5, 6]])
        assert 30.0 - 1e-9 <= abs(el[b, 2] - el[c, 2]) / DEG <= 150.0 + 1e-9
        assert 0.0 <= el[b, 2] <= math.pi and 0.0 <= el[c, 2] <= math.pi
        pb, pc = O.position(el[b], float(tc)), O.position(el[c], float(tc))
        assert np.max(np.abs(pb - pc)) < 1e-6
        # both on the equator (the ascending node) there
        assert abs(pb[2]) < 1e-6
        # five seconds earlier they are tens of km apart (they cross, not fly together)
        qb, qc = O.position(el[b], tc - 5.0), O.position(el[c], tc - 5.0)
        assert np.max(np.abs(qb - qc)) > 10.0


def test_dense_shells_weight():
    n = 100_000
    el = P.catalog_mixture(n, seed=P.SEED_BASE + 5, dense_shells=True)
    alt = el[:, 0] - RE
    leo = (alt >= 300.0) & (alt <= 2000.0) & (el[:, 1] <= 0.02)
    n_leo = round(0.72 * n)
    # a shell's peak density is four times the background's: its share of
    # the LEO objects w / (1 + 2 w), w = 4 sigma sqrt(2 pi) / 1700 km
    w = 4.0 * 10.0 * math.sqrt(2.0 * math.pi) / 1700.0
    expect = w / (1.0 + 2.0 * w) * n_leo
    s1 = leo & (np.abs(el[:, 2] - 53.0 * DEG) < 1e-12)
    s2 = leo & (np.abs(el[:, 2] - 87.0 * DEG) < 1e-12)
    for s, centre in ((s1, 550.0), (s2, 1150.0)):
        assert abs(s.sum() - expect) < 5.0 * math.sqrt(expect)
        assert abs(np.mean(alt[s]) - centre) < 1.0
        assert abs(np.std(alt[s]) - 10.0) < 0.6


def test_uniform_leo_ranges():
    el = P.uniform_leo(4096, seed=11, radius_km=1.5)
    assert np.all((el[:, 0] >= 6678.0) & (el[:, 0] <= 8378.0))
    assert np.all((el[:, 1] >= 0.0) & (el[:, 1] <= 0.01))
    assert np.all((el[:, 2] >= 0.0) & (el[:, 2] <= 100.0 * DEG))
    assert np.all(el[:, 6] == 1.5)
    # uniform: each tenth of the semi-major axis range holds about a tenth
    h, _ = np.histogram(el[:, 0], bins=10, range=(6678.0, 8378.0))
    assert np.all(np.abs(h - 409.6) < 5.0 * math.sqrt(409.6))


def test_batch_scenes_and_band_table():
    scenes = P.batch_scenes()
    assert len(scenes) == 64
    sizes = np.array([len(e) for e, _ in scenes])
    assert abs(sizes.sum() - 1_200_000) <= 120_000
    assert np.all((sizes >= 1000) & (sizes <= 60000))
    hours = np.array([h for _, h in scenes]) / 3600.0
    assert np.all(hours == np.round(hours)) and np.all((hours >= 6) & (hours <= 72))
    # every scene is a mixture of its own seed
    e0, _ = scenes[0]
    assert np.array_equal(e0, P.catalog_mixture(len(e0), seed=(P.SEED_BASE + 4) * 1000))
    edges, fracs = P.band_table_config3()
    assert edges.tolist() == [1000.0, 2000.0, 30000.0]
    assert fracs.tolist() == [200.0, 100.0, 50.0, 400.0]

"""Pins of the serial 4D search (Alg 3 with Algs 4-6) against Alg 1, with the
loop invariants of Sec. 7.2 checked at every iteration, and of the static
decomposition (Sec. 5, Sec. 6.1)."""
import math

import numpy as np
import pytest

import oracle as O
import population as P


@pytest.mark.parametrize("mode", [O.BOX_SPEED, O.BOX_INTERVAL])
@pytest.mark.parametrize("seed", range(6))
def test_alg3_first_witness_matches_alg1(mode, seed):
    els = P.uniform_leo(10, seed=300 + seed, radius_km=150.0)
    T = 300
    wit = O.alg1_witnesses(els, T, 1.0)
    t_first = int(wit["t"].min()) if len(wit) else -1
    rc, w, iters = O.alg3(els, T, 1.0, mode, t_first)
    assert rc >= 0, "a loop invariant failed"
    if t_first < 0:
        assert rc == 0 and w is None
    else:
        assert rc == 1
        assert w[2] == t_first
        earliest = {(a, b) for a, b, t in wit.tolist() if t == t_first}
        assert (w[0], w[1]) in earliest


def test_alg3_none_when_far_apart_and_logarithmic_advances():
    # two objects on far apart circular orbits whose boxes never meet within
    # the horizon: no collision, and the interval doubling of Alg 5 keeps the
    # iteration count logarithmic in T
    els = np.array([[7000.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0],
                    [42164.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    T = 1000
    rc, w, iters = O.alg3(els, T, 1.0, O.BOX_SPEED, -1)
    assert rc == 0 and w is None
    assert iters <= 2 * (math.ceil(math.log2(T + 1)) + 1)


def test_alg3_identical_elements_collide_at_zero():
    els = P.uniform_leo(5, seed=9)
    els[3] = els[0]
    rc, w, _ = O.alg3(els, 100, 1.0, O.BOX_SPEED, 0)
    assert rc == 1 and w == (0, 3, 0)


def test_alg3_invariant_2_is_checked():
    # hand Alg 3 a wrong "first collision" tick: the invariant check fires
    els = np.array([[7000.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0],
                    [42164.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    rc, _, _ = O.alg3(els, 1000, 1.0, O.BOX_SPEED, 500)
    assert rc == -2


def test_band_edges_and_counts():
    els = P.catalog_mixture(n=3000, seed=4, crossing_frac=0.0)
    p = 16
    edges = O.band_edges(els, p)
    a = np.sort(els[:, 0])
    d = len(els) // p
    assert edges.tolist() == [a[k * d] for k in range(1, p)]
    counts = O.band_counts(els, p)
    assert counts.sum() >= len(els)
    # p = 1 keeps everything in one band
    assert O.band_counts(els, 1).tolist() == [len(els)]
    # more bands never raise the largest band (diminishing returns, Fig. 3)
    mx = [O.band_counts(els, q).max() for q in (1, 2, 4, 8, 16)]
    assert all(x >= y for x, y in zip(mx, mx[1:]))


def test_radial_range_bounds_every_position():
    els = P.catalog_mixture(n=100, seed=8, crossing_frac=0.0)
    for e0 in els:
        lo, hi = O.radial_range(e0)
        for t in np.linspace(0, 86400, 50):
            r = np.linalg.norm(O.position(e0, t))
            assert lo <= r <= hi

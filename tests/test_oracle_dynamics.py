"""Pins of the oracle's propagation (Sec. 6.1, Eq. 1) against textbook
two-body facts and against direct integration of Eq. 1."""
import math

import numpy as np
import pytest

import oracle as O

MU = 398600.4418


def el(a=7000.0, e=0.0, i=0.0, raan=0.0, argp=0.0, m0=0.0, r=1.0):
    return np.array([a, e, i, raan, argp, m0, r])


@pytest.mark.parametrize("e", [0.0, 0.01, 0.1, 0.5, 0.75])
def test_kepler_small_e_series_and_symmetry(e):
    # Lagrange series E = M + e sin M + e^2/2 sin 2M + e^3/8 (3 sin 3M - sin M) + O(e^4)
    for M in np.linspace(-3.0, 3.0, 13):
        E, _ = O.solve_kepler(M, e)
        Em, _ = O.solve_kepler(-M, e)
        assert abs(E + Em) < 1e-14  # odd in M
        if e <= 0.1:
            series = M + e * math.sin(M) + 0.5 * e * e * math.sin(2 * M) + e ** 3 / 8 * (
                3 * math.sin(3 * M) - math.sin(M))
            assert abs(E - series) < 3 * e ** 4 + 1e-15
    assert O.solve_kepler(math.pi, e)[0] == pytest.approx(math.pi, abs=1e-15)
    assert O.solve_kepler(0.0, e)[0] == 0.0


def test_circular_orbit_radius_and_uniform_rate():
    e0 = el(a=7000.0, e=0.0, i=0.7, raan=1.1, argp=0.3, m0=0.2)
    n = math.sqrt(MU / 7000.0 ** 3)
    p0 = O.position(e0, 0.0)
    for t in [1.0, 100.0, 1234.5, 5000.0]:
        p = O.position(e0, t)
        assert np.linalg.norm(p) == pytest.approx(7000.0, abs=1e-9)
        ang = math.acos(np.clip(np.dot(p0, p) / 7000.0 ** 2, -1, 1))
        want = (n * t) % (2 * math.pi)
        want = min(want, 2 * math.pi - want)
        assert ang == pytest.approx(want, abs=1e-9)


def test_node_and_plane_geometry():
    # argument of latitude 0 on a circular orbit: the ascending node, on the
    # equator at longitude RAAN; a quarter orbit later z = a sin i
    a, raan, inc = 8000.0, 0.9, 1.2
    e0 = el(a=a, e=0.0, i=inc, raan=raan, argp=0.0, m0=0.0)
    p = O.position(e0, 0.0)
    assert p == pytest.approx([a * math.cos(raan), a * math.sin(raan), 0.0], abs=1e-9)
    quarter = 0.25 * O.period(e0)
    q = O.position(e0, quarter)
    assert q[2] == pytest.approx(a * math.sin(inc), abs=1e-8)
    # moving north through the ascending node
    assert O.position(e0, 1.0)[2] > 0


@pytest.mark.parametrize("e", [0.0, 0.02, 0.5, 0.74])
def test_perigee_direction_textbook_P_vector(e):
    raan, argp, inc, a = 0.4, 1.3, 0.9, 12000.0
    e0 = el(a=a, e=e, i=inc, raan=raan, argp=argp, m0=0.0)
    cO, sO, cw, sw, ci, si = (math.cos(raan), math.sin(raan), math.cos(argp), math.sin(argp),
                              math.cos(inc), math.sin(inc))
    Pvec = np.array([cO * cw - sO * sw * ci, sO * cw + cO * sw * ci, sw * si])
    p = O.position(e0, 0.0)
    assert p == pytest.approx(a * (1 - e) * Pvec, abs=1e-8)


@pytest.mark.parametrize("e", [0.0, 0.01, 0.3, 0.75])
def test_period_closure_vis_viva_and_angular_momentum(e):
    e0 = el(a=15000.0, e=e, i=0.5, raan=2.0, argp=4.0, m0=1.0)
    P = O.period(e0)
    assert P == pytest.approx(2 * math.pi * math.sqrt(15000.0 ** 3 / MU), rel=1e-15)
    h0 = None
    for t in [0.0, 333.3, 4000.0, 9000.0]:
        p = O.position(e0, t)
        assert O.position(e0, t + P) == pytest.approx(p, abs=1e-7)
        v = O.velocity_fd(e0, t, 1e-3)
        r = np.linalg.norm(p)
        assert np.dot(v, v) == pytest.approx(MU * (2 / r - 1 / 15000.0), rel=1e-7)
        h = np.linalg.norm(np.cross(p, v))
        assert h == pytest.approx(math.sqrt(MU * 15000.0 * (1 - e * e)), rel=1e-7)
    # the speed bound used for bloating is the largest speed on the orbit
    vmax = O.max_speed(e0)
    speeds = [np.linalg.norm(O.velocity_fd(e0, t, 1e-3)) for t in np.linspace(0.0, P, 2001)]
    assert max(speeds) <= vmax * (1 + 1e-7)
    assert max(speeds) >= vmax * (1 - 1e-3)
    rp = 15000.0 * (1 - e)
    assert vmax == pytest.approx(math.sqrt(MU * (2 / rp - 1 / 15000.0)), rel=1e-12)


@pytest.mark.parametrize("e", [0.01, 0.3, 0.75])
def test_closed_form_matches_rk4_of_eq1(e):
    e0 = el(a=9000.0, e=e, i=0.3, raan=0.1, argp=0.2, m0=0.5)
    for t in [60.0, 1500.0, 6000.0]:
        nu_c = O.true_anomaly(e0, t)
        nu_r = O.nu_rk4(e0, t, 0.01)
        assert nu_c == pytest.approx(nu_r, abs=1e-9)
        # position from the integrated nu agrees to far below 1e-6 km
        d = O.position(e0, t) - O.position_from_nu(e0, nu_r)
        assert np.abs(d).max() < 1e-5 * 1e-1


def test_step_ticks_policies():
    geo = el(a=42164.17, e=0.0)
    P = O.period(geo)
    k = O.step_ticks(geo, O.STEP_PERIOD_FRACTION, 1.0, frac=100.0)[0]
    assert k * 100.0 <= P < (k + 1) * 100.0
    assert O.step_ticks(geo, O.STEP_FIXED, 1.0, fixed_ticks=10)[0] == 10
    assert O.step_ticks(geo, O.STEP_FIXED, 1.0, fixed_ticks=0)[0] == 1
    # a step never drops below one tick
    assert O.step_ticks(el(a=6600.0), O.STEP_PERIOD_FRACTION, 1.0, frac=1e9)[0] == 1
    # band table by perigee altitude
    edges, fr = [1000.0, 2000.0, 30000.0], [200.0, 100.0, 50.0, 400.0]
    low = el(a=6378.137 + 500.0)
    mid = el(a=6378.137 + 1500.0)
    meo = el(a=6378.137 + 20000.0)
    geo2 = el(a=6378.137 + 35786.0)
    for obj, f in [(low, 200.0), (mid, 100.0), (meo, 50.0), (geo2, 400.0)]:
        kb = O.step_ticks(obj, O.STEP_BAND_TABLE, 1.0, band_edges_km=edges, band_fracs=fr)[0]
        assert kb == math.floor(O.period(obj) / f)

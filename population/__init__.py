"""Seeded synthetic orbital populations (inputs only).

These catalog-shaped element sets stand in for the space-track TLE catalog of
3 April 2018 that the paper evaluates on (Sec. 6.2), which is not available.
Both the CUDA path and the oracle take their inputs from here; the module
holds no screening arithmetic.  The one orbital relation it uses is the mean
motion sqrt(mu / a^3), to place the tick at which a seeded crossing pair
meets.

Element rows: a [km], e, i, RAAN, argument of perigee, M0 [rad], radius [km].
Random numbers come from numpy's counter-based Philox generator; the seed of
workload ``c`` is 190110475 + c.
"""
from __future__ import annotations

import math

import numpy as np

MU = 398600.4418
RE = 6378.137
DEG = math.pi / 180.0
SEED_BASE = 190110475


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def _angles(g: np.random.Generator, n: int):
    return (g.uniform(0.0, 2.0 * math.pi, n), g.uniform(0.0, 2.0 * math.pi, n),
            g.uniform(0.0, 2.0 * math.pi, n))


def uniform_leo(n: int = 512, seed: int = SEED_BASE + 1, radius_km: float = 2.5) -> np.ndarray:
    """Uniform LEO shell: a ~ U(6678, 8378) km, e ~ U(0, 0.01), i ~ U(0, 100 deg),
    RAAN, argument of perigee, M0 ~ U(0, 360 deg)."""
    g = rng(seed)
    el = np.zeros((n, 7))
    el[:, 0] = g.uniform(6678.0, 8378.0, n)
    el[:, 1] = g.uniform(0.0, 0.01, n)
    el[:, 2] = g.uniform(0.0, 100.0 * DEG, n)
    el[:, 3], el[:, 4], el[:, 5] = _angles(g, n)
    el[:, 6] = radius_km
    return el


def _leo_inclinations(g, n):
    """a third near 0 deg (0-2), a third at 51.6 +- 1 deg, a third U(65, 100) deg"""
    which = g.integers(0, 3, n)
    inc = np.where(which == 0, g.uniform(0.0, 2.0, n),
                   np.where(which == 1, g.uniform(50.6, 52.6, n), g.uniform(65.0, 100.0, n)))
    return inc * DEG


def catalog_mixture(n: int = 16848, seed: int = SEED_BASE + 2, radius_km: float = 2.5,
                    crossing_frac: float = 0.001, horizon_s: float = 86400.0, tick_s: float = 1.0,
                    dense_shells: bool = False, return_crossings: bool = False):
    """Catalog-shaped mixture: 72% LEO (altitude 300-2000 km, e < 0.02,
    inclination clusters), 8% MEO (19000-24000 km), 10% GEO (35786 +- 50 km,
    i < 5 deg), 10% HEO (e 0.5-0.75, perigee altitude 200-1000 km).

    ``crossing_frac`` of the objects are made into crossing pairs: a circular
    LEO object and a copy of it whose orbital plane is turned by 30-150 deg
    about the line of nodes; both sit at the ascending node at one seeded tick
    t_c, so their distance there is zero.

    ``dense_shells`` adds two Gaussian LEO shells (sigma 10 km) at 550 km
    (i = 53 deg) and 1150 km (i = 87 deg) whose peak density is four times the
    LEO background density.
    """
    g = rng(seed)
    n_leo = int(round(0.72 * n))
    n_meo = int(round(0.08 * n))
    n_geo = int(round(0.10 * n))
    n_heo = n - n_leo - n_meo - n_geo
    el = np.zeros((n, 7))
    s = 0
    # LEO
    alt = g.uniform(300.0, 2000.0, n_leo)
    inc = _leo_inclinations(g, n_leo)
    if dense_shells:
        # each shell's weight w_s relative to the background w_b so that
        # w_s / (sigma sqrt(2 pi)) = 4 w_b / 1700 km
        w_s = 4.0 * 10.0 * math.sqrt(2.0 * math.pi) / 1700.0
        p_shell = w_s / (1.0 + 2.0 * w_s)
        u = g.uniform(0.0, 1.0, n_leo)
        s1 = u < p_shell
        s2 = (u >= p_shell) & (u < 2.0 * p_shell)
        alt = np.where(s1, g.normal(550.0, 10.0, n_leo), alt)
        alt = np.where(s2, g.normal(1150.0, 10.0, n_leo), alt)
        inc = np.where(s1, 53.0 * DEG, np.where(s2, 87.0 * DEG, inc))
    el[s:s + n_leo, 0] = RE + alt
    el[s:s + n_leo, 1] = g.uniform(0.0, 0.02, n_leo)
    el[s:s + n_leo, 2] = inc
    s += n_leo
    # MEO
    el[s:s + n_meo, 0] = RE + g.uniform(19000.0, 24000.0, n_meo)
    el[s:s + n_meo, 1] = g.uniform(0.0, 0.01, n_meo)
    el[s:s + n_meo, 2] = g.uniform(50.0, 65.0, n_meo) * DEG
    s += n_meo
    # GEO
    el[s:s + n_geo, 0] = RE + g.uniform(35736.0, 35836.0, n_geo)
    el[s:s + n_geo, 1] = g.uniform(0.0, 0.001, n_geo)
    el[s:s + n_geo, 2] = g.uniform(0.0, 5.0, n_geo) * DEG
    s += n_geo
    # HEO
    ecc = g.uniform(0.5, 0.75, n_heo)
    hp = g.uniform(200.0, 1000.0, n_heo)
    el[s:s + n_heo, 0] = (RE + hp) / (1.0 - ecc)
    el[s:s + n_heo, 1] = ecc
    el[s:s + n_heo, 2] = g.uniform(55.0, 65.0, n_heo) * DEG
    s += n_heo
    el[:, 3], el[:, 4], el[:, 5] = _angles(g, n)
    el[:, 6] = radius_km

    crossings = []
    n_pairs = int(round(crossing_frac * n / 2.0))
    if n_pairs > 0:
        idx = g.permutation(n_leo)[:2 * n_pairs]
        T_ticks = int(round(horizon_s / tick_s))
        for p in range(n_pairs):
            b, c = int(idx[2 * p]), int(idx[2 * p + 1])
            tc = int(g.integers(0, T_ticks + 1))
            while True:
                d = g.uniform(30.0, 150.0) * DEG
                i0 = el[b, 2]
                if i0 + d <= math.pi:
                    i1 = i0 + d
                    break
                if i0 - d >= 0.0:
                    i1 = i0 - d
                    break
            el[b, 1] = 0.0
            n_mot = math.sqrt(MU / el[b, 0] ** 3)
            # argument of latitude omega + M0 + n t is zero at t_c
            m0 = math.fmod(-el[b, 4] - n_mot * tc * tick_s, 2.0 * math.pi)
            if m0 < 0.0:
                m0 += 2.0 * math.pi
            el[b, 5] = m0
            el[c] = el[b]
            el[c, 2] = i1
            crossings.append((min(b, c), max(b, c), tc))
    if return_crossings:
        return el, crossings
    return el


def band_table_config3():
    """Step fractions by perigee altitude band: below 1000 km P/200,
    1000-2000 km P/100, 2000-30000 km P/50, above 30000 km P/400."""
    return np.array([1000.0, 2000.0, 30000.0]), np.array([200.0, 100.0, 50.0, 400.0])


def batch_scenes(n_scenes: int = 64, seed: int = SEED_BASE + 4, total: int = 1_200_000,
                 lo: float = 1e3, hi: float = 6e4):
    """Scene sizes log-uniform on [lo, hi], redrawn until their total is within
    10% of ``total``; horizons are whole hours uniform on [6, 72]."""
    g = rng(seed)
    while True:
        sizes = np.exp(g.uniform(math.log(lo), math.log(hi), n_scenes)).astype(np.int64)
        if abs(int(sizes.sum()) - total) <= 0.1 * total:
            break
    hours = g.integers(6, 73, n_scenes)
    scenes = []
    for s in range(n_scenes):
        el = catalog_mixture(int(sizes[s]), seed=seed * 1000 + s)
        scenes.append((el, float(hours[s]) * 3600.0))
    return scenes

"""Pins of the step-network oracle: its gradient against central finite
differences of its own loss in FP64 (independent of the chain-rule code),
a hand-computed network, BF16 rounding against bit-level definitions."""
import numpy as np
import pytest

from oracle import stepnet as S


def _params(seed, scale=0.5):
    g = np.random.default_rng(seed)
    return (g.standard_normal(S.N_PARAMS) * scale).astype(np.float32)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences(seed):
    g = np.random.default_rng(10 + seed)
    p = _params(seed).astype(np.float64)
    X = g.standard_normal((16, S.IN))
    T = g.standard_normal(16)
    _, grad = S.loss_and_grad(p, X, T, round_weights=False)

    def loss_at(q):
        # evaluate in FP64 without the FP32 round trip of unpack
        o = 0
        W1 = q[o:o + 512].reshape(8, 64); o += 512
        b1 = q[o:o + 64]; o += 64
        W2 = q[o:o + 4096].reshape(64, 64); o += 4096
        b2 = q[o:o + 64]; o += 64
        w3 = q[o:o + 64]; o += 64
        b3 = q[o]
        y = np.maximum(np.maximum(X @ W1 + b1, 0) @ W2 + b2, 0) @ w3 + b3
        return np.mean((y - T) ** 2)

    idx = g.choice(S.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [S.N_PARAMS - 1, 0, 512, 4672]])
    p32 = p.astype(np.float32).astype(np.float64)
    for k in idx:
        h = 1e-6
        e = np.zeros_like(p32)
        e[k] = h
        fd = (loss_at(p32 + e) - loss_at(p32 - e)) / (2 * h)
        assert fd == pytest.approx(grad[k], rel=1e-4, abs=1e-7), k


def test_hand_computed_network():
    # W1 passes x0 to unit 0 and -x0 to unit 1; W2 copies them; w3 = (1, 1):
    # y = relu(x0) + relu(-x0) + b3 = |x0| + b3
    p = np.zeros(S.N_PARAMS, np.float32)
    p[0 * 64 + 0] = 1.0
    p[0 * 64 + 1] = -1.0
    w2 = 512 + 64
    p[w2 + 0 * 64 + 0] = 1.0
    p[w2 + 1 * 64 + 1] = 1.0
    w3 = w2 + 4096 + 64
    p[w3 + 0] = 1.0
    p[w3 + 1] = 1.0
    p[-1] = 0.25
    X = np.zeros((4, 8))
    X[:, 0] = [-2.0, -0.5, 0.0, 3.0]
    assert S.forward(p, X).tolist() == [2.25, 0.75, 0.25, 3.25]


def test_bf16_rounding_definition():
    vals = np.array([1.0, 1.00390625, 1.005859375, 1.0078125 + 2 ** -9, -3.3, 1e-30], np.float32)
    got = S.bf16(vals)
    # 1 + 2^-8 is the midpoint between 1 and 1 + 2^-7: ties to even -> 1
    assert got[0] == 1.0 and got[1] == 1.0
    # 1 + 3*2^-9 is above that midpoint -> 1 + 2^-7
    assert got[2] == 1.0078125
    for v, r in zip(vals, got):
        assert abs(r - v) <= abs(v) * 2 ** -8


def test_features_and_learned_step_clamp():
    els = np.array([[7000.0, 0.01, 0.5, 0, 0, 0, 1.0], [42164.0, 0.0, 0.0, 0, 0, 0, 1.0],
                    [7030.0, 0.0, 1.0, 0, 0, 0, 1.0]])
    f = S.features(els)
    assert f[0, 1] == 0.01 and f[1, 7] == 0.0 and f[0, 7] == pytest.approx(np.log(2.0))
    assert f[1, 6] == pytest.approx(np.log(2 * np.pi * np.sqrt(42164.0 ** 3 / S.MU) / 3600))
    P = 2 * np.pi * np.sqrt(els[:, 0] ** 3 / S.MU)
    ks = S.learned_step_seconds(els, [100.0, -100.0, np.log(P[2] / 100)])
    assert ks[0] == pytest.approx(P[0] / 50) and ks[1] == pytest.approx(P[1] / 400)
    assert ks[2] == pytest.approx(P[2] / 100)


def test_feature_columns_by_hand():
    """Every feature column against values worked out by hand for objects
    chosen so that most of them are round numbers: a circular orbit 100 km up
    at i = 0, a polar orbit with perigee 100 km and apogee 10000 km up, and
    three circular orbits at inclination 30 deg whose middle one has a period
    of exactly one day, 30 km above and below it the other two."""
    RE, MU = 6378.137, 398600.4418
    a_day = (MU * (86400.0 / (2 * np.pi)) ** 2) ** (1.0 / 3.0)  # Kepler's third law
    a_polar = RE + (100.0 + 10000.0) / 2.0
    e_polar = (10000.0 - 100.0) / 2.0 / a_polar
    els = np.array([
        [RE + 100.0, 0.0, 0.0, 0.1, 0.2, 0.3, 1.0],
        [a_polar, e_polar, np.pi / 2, 0.1, 0.2, 0.3, 1.0],
        [a_day, 0.0, np.pi / 6, 0.1, 0.2, 0.3, 1.0],
        [a_day + 30.0, 0.0, np.pi / 6, 0.1, 0.2, 0.3, 1.0],
        [a_day - 30.0, 0.0, np.pi / 6, 0.1, 0.2, 0.3, 1.0],
    ])
    f = S.features(els)
    h_day = a_day - RE
    want = np.array([
        # log(a/RE), e, sin i, cos i, log(hp/100), log(ha/100), log(P/1h), log(1+density)
        [np.log((RE + 100.0) / RE), 0.0, 0.0, 1.0, 0.0, 0.0,
         np.log(2 * np.pi / np.sqrt(MU / (RE + 100.0) ** 3) / 3600.0), 0.0],
        [np.log(a_polar / RE), 4950.0 / a_polar, 1.0, 0.0, 0.0, np.log(100.0),
         np.log(2 * np.pi / np.sqrt(MU / a_polar ** 3) / 3600.0), 0.0],
        [np.log(a_day / RE), 0.0, 0.5, np.sqrt(3) / 2, np.log(h_day / 100.0),
         np.log(h_day / 100.0), np.log(24.0), np.log(3.0)],
        [np.log((a_day + 30.0) / RE), 0.0, 0.5, np.sqrt(3) / 2, np.log((h_day + 30.0) / 100.0),
         np.log((h_day + 30.0) / 100.0), None, np.log(2.0)],
        [np.log((a_day - 30.0) / RE), 0.0, 0.5, np.sqrt(3) / 2, np.log((h_day - 30.0) / 100.0),
         np.log((h_day - 30.0) / 100.0), None, np.log(2.0)],
    ], dtype=object)
    for r in range(len(els)):
        for c in range(8):
            if want[r, c] is not None:
                assert f[r, c] == pytest.approx(float(want[r, c]), abs=1e-12), (r, c)
    # the period grows as a^1.5: 30 km more on a one-day orbit is +0.107%
    assert f[3, 6] - f[2, 6] == pytest.approx(1.5 * np.log1p(30.0 / a_day), abs=1e-12)
    # the pins have teeth: a swap of sin i and cos i, or of the perigee and
    # apogee altitudes, or of log a and log P, changes some row
    for c1, c2 in ((2, 3), (4, 5), (0, 6)):
        assert np.abs(f[:, c1] - f[:, c2]).max() > 0.1

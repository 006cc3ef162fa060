"""Parity of the CUDA narrow phase (scd_narrow_phase, through the C ABI) with
the oracle's narrow phase, which tests every tick of every candidate with
Alg 1's predicate (Defs 2-4).

The per-candidate first witness tick and witness count are integers decided
by FP64 comparisons of positions that agree with the oracle's within 1e-6
km each; the infinity-norm distance of two of them then agrees within
2e-6 km, so they must be equal for every candidate whose oracle distances
stay more than 2e-6 km away from r_i + r_j at every tick of its interval (a
decision closer than that could go either way between the two
propagations; such candidates are counted and must be rare).  The earliest
witness (Def 5, in Alg 1's order of tick, then i, then j) must be equal.
"""
import numpy as np
import pytest
import torch

import oracle as O
import population as P

pytestmark = pytest.mark.gpu

# two positions within 1e-6 km each: their distance within 2e-6 km
BOUNDARY_KM = 2e-6


@pytest.fixture(scope="module")
def scd():
    import paper_1901_10475_gb300 as m
    torch.cuda.set_device(0)
    return m


def _screen(scd, els, horizon_s, step, mode=None):
    kw = {} if mode is None else {"mode": mode}
    sc = scd.Scene(els, horizon_s, 1.0, step=step, **kw)
    sc.build_boxes()
    pairs = sc.find_pairs_device()
    return sc, pairs


def _cells(scd, pairs):
    return scd.pairs_from_device(pairs).astype(O.CELL_DTYPE)


def _check(els, cells, first, count):
    """GPU first/count (host arrays) against the oracle on the host candidate
    list cells; returns the number of boundary candidates left out."""
    of, oc, om, _ = O.narrow_phase(els, cells, 1.0, witnesses=False)
    gf = np.asarray(first)
    gc = np.asarray(count).view(np.uint32)
    ok = om > BOUNDARY_KM
    assert np.array_equal(gf[ok], of[ok])
    assert np.array_equal(gc[ok], oc[ok])
    return int((~ok).sum())


def _host(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed,kfix", [(300, 1), (302, 7), (310, 30), (300, 61)])
def test_small_large_radii_equals_oracle_and_alg1(scd, mode, seed, kfix):
    els = P.uniform_leo(10, seed=seed, radius_km=400.0)
    step = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=kfix)
    sc, pairs = _screen(scd, els, 300.0, step, mode)
    cells = _cells(scd, pairs)
    first, count, w = sc.narrow_phase(pairs)
    assert _check(els, cells, _host(first), _host(count)) == 0
    ref = O.alg1_witnesses(els, 300, 1.0)
    assert int(count.cpu().numpy().sum()) == len(ref)
    assert w == (int(ref["i"][0]), int(ref["j"][0]), int(ref["t"][0]))
    sc.close()


def test_uniform_512_six_thousand_seconds(scd):
    # n = 512, 6000 s, fixed 10 s steps, r = 2.5 km; plus one pair of
    # identical elements, which collide at every tick
    els = P.uniform_leo(512)
    els[511] = els[7]
    step = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    sc, pairs = _screen(scd, els, 6000.0, step)
    cells = _cells(scd, pairs)
    first, count, w = sc.narrow_phase(pairs)
    assert _check(els, cells, _host(first), _host(count)) == 0
    m = (cells["i"] == 7) & (cells["j"] == 511)
    assert cells[m].tolist() == [(7, 511, 0, 6000)]
    assert count.cpu().numpy()[m].tolist() == [6001]
    _, _, _, wit = O.narrow_phase(els, cells, 1.0)
    assert w == O.earliest_witness(wit) == (7, 511, 0)
    sc.close()


def test_catalog_mixture_crossings(scd):
    els, cr = P.catalog_mixture(n=2000, seed=21, crossing_frac=0.004, horizon_s=1800.0,
                                return_crossings=True)
    step = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc, pairs = _screen(scd, els, 1800.0, step)
    cells = _cells(scd, pairs)
    first, count, w = sc.narrow_phase(pairs)
    skipped = _check(els, cells, _host(first), _host(count))
    assert skipped <= 2
    gf = first.cpu().numpy()
    for (b, c, tc) in cr:
        m = np.nonzero((cells["i"] == b) & (cells["j"] == c) & (cells["tlo"] <= tc) &
                       (tc <= cells["thi"]))[0]
        assert len(m) == 1 and 0 <= gf[m[0]] <= tc
    _, _, _, wit = O.narrow_phase(els, cells, 1.0)
    assert w == O.earliest_witness(wit)
    sc.close()


def test_full_24h_catalog_sampled(scd):
    """The 24 h screen of the 16,848-object catalog mixture (P/100 steps,
    SPEED boxes) as the benchmark runs it: 3000 sampled candidates, up to
    2000 candidates with a witness and the planted crossings against the
    oracle; the earliest witness is the smallest first tick (Alg 1 order)."""
    els, cr = P.catalog_mixture(return_crossings=True)
    step = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc, pairs = _screen(scd, els, 86400.0, step)
    first, count, w = sc.narrow_phase(pairs)
    m = pairs.shape[0]
    hit = torch.nonzero(first >= 0).flatten()
    g = np.random.default_rng(5)
    sel = np.union1d(g.choice(m, 3000, replace=False), _host(hit[:2000]))
    sel_d = torch.as_tensor(sel, device="cuda")
    cells = _cells(scd, pairs[sel_d].contiguous())
    assert _check(els, cells, _host(first[sel_d]), _host(count[sel_d])) <= 2
    for (b, c, tc) in cr:
        q = torch.nonzero((pairs[:, 0] == b) & (pairs[:, 1] == c) & (pairs[:, 2] <= tc) &
                          (pairs[:, 3] >= tc)).flatten()
        assert q.numel() == 1
        assert 0 <= int(first[q[0]]) <= tc
    # Alg 1 order over the candidates with a witness
    assert hit.numel() > 0 and w is not None
    t0 = int(first[hit].min())
    at_t0 = hit[first[hit] == t0]
    ij = sorted((int(pairs[q, 0]), int(pairs[q, 1])) for q in _host(at_t0))
    assert w == (ij[0][0], ij[0][1], t0)
    mt = sc.metrics()
    ev, ev64 = mt["narrow_evals"], mt["narrow_evals_fp64"]
    ticks = int((pairs[:, 3].long() - pairs[:, 2].long() + 1).sum())
    assert 0 < ev < ticks  # the skip bound does skip (parity above: soundly)
    assert 0 < ev64 < ev  # most ticks are decided by the FP32 tier's bounds
    sc.close()


def test_edge_cases(scd):
    els = P.uniform_leo(16, seed=3)
    step = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    sc = scd.Scene(els, 600.0, 1.0, step=step)
    empty = torch.zeros((0, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(scd.ScdError) as e:
        sc.narrow_phase(empty)  # boxes not built yet
    assert e.value.status == scd.SCD_ERR_STATE
    sc.build_boxes()
    first, count, w = sc.narrow_phase(empty)
    assert w is None and first.numel() == 0
    # an object index out of range and an empty interval are refused; the
    # valid candidate beside them is still answered
    bad = torch.tensor([[0, 16, 0, 5], [3, 3, 0, 4], [1, 2, 9, 8]], dtype=torch.int32,
                       device="cuda")
    with pytest.raises(scd.ScdError) as e:
        sc.narrow_phase(bad)
    assert e.value.status == scd.SCD_ERR_INVALID_ARG
    # one object paired with itself: distance 0 at every tick of [0, 4]
    first, count, w = sc.narrow_phase(bad[1:2].contiguous())
    assert first.cpu().tolist() == [0] and count.cpu().tolist() == [5] and w == (3, 3, 0)
    # a tick beyond the horizon is refused
    with pytest.raises(scd.ScdError):
        sc.narrow_phase(torch.tensor([[0, 1, 590, 601]], dtype=torch.int32, device="cuda"))
    sc.close()

"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: positions within 1e-6 km of the FP64 oracle; integer step
lengths and tick fields bit-exact; FP32 box faces equal to the oracle's
outward-rounded faces up to one FP32 ulp (both round FP64 values that agree
to ~1e-12 km, so only values within 1e-12 km of a rounding boundary may land
one ulp apart); candidate pair sets bit-exact against the oracle run on the
same FP32 boxes.
"""
import numpy as np
import pytest
import torch

import oracle as O
import population as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scd():
    import paper_1901_10475_gb300 as m
    torch.cuda.set_device(0)
    return m


def _host_boxes(sc):
    lo, hi, obj = sc.boxes()
    return lo.cpu().numpy(), hi.cpu().numpy(), obj.cpu().numpy().view(np.uint32)


def _same(got, want):
    g = np.asarray(got).view(np.int32).reshape(-1, 4)
    w = np.asarray(want).view(np.int32).reshape(-1, 4)
    return g.shape == w.shape and bool((g == w).all())


def _gpu_positions(scd, els, obj, t):
    d_el = torch.as_tensor(np.ascontiguousarray(els), device="cuda")
    d_obj = torch.as_tensor(np.asarray(obj, np.int32), device="cuda")
    d_t = torch.as_tensor(np.asarray(t, np.float64), device="cuda")
    out = torch.zeros((len(t), 3), dtype=torch.float64, device="cuda")
    scd.scd_propagate(d_el.data_ptr(), len(els), d_obj.data_ptr(), d_t.data_ptr(), len(t),
                      out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_positions_match_fp64_oracle(scd):
    els = P.catalog_mixture(n=3000, seed=11)
    g = np.random.default_rng(0)
    obj = g.integers(0, len(els), 20000)
    t = g.uniform(0, 3 * 86400.0, 20000)
    gp = _gpu_positions(scd, els, obj, t)
    op = O.positions(els, obj, t)
    assert np.abs(gp - op).max() < 1e-6


def _high_e_elements(n=400, seed=19):
    """Closed orbits with e in [0.9, 0.99] and perigee 300-2000 km above the
    surface: the mixed-precision Kepler solve's hardest cases (perigee)."""
    g = np.random.default_rng(seed)
    e = g.uniform(0.9, 0.99, n)
    rp = 6378.137 + g.uniform(300.0, 2000.0, n)
    els = np.zeros((n, 7))
    els[:, 0] = rp / (1.0 - e)
    els[:, 1] = e
    els[:, 2] = g.uniform(0.0, np.pi, n)
    els[:, 3:6] = g.uniform(0.0, 2 * np.pi, (n, 3))
    els[:, 6] = 2.5
    return els


def test_positions_high_eccentricity(scd):
    els = _high_e_elements()
    g = np.random.default_rng(1)
    obj = g.integers(0, len(els), 20000)
    t = g.uniform(0, 86400.0, 20000)
    gp = _gpu_positions(scd, els, obj, t)
    op = O.positions(els, obj, t)
    assert np.abs(gp - op).max() < 1e-6


@pytest.mark.parametrize("mode", [0, 1])
def test_boxes_high_eccentricity(scd, mode):
    """Box faces within one FP32 ulp of the oracle's for e up to 0.99."""
    els = _high_e_elements(n=120, seed=20)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc = scd.Scene(els, 43200.0, 1.0, pol, mode=mode).build_boxes()
    lo, hi, obj = _host_boxes(sc)
    k = O.step_ticks(els, O.STEP_PERIOD_FRACTION, 1.0, frac=100.0)
    olo, ohi, oobj = O.boxes(els, 43200, 1.0, k, mode)
    assert (obj == oobj).all()
    for a, b, direction in [(lo, olo, -np.inf), (hi, ohi, np.inf)]:
        a3, b3 = a[:, :3], b[:, :3]
        near = (a3 == b3) | (np.nextafter(b3, np.float32(direction)) == a3) | (
            np.nextafter(a3, np.float32(direction)) == b3)
        assert near.all()
    sc.close()


@pytest.mark.parametrize("policy", ["fixed", "period", "band"])
def test_step_lengths_bit_exact(scd, policy):
    els = P.catalog_mixture(n=4000, seed=12)
    if policy == "fixed":
        pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=37)
        want = O.step_ticks(els, O.STEP_FIXED, 1.0, fixed_ticks=37)
    elif policy == "period":
        pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
        want = O.step_ticks(els, O.STEP_PERIOD_FRACTION, 1.0, frac=100.0)
    else:
        edges, fr = P.band_table_config3()
        pol = scd.make_step_policy(scd.SCD_STEP_BAND_TABLE, band_edges_km=edges, band_fractions=fr)
        want = O.step_ticks(els, O.STEP_BAND_TABLE, 1.0, band_edges_km=edges, band_fracs=fr)
    sc = scd.Scene(els, 86400.0, 1.0, pol).build_boxes()
    got = sc.steps().cpu().numpy()
    assert (got == want).all()
    sc.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_boxes_match_oracle(scd, mode):
    els = P.catalog_mixture(n=300, seed=13)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc = scd.Scene(els, 21600.0, 1.0, pol, mode=mode).build_boxes()
    lo, hi, obj = _host_boxes(sc)
    k = O.step_ticks(els, O.STEP_PERIOD_FRACTION, 1.0, frac=100.0)
    olo, ohi, oobj = O.boxes(els, 21600, 1.0, k, mode)
    assert (obj == oobj).all()
    assert (lo[:, 3] == olo[:, 3]).all() and (hi[:, 3] == ohi[:, 3]).all()
    for a, b, direction in [(lo, olo, -np.inf), (hi, ohi, np.inf)]:
        a3, b3 = a[:, :3], b[:, :3]
        near = (a3 == b3) | (np.nextafter(b3, np.float32(direction)) == a3) | (
            np.nextafter(a3, np.float32(direction)) == b3)
        assert near.all()
        assert (a3 == b3).mean() > 0.999
    sc.close()


def _screen_parity(scd, els, T, pol, mode=0, tuning=None, raw_too=True):
    sc = scd.Scene(els, float(T), 1.0, pol, mode=mode, tuning=tuning).build_boxes()
    got = sc.find_pairs()
    lo, hi, obj = _host_boxes(sc)
    raw = O.raw_cells_sweep(lo, hi, obj)
    want = O.canonicalize(raw)
    assert _same(got, want), (len(got), len(want))
    if raw_too:
        graw = scd.pairs_from_device(sc.find_raw_cells_device())
        order = np.lexsort((raw["thi"], raw["tlo"], raw["j"], raw["i"]))
        assert _same(graw, raw[order]), (len(graw), len(raw))
    m = sc.metrics()
    sc.close()
    return got, m


def test_config1_uniform_leo_pair_set_bit_exact(scd):
    """n=512, 6000 s, fixed 10 s steps (the small workload)."""
    els = P.uniform_leo(512)
    pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    got, m = _screen_parity(scd, els, 6000, pol)
    assert m["boxes"] == 512 * 601
    # the second oracle: the paper's incrementally built AABB tree
    sc = scd.Scene(els, 6000.0, 1.0, pol).build_boxes()
    lo, hi, obj = _host_boxes(sc)
    sc.close()
    assert _same(got, O.canonicalize(O.raw_cells_tree(lo, hi, obj)))


@pytest.mark.parametrize("leaf", [1, 2, 4, 8])
@pytest.mark.parametrize("bits", [8, 10, 16])
def test_tunings_give_identical_sets(scd, leaf, bits):
    els = P.uniform_leo(200, seed=77, radius_km=40.0)
    pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=7)
    tuning = dict(leaf_size=leaf, morton_bits=bits, stack_depth=32, block_threads=64,
                  space_warp=int(bits == 10),
                  time_scale={8: 4.0, 10: 1.0, 16: 0.5}[bits],
                  nodes_per_step=1 if bits == 10 else 2,
                  node_width=4 if leaf == 1 and bits != 10 else 2)
    _screen_parity(scd, els, 1500, pol, tuning=tuning, raw_too=(leaf == 4))


@pytest.mark.parametrize("mode", [0, 1])
def test_mixture_variable_steps_bit_exact(scd, mode):
    els = P.catalog_mixture(n=600, seed=31, radius_km=25.0)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    got, m = _screen_parity(scd, els, 20000, pol, mode=mode)
    assert len(got) > 100


@pytest.mark.parametrize("split_km,time_scale", [(0.0, 1.0), (-1000.0, 4.0), (1000.0, 16.0),
                                                 (-300.0, 0.25)])
def test_key_order_options_bit_exact(scd, split_km, time_scale):
    # the mixture has boxes on both sides of every threshold (LEO, MEO, GEO,
    # HEO SPEED boxes): the size split and the time weight only reorder the
    # tree, so the pair list stays the oracle's
    els = P.catalog_mixture(n=600, seed=32, radius_km=25.0)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    tuning = dict(split_km=split_km, time_scale=time_scale)
    got, m = _screen_parity(scd, els, 20000, pol, tuning=tuning)
    assert len(got) > 100


@pytest.mark.parametrize("leaf", [1, 4])
def test_runs_too_wide_to_pack(scd, leaf):
    """1 ms ticks over 6000 s (23 tick bits) and 600 objects (10 bits): a run
    record's key and last tick no longer fit one 64-bit word together, so the
    last tick travels as a sort value."""
    els = P.catalog_mixture(n=600, seed=34, radius_km=25.0)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc = scd.Scene(els, 6000.0, 0.001, pol, tuning=dict(leaf_size=leaf)).build_boxes()
    got = sc.find_pairs()
    lo, hi, obj = _host_boxes(sc)
    want = O.canonicalize(O.raw_cells_sweep(lo, hi, obj))
    assert len(want) > 50 and int(want["thi"].max()) >= 1 << 22
    assert _same(got, want), (len(got), len(want))
    sc.close()


def test_band_table_steps_bit_exact(scd):
    els = P.catalog_mixture(n=500, seed=32, radius_km=25.0)
    edges, fr = P.band_table_config3()
    pol = scd.make_step_policy(scd.SCD_STEP_BAND_TABLE, band_edges_km=edges, band_fractions=fr)
    _screen_parity(scd, els, 15000, pol)


@pytest.mark.parametrize("case", ["one", "two_identical", "one_tick", "single_segment",
                                  "ragged", "far_apart"])
def test_edge_cases(scd, case):
    base = P.uniform_leo(40, seed=5, radius_km=30.0)
    pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    T = 600
    if case == "one":
        els = base[:1]
    elif case == "two_identical":
        els = np.stack([base[0], base[0]])
    elif case == "one_tick":
        els, T = base, 1
    elif case == "single_segment":
        els, T = base[:8], 600
        pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=5000)
    elif case == "ragged":
        els, T = base[:37], 613
        pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=7)
    else:
        els = np.array([[42164.0, 0, 0, 0, 0, 0, 1.0], [7000.0, 0, 0, 0, 0, 0, 1.0]])
    got, _ = _screen_parity(scd, els, T, pol)
    if case == "one" or case == "far_apart":
        assert len(got) == 0
    if case == "two_identical":
        assert got.tolist() == [(0, 1, 0, T)]


def test_soundness_covers_every_alg1_witness(scd):
    els = P.uniform_leo(24, seed=101, radius_km=300.0)
    T = 400
    wit = O.alg1_witnesses(els, T, 1.0)
    assert len(wit) > 0
    pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=13)
    sc = scd.Scene(els, float(T), 1.0, pol).build_boxes()
    got = sc.find_pairs()
    for w in wit.tolist():
        m = got[(got["i"] == w[0]) & (got["j"] == w[1])]
        assert np.any((m["tlo"] <= w[2]) & (w[2] <= m["thi"])), w
    sc.close()


def test_buffer_too_small_reports_count_and_state_errors(scd):
    els = P.uniform_leo(100, seed=9, radius_km=80.0)
    pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    sc = scd.Scene(els, 600.0, 1.0, pol)
    with pytest.raises(scd.ScdError) as e:
        sc.find_pairs()
    assert e.value.status == scd._binding.SCD_ERR_STATE
    sc.build_boxes()
    full = sc.find_pairs()
    assert len(full) > 2
    out = np.zeros(1, scd.PAIR_DTYPE)
    import ctypes
    n = ctypes.c_int64(0)
    rc = scd._binding.lib().scd_find_pairs(sc.handle, None, out.ctypes.data, 1, ctypes.byref(n))
    assert rc == scd._binding.SCD_ERR_BUFFER_TOO_SMALL and n.value == len(full)
    sc.close()


def test_full_size_catalog_sampled_parity(scd):
    """n=16848, 24 h, steps P/100 (the timed workload, same launch path as
    the benchmark): every pair involving a sample of objects, including all
    seeded crossing pairs, equals the oracle's on the same boxes; boxes are
    spot-checked against the oracle one by one."""
    els, cr = P.catalog_mixture(n=16848, seed=P.SEED_BASE + 2, return_crossings=True)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    sc = scd.Scene(els, 86400.0, 1.0, pol).build_boxes()
    got = sc.find_pairs()
    lo, hi, obj = _host_boxes(sc)
    g = np.random.default_rng(5)
    sel_ids = sorted(set(g.choice(len(els), 6, replace=False).tolist()) | {cr[0][0], cr[0][1]})
    sel = np.zeros(len(els), np.uint8)
    sel[sel_ids] = 1
    want = O.canonicalize(O.raw_cells_selected(lo, hi, obj, sel))
    mine = got[(sel[got["i"]] == 1) | (sel[got["j"]] == 1)]
    assert _same(mine, want), (len(mine), len(want))
    # every seeded crossing is reported at its tick
    for b, c, tc in cr:
        m = got[(got["i"] == b) & (got["j"] == c)]
        assert np.any((m["tlo"] <= tc) & (tc <= m["thi"])), (b, c, tc)
    # output is sorted and merged
    key = got["i"].astype(np.int64) << 40 | got["j"].astype(np.int64) << 20 | got["tlo"]
    assert np.all(np.diff(key) > 0)
    same = (got["i"][1:] == got["i"][:-1]) & (got["j"][1:] == got["j"][:-1])
    assert np.all(got["tlo"][1:][same] > got["thi"][:-1][same] + 1)
    # spot-check boxes against the oracle
    k = O.step_ticks(els, O.STEP_PERIOD_FRACTION, 1.0, frac=100.0)
    idx = g.choice(len(lo), 3000, replace=False)
    for b in idx:
        i = int(obj[b])
        olo, ohi, _, _ = O.box(els[i], 0, int(lo[b, 3]), int(hi[b, 3]), 1.0)
        assert np.all(np.abs(olo.astype(np.float64) - lo[b]) <= np.spacing(np.abs(olo)))
        assert np.all(np.abs(ohi.astype(np.float64) - hi[b]) <= np.spacing(np.abs(ohi)))
    sc.close()

"""The step network's GPU kernels against the FP64 oracle (forward pass,
gradient, features), its training and checkpoint, the LEARNED step policy,
and what the trained network gains over the period rule."""
import numpy as np
import pytest
import torch

import oracle as O
import population as P
from oracle import stepnet as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import paper_1901_10475_gb300 as m
    from paper_1901_10475_gb300 import stepnet as sn
    torch.cuda.set_device(0)
    return m, sn


def test_forward_and_gradient_match_oracle(mods):
    scd, sn = mods
    net = sn.StepNet(seed=3)
    g = np.random.default_rng(0)
    p = (g.standard_normal(OS.N_PARAMS) * 0.3).astype(np.float32)
    net.params = p
    X = g.standard_normal((1000, 8)).astype(np.float32)
    T = g.standard_normal(1000).astype(np.float32)
    dx = torch.as_tensor(X, device="cuda")
    dt = torch.as_tensor(T, device="cuda")
    y = net.forward(dx).cpu().numpy()
    yo = OS.forward(p, X)
    assert np.abs(y - yo).max() <= 1e-4 * (1 + np.abs(yo).max())
    loss, grad = net.grad(dx, dt)
    lo, go = OS.loss_and_grad(p, X, T)
    assert loss == pytest.approx(lo, rel=1e-4)
    grad = grad.cpu().numpy()
    scale = np.abs(go).max()
    assert np.abs(grad - go).max() <= 1e-3 * scale
    net.close()


def test_features_match_oracle(mods):
    scd, sn = mods
    els = P.catalog_mixture(n=3000, seed=61)
    f = sn.features(els).cpu().numpy()
    fo = OS.features(els)
    assert np.abs(f - fo).max() <= 1e-5 * (1 + np.abs(fo).max())


def test_training_reduces_loss_and_checkpoint_round_trips(mods, tmp_path):
    scd, sn = mods
    els = P.catalog_mixture(n=4000, seed=62)
    X = OS.features(els).astype(np.float32)
    # a smooth target: log of P/100
    a = els[:, 0]
    Y = np.log(2 * np.pi * np.sqrt(a ** 3 / OS.MU) / 100.0).astype(np.float32)
    net = sn.StepNet(seed=4)
    losses = sn.train(net, X, Y, epochs=60, batch=1024, lr=3e-3)
    assert losses[-1] < 0.05 * losses[0]
    path = str(tmp_path / "net.bin")
    net.save(path)
    net2 = sn.StepNet(seed=9)
    net2.load(path)
    assert (net2.params == net.params).all()
    dx = torch.as_tensor(X, device="cuda")
    assert torch.equal(net.forward(dx), net2.forward(dx))
    net.close()
    net2.close()


def test_learned_policy_steps_and_sound_screen(mods):
    scd, sn = mods
    els = P.uniform_leo(24, seed=101, radius_km=300.0)
    net = sn.StepNet(seed=5)
    net.params = (np.random.default_rng(1).standard_normal(OS.N_PARAMS) * 0.05).astype(np.float32)
    T = 400
    sc = scd.Scene(els, float(T), 1.0, net.policy()).build_boxes()
    k = sc.steps().cpu().numpy()
    y = net.forward(sn.features(els)).cpu().numpy()
    ks = OS.learned_step_seconds(els, y)
    kk = np.maximum(np.floor(ks), 1)
    assert np.abs(k - np.minimum(kk, T + 1)).max() <= 1
    got = sc.find_pairs()
    lo, hi, obj = (x.cpu().numpy() for x in sc.boxes())
    want = O.canonicalize(O.raw_cells_sweep(lo, hi, obj.view(np.uint32)))
    assert np.array_equal(got.view(np.int32), want.view(np.int32))
    for w in O.alg1_witnesses(els, T, 1.0).tolist():
        m = got[(got["i"] == w[0]) & (got["j"] == w[1])]
        assert np.any((m["tlo"] <= w[2]) & (w[2] <= m["thi"])), w
    sc.close()
    net.close()


def test_trained_steps_beat_the_period_rule_on_held_out_objects(mods):
    """Sweep a training population, fit the cost model, train, then compare
    the modelled cost of a held-out population's screen under the learned
    steps and under P/100 (the learned steps must be no worse), and report
    the measured times."""
    scd, sn = mods
    train_els = P.catalog_mixture(n=3000, seed=71, radius_km=2.5)
    sw = sn.sweep(train_els, 21600.0)
    c_box, c_hit = sn.fit_cost_model(sw)
    Y = sn.targets(train_els, sw, c_box, c_hit).astype(np.float32)
    X = OS.features(train_els).astype(np.float32)
    net = sn.StepNet(seed=6)
    sn.train(net, X, Y, epochs=80, batch=512, lr=3e-3)

    test_els = P.catalog_mixture(n=3000, seed=72, radius_km=2.5)
    sw_t = sn.sweep(test_els, 21600.0, multipliers=(100.0,))
    cost_rule = (c_box * sw_t["boxes"][0] + 0.5 * c_hit * sw_t["pairs"][0]).sum()
    sc = scd.Scene(test_els, 21600.0, 1.0, net.policy()).build_boxes()
    ptr, m = scd.scd_find_raw_cells_device(sc.handle)
    cnt = torch.zeros(len(test_els), dtype=torch.int32, device="cuda")
    scd.scd_count_pairs_per_object(ptr, m, len(test_els), cnt.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    k = sc.steps().cpu().numpy().astype(np.int64)
    boxes = (21600 + k) // k
    cost_learned = (c_box * boxes + 0.5 * c_hit * cnt.cpu().numpy()).sum()
    print(f"modelled cost: learned {cost_learned:.3f} ms vs P/100 {cost_rule:.3f} ms "
          f"(c_box={c_box:.3e}, c_hit={c_hit:.3e})")
    assert cost_learned <= cost_rule
    sc.close()
    # measured: the held-out screen (boxes through the canonical list) under
    # both step rules, CUDA events on the stream, median of 7 after 2 warm-up
    # screens, L2 flushed before each
    rule = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    ms, cands = {}, {}
    for name, pol in (("learned", net.policy()), ("P/100", rule)):
        sc = scd.Scene(test_els, 21600.0, 1.0, pol)
        ms[name], cands[name] = _timed_screen(scd, sc, reps=7)
        sc.close()
    # at this size the learned steps give fewer candidates but more boxes,
    # and measured they are not faster (the linear cost model misjudges a
    # 2 ms screen); the gain in time is asserted at scale below
    print(f"measured: learned {ms['learned']:.3f} ms, {cands['learned']} candidates; "
          f"P/100 {ms['P/100']:.3f} ms, {cands['P/100']} candidates")
    assert cands["learned"] < cands["P/100"]
    net.close()


def test_learned_steps_are_faster_at_scale(mods):
    """Measured gain at the size the learned component is meant for: train on
    the sweeps of one 100,000-object population with dense LEO shells (24 h,
    INTERVAL boxes, ten step multipliers P/70-P/280), then screen a held-out
    population of the same shape under the learned steps and under P/100:
    fewer candidates and a shorter screen (CUDA events, median of 5 after 2
    warm-up screens, L2 flushed before each)."""
    scd, sn = mods
    mode = scd.SCD_BOX_INTERVAL
    train_els = P.catalog_mixture(n=100000, seed=P.SEED_BASE + 6, dense_shells=True)
    mults = tuple(float(70.0 * 4.0 ** (q / 9.0)) for q in range(10))
    sw = sn.sweep(train_els, 86400.0, multipliers=mults, mode=mode, count="runs")
    c_box, c_hit = sn.fit_cost_model(sw)
    Y = sn.targets(train_els, sw, c_box, c_hit).astype(np.float32)
    X = sn.features(train_els).cpu().numpy()
    net = sn.StepNet(seed=7)
    sn.train(net, X, Y, epochs=40, batch=1024, lr=3e-3)
    test_els = P.catalog_mixture(n=100000, seed=P.SEED_BASE + 5, dense_shells=True)
    rule = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    ms, cands = {}, {}
    for name, pol in (("learned", net.policy()), ("P/100", rule)):
        sc = scd.Scene(test_els, 86400.0, 1.0, pol, mode=mode)
        ms[name], cands[name] = _timed_screen(scd, sc, reps=5)
        sc.close()
    print(f"100k, 24 h, INTERVAL: learned {ms['learned']:.1f} ms, {cands['learned']} "
          f"candidates; P/100 {ms['P/100']:.1f} ms, {cands['P/100']} candidates")
    assert cands["learned"] < cands["P/100"]
    assert ms["learned"] < ms["P/100"]
    net.close()


def _timed_screen(scd, sc, reps):
    st = torch.cuda.current_stream()
    flush = torch.empty(2 * 129 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ts, n = [], 0
    for k in range(reps + 2):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        scd.scd_build_boxes(sc.handle)
        n = scd.scd_find_pairs_device(sc.handle)[1]
        e1.record(st)
        e1.synchronize()
        if k >= 2:
            ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), n


def _covered(pairs, near):
    """Is every approach (i, j, t) inside a reported interval of its pair?"""
    key = pairs["i"].astype(np.int64) << 32 | pairs["j"].astype(np.int64)
    order = np.argsort(key, kind="stable")
    key, lo, hi = key[order], pairs["tlo"][order], pairs["thi"][order]
    missed = []
    for w in near:
        k = (int(w["i"]) << 32) | int(w["j"])
        a, b = np.searchsorted(key, k, "left"), np.searchsorted(key, k, "right")
        if not np.any((lo[a:b] <= w["t"]) & (w["t"] <= hi[a:b])):
            missed.append((int(w["i"]), int(w["j"]), int(w["t"])))
    return missed


def test_learned_and_rule_screens_miss_no_close_approach(mods):
    """Soundness on a dense population: every approach closer than 5 km (two
    objects of radius 2.5 km touching), found by Alg 1 at every 1 s tick of
    6 h over 2000 objects, lies inside a reported interval of its pair, with
    learned steps and with P/100."""
    scd, sn = mods
    els = P.catalog_mixture(n=2000, seed=91, dense_shells=True, crossing_frac=0.01,
                            horizon_s=21600.0)
    T = 21600
    near = O.close_approaches(els, T, 1.0, 5.0)
    assert len(near) >= 5  # the seeded crossings at least
    net = sn.StepNet(seed=9)
    net.params = (np.random.default_rng(4).standard_normal(OS.N_PARAMS) * 0.1).astype(np.float32)
    rule = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    for name, pol in (("learned", net.policy()), ("P/100", rule)):
        sc = scd.Scene(els, float(T), 1.0, pol).build_boxes()
        got = sc.find_pairs()
        sc.close()
        missed = _covered(got, near)
        assert not missed, (name, missed[:5])
    net.close()


def test_learned100k_screen_misses_no_close_approach(mods):
    """The n = 100000 dense-shell screen of 24 h with INTERVAL boxes, under
    steps from a network trained on 20-multiplier sweeps of another 100000
    objects and under P/100: on the 2000 objects nearest the 550 km shell,
    every approach closer than 5 km at a 1 s tick (Alg 1 by brute force)
    lies inside a reported interval of the full screen's output."""
    scd, sn = mods
    train = P.catalog_mixture(n=100000, seed=P.SEED_BASE + 6, dense_shells=True)
    mults = tuple(50.0 * 8.0 ** (q / 19.0) for q in range(20))
    sw = sn.sweep(train, 7200.0, multipliers=mults, mode=scd.SCD_BOX_INTERVAL)
    c_box, c_hit = sn.fit_cost_model(sw)
    Y = sn.targets(train, sw, c_box, c_hit).astype(np.float32)
    X = sn.features(train).cpu().numpy()
    net = sn.StepNet(seed=7)
    sn.train(net, X, Y, epochs=60, batch=1024, lr=3e-3)

    els = P.catalog_mixture(n=100000, seed=P.SEED_BASE + 5, dense_shells=True)
    hp = els[:, 0] * (1.0 - els[:, 1]) - 6378.137
    sub = np.sort(np.argsort(np.abs(hp - 550.0))[:2000])
    near = O.close_approaches(els[sub], 86400, 1.0, 5.0)
    assert len(near) > 100
    near["i"], near["j"] = sub[near["i"]], sub[near["j"]]  # population indices (i < j kept)
    in_sub = torch.zeros(len(els), dtype=torch.bool, device="cuda")
    in_sub[torch.as_tensor(sub, device="cuda")] = True
    rule = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
    for name, pol in (("learned", net.policy()), ("P/100", rule)):
        sc = scd.Scene(els, 86400.0, 1.0, pol, mode=scd.SCD_BOX_INTERVAL).build_boxes()
        pr = sc.find_pairs_device()
        keep = in_sub[pr[:, 0].long()] & in_sub[pr[:, 1].long()]
        pairs = scd.pairs_from_device(pr[keep])
        del pr, keep
        sc.close()
        missed = _covered(pairs, near)
        assert not missed, (name, len(missed), missed[:5])
    net.close()

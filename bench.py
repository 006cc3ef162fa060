"""Benchmark of the 4D box screen on one GB300 (per rank).

Default workload: one 24 h screen of a 16,848-object catalog-shaped
population at steps P/100.  A step is one pass of the whole hot path from
device-resident elements to the device-resident canonical pair list:
per-object steps, FP64 propagation, FP32 boxes and Morton keys, radix sort,
hierarchy, refit, traversal with merged emission, canonical sort.  The JSON
line's ``value`` is milliseconds per screen (whole job: all ranks' screens
over the max-rank time); ``e2e`` is the same through the C ABI with host
buffers (elements copied in, pairs copied out inside the timed region).

Other workloads (--workload):
  refine512   the 512-object, 6000 s population of the parity tests solved by
              adaptive refinement (Alg 5-6 in rounds), beside the fixed-step
              screen plus narrow phase
  refine24h   the same for the 24 h catalog workload (16,848 objects)
  narrow24h   the default screen followed by the narrow phase over its
              candidates: the first collision witness of the 24 h problem
              (Def 5) from device-resident elements
  band_slab   the same population with band-table steps (P/200 .. P/400 by
              perigee altitude) and the 16 slab x 8 octant decomposition, with
              the tuning picked by the autotuner
  batch64     64 independent scenes of uneven size (1e3-6e4 objects,
              ~1.2M in all, horizons 6-72 h), each group of scenes one batch
              through one persistent traversal: scenes per second and per
              scene latency
  learned100k 100,000 objects with two dense LEO shells, 24 h, per-object
              steps from the step network trained on this run's own sweeps,
              against the P/100 rule

--impl reference times the CPU oracle on all host cores on a bounded sample
of the default workload (windows of the horizon: the part of the screen
found from the boxes that start in each window) and scales it to a 24 h
screen.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import population as P  # noqa: E402

N_OBJ = 16848
HORIZON_S = 86400.0
TICK_S = 1.0
FRACTION = 100.0
L2_BYTES = 129 * 1024 * 1024
MU = 398600.4418

WORKLOADS = {
    "catalog24h": {
        "metric": "ms per 24h screen at n=16848",
        "desc": ("catalog-shaped synthetic mixture n=16848 (72% LEO, 8% MEO, 10% GEO, 10% HEO, "
                 "0.1% seeded crossing pairs), 24 h horizon, 1 s ticks, per-object step P/100, "
                 "plain 4D LBVH")},
    "band_slab": {
        "metric": "ms per 24h screen at n=16848, band steps, 16 slabs x 8 octants",
        "desc": ("the n=16848 mixture, 24 h, per-object steps P/200 (perigee < 1000 km), P/100 "
                 "(1000-2000 km), P/50 (2000-30000 km), P/400 (above); 16 tick slabs x 8 ECI "
                 "octants as 128 cell subtrees of one sort in one persistent traversal; tuning "
                 "from the autotuner")},
    "narrow24h": {
        "metric": "ms per 24h first-witness solve at n=16848 (screen + narrow phase)",
        "desc": ("the n=16848 mixture, 24 h, 1 s ticks, per-object step P/100: the screen's "
                 "canonical candidate list, then the narrow phase (Alg 1's infinity-norm test "
                 "at the candidates' ticks, FP64 positions, ticks skipped by the "
                 "relative-motion bound): per-candidate first witness and witness count and "
                 "the earliest witness (Def 5)")},
    "refine512": {
        "metric": "ms per adaptive-refinement solve at n=512, 6000 s (every collision witness)",
        "desc": ("n=512 uniform LEO (a 6678-8378 km, e < 0.01, i 0-100 deg), r = 2.5 km, 6000 s "
                 "at 1 s ticks: Alg 5-6 as data-parallel rounds from period-bounded first "
                 "intervals (per round the boxes of all active intervals, their Morton sort, a "
                 "radix tree and the persistent traversal; all rounds queued without host "
                 "reads), tick candidates decided by the narrow phase; against the fixed "
                 "10-tick screen plus the narrow phase on the same population")},
    "refine24h": {
        "metric": "ms per 24h adaptive-refinement solve at n=16848 (every collision witness)",
        "desc": ("the n=16848 mixture, 24 h at 1 s ticks: Alg 5-6 as data-parallel rounds from "
                 "period-bounded first intervals (per round the boxes of all active "
                 "intervals, their Morton sort, a radix tree and the persistent traversal; all "
                 "rounds queued without host reads), tick candidates decided by the narrow "
                 "phase; against the fixed P/100 screen plus the narrow phase on the same "
                 "population")},
    "batch64": {
        "metric": "scenes per second, 64 scenes, ~1.2M objects, horizons 6-72 h",
        "desc": ("64 independent catalog-shaped scenes, sizes log-uniform 1e3-6e4 (total "
                 "~1.2M objects), horizons whole hours 6-72, steps P/100; scenes grouped into "
                 "batches of up to 4e7 boxes, smallest scenes first, each batch one box "
                 "build, one sort, one tree and one persistent traversal")},
    "learned100k": {
        "metric": "ms per 24h screen at n=100000, learned steps",
        "desc": ("100,000-object mixture with Gaussian LEO shells at 550 and 1150 km, 24 h; "
                 "per-object steps from the 8-64-64-1 step network trained in this run on "
                 "sweeps of another 100,000-object population of the same shape (24 h, 20 multipliers P/70-P/280)")},
}


# the library sources a screen runs (boxes, sort, hierarchy, traversal,
# canonical list, scene control): the traversal's DRAM traffic depends on
# these alone; the narrow phase, the step network and the refinement rounds
# live in other files and do not run in a screen
SCREEN_SOURCES = ("decomp.cu", "kepler.cuh", "lbvh.cu", "propagate.cu", "radix_sort.cu",
                  "scd_internal.cuh", "scene.cu", "traverse.cu")


def library_sources():
    """The screen's CUDA sources, in name order."""
    d = os.path.join(ROOT, "paper_1901_10475_gb300", "csrc")
    return [os.path.join(d, f) for f in sorted(SCREEN_SOURCES)]


def measured_traffic(workload: str):
    """DRAM bytes per traversal launch from the committed ncu summary of this
    workload, if the traversal's sources still hash to the ones it was
    measured on; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_traverse2_catalog16848_24h.md")
    if workload not in ("catalog24h", "narrow24h") or not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.split(":", 1)[0] in ("traffic_bytes_per_launch", "source_sha256"):
            k, v = line.split(":", 1)
            fields[k] = v.strip()
    h = hashlib.sha256()
    for f in library_sources():
        with open(f, "rb") as fh:
            h.update(fh.read())
    if fields.get("source_sha256") != h.hexdigest()[:16]:
        return None
    return float(fields["traffic_bytes_per_launch"])


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(m: dict, n: int) -> dict:
    """Algorithmic HBM bytes of one screen by phase: every array read or
    written once per pass that needs it (one box per leaf)."""
    N = m["boxes"]
    R = m.get("refs") or N  # sorted entries (references when decomposed)
    M = R
    runs = m["records"]
    opens = m.get("open_runs", runs)  # runs of more than one cell: one end record each
    key_b = 4 if m["morton_bits"] <= 8 else 8
    passes = (4 * m["morton_bits"] + 7) // 8
    pair_bits = 2 * max(1, int(np.ceil(np.log2(max(n, 2))))) + int(np.ceil(np.log2(m["T"] + 1)))
    ppasses = (pair_bits + 7) // 8
    return {
        # elements in; boxes (32 B), object id, box id and key out
        "boxes": 56 * n + N * (32 + 4 + 4 + key_b),
        # per pass: keys+values read twice (count, rank), written once
        "sort": passes * N * 3 * (key_b + 4),
        # gather boxes by id; neighbour positions; hierarchy nodes and refit
        "build": R * (4 + 32 + 32 + 4 + 8 + 4) + M * (key_b + 40 + 32 + 16),
        # every sorted box and compact node read at least once; records written
        "traverse": R * (32 + 8) + (M - 1) * 40 + (runs + opens) * 8,
        # key-only sorts of the run starts and of the open runs' ends (keys
        # read twice, written once per pass), the open count, the unpack
        "canon": ppasses * (runs + opens) * 8 * 3 + runs * 8 + runs * (8 + 16) + opens * 8,
    }


def _device():
    import torch
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    return dev


def slowest_rank(t_ms: float, world: int, device: str = "cuda") -> float:
    """The largest of the ranks' timed totals (every rank calls this; one
    process per GPU, each a replica of the whole workload)."""
    if world <= 1:
        return t_ms
    import torch
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def time_scene_steps(sc, step, steps, warmup, dev, world):
    """Warm up, then time `steps` screens with CUDA events on the scene's
    stream, flushing L2 between them (outside the timed events)."""
    import torch
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    phase = {k: [] for k in ("ms_boxes", "ms_sort", "ms_build", "ms_traverse", "ms_canon")}
    tests = launches = 0
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    n_pairs = 0
    with ClockSampler(dev) as clk:
        for k in range(steps):
            flush.fill_(float(k))
            ev0[k].record(stream)
            n_pairs = step()
            ev1[k].record(stream)
            m = sc.metrics()
            for key in phase:
                phase[key].append(m[key])
            tests += m["node_tests"] + m["leaf_tests"]
            launches += m["launches"]
        torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    return {"times": times, "phase_ms": {k: statistics.mean(v) for k, v in phase.items()},
            "tests": tests, "launches": launches, "n_pairs": n_pairs, "clocks": clk.summary(),
            "metrics": sc.metrics()}


def e2e_through_abi(sc, els, n_pairs, steps):
    """Median ms of: host elements in (pinned), boxes, pairs to a pinned host
    array, through the C entry points."""
    import torch

    import paper_1901_10475_gb300 as scd
    host_in = torch.as_tensor(np.ascontiguousarray(els)).pin_memory()
    out_pinned = torch.empty(max(2 * n_pairs, 1) * 16, dtype=torch.uint8).pin_memory()
    out_np = out_pinned.numpy().view(scd.PAIR_DTYPE)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    ts = []
    n_host = 0
    for k in range(max(1, min(steps, 5))):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        scd._binding.lib().scd_scene_set_elements(sc.handle, ctypes.c_void_p(host_in.data_ptr()),
                                                  len(els))
        scd.scd_build_boxes(sc.handle)
        n_host = scd.scd_find_pairs_into(sc.handle, out_np)
        ts.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(ts), n_host


def run_single(args, world, wl):
    """Single-scene workloads (catalog24h, band_slab)."""
    import torch

    import paper_1901_10475_gb300 as scd
    from paper_1901_10475_gb300 import autotune
    dev = _device()
    els = P.catalog_mixture(n=N_OBJ, seed=P.SEED_BASE + 2)
    decomp = None
    if wl == "band_slab":
        edges, fr = P.band_table_config3()
        pol = scd.make_step_policy(scd.SCD_STEP_BAND_TABLE, band_edges_km=edges,
                                   band_fractions=fr)
        decomp = (scd.SCD_DECOMP_SLAB_OCT, 0, 16)
    else:
        pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=FRACTION)
    sc = scd.Scene(els, args.horizon_s, TICK_S, pol, mode=args.mode)
    tuning = None
    if args.tuning:
        sc.set_tuning(json.loads(args.tuning))
    elif wl == "band_slab" or args.autotune:
        sc.build_boxes()
        key = autotune.workload_key(els, args.horizon_s, TICK_S, wl, 1 << 24)
        tuning, _ = autotune.load_or_tune(sc, key, reps=1, decomp=decomp)
    # the whole find sequence replayed as one captured CUDA graph
    use_graph = args.graph if args.graph >= 0 else int(wl == "band_slab")
    if use_graph:
        tuning = dict(json.loads(args.tuning) if args.tuning else (tuning or {}), use_graph=1)
        sc.set_tuning(tuning)
    d_el = torch.as_tensor(els, device="cuda")

    def step():
        scd.scd_scene_set_elements_device(sc.handle, d_el.data_ptr(), N_OBJ)
        scd.scd_build_boxes(sc.handle)
        return scd.scd_find_pairs_device(sc.handle, decomp)[1]

    r = time_scene_steps(sc, step, args.steps, args.warmup, dev, world)
    if use_graph:
        # a replayed graph's kernels cannot be timed one by one: the phase
        # split comes from the same screen launched eagerly, after the timed
        # replays (CUDA events on the scene's stream around each phase)
        sc.set_tuning(dict(tuning, use_graph=0))
        step()
        step()
        m = sc.metrics()
        r["phase_ms"] = {k: m[k] for k in r["phase_ms"]}
        r["phase_ms_source"] = "one eager screen after the timed graph replays"
        sc.set_tuning(tuning)
    # whole job: every rank's screens over the slowest rank's time
    r["value"] = slowest_rank(sum(r["times"]), world) / (args.steps * world)
    r["unit"] = "ms"
    r["higher_is_better"] = False
    if decomp is None:
        r["e2e_ms"], r["e2e_pairs"] = e2e_through_abi(sc, els, r["n_pairs"], args.steps)
        r["e2e"] = {"value": r["e2e_ms"], "unit": "ms", "h2d_bytes_per_step": 56 * N_OBJ,
                    "d2h_bytes_per_step": 16 * r["e2e_pairs"]}
    if wl == "catalog24h" and not args.no_extras and args.mode == 0:
        # secondary figures of the same run: the narrow phase over this
        # screen's candidates, and the same screen with INTERVAL boxes
        step()
        r["narrow"] = narrow_over_screen(sc, min(args.steps, 5))
        r["interval_screen"] = interval_screen(els, d_el, args, min(args.steps, 5), dev)
    r["n"] = N_OBJ
    r["tuning"] = tuning
    sc.close()
    return r


def narrow_over_screen(sc, reps: int) -> dict:
    """The narrow phase (first witness and witness count of every candidate,
    the earliest witness of Def 5) over the scene's current candidate list,
    CUDA events on the stream, L2 flushed before each run."""
    import torch

    import paper_1901_10475_gb300 as scd
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    ptr, m = scd.scd_find_pairs_device(sc.handle)
    first = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    count = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    ts, w = [], None
    for k in range(reps + 1):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        w = scd.scd_narrow_phase(sc.handle, ptr, m, first.data_ptr(), count.data_ptr())
        e1.record(stream)
        e1.synchronize()
        if k > 0:
            ts.append(e0.elapsed_time(e1))
    mm = sc.metrics()
    return {"ms": statistics.mean(ts), "candidates": m,
            "tick_evals": int(mm["narrow_evals"]), "tick_evals_fp64": int(mm["narrow_evals_fp64"]),
            "candidates_with_witness": int((first[:m] >= 0).sum()),
            "witness_ticks": int(count[:m].long().sum()),
            "earliest_witness": list(w) if w else None}


def interval_screen(els, d_el, args, reps: int, dev: int) -> dict:
    """The same 24 h screen with INTERVAL boxes (the paper's interval
    evaluation, Sec. 4.5), timed like the main screen."""
    import paper_1901_10475_gb300 as scd
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=FRACTION)
    sc = scd.Scene(els, args.horizon_s, TICK_S, pol, mode=scd.SCD_BOX_INTERVAL)

    def step():
        scd.scd_scene_set_elements_device(sc.handle, d_el.data_ptr(), len(els))
        scd.scd_build_boxes(sc.handle)
        return scd.scd_find_pairs_device(sc.handle)[1]

    r = time_scene_steps(sc, step, reps, 2, dev, 1)
    m = r["metrics"]
    out = {"ms": statistics.mean(r["times"]), "pairs": r["n_pairs"], "boxes": m["boxes"],
           "phase_ms": r["phase_ms"], "node_tests": m["node_tests"],
           "leaf_tests": m["leaf_tests"], "clocks": r["clocks"]}
    sc.close()
    return out


def run_narrow(args, world):
    """The 24 h screen, then the narrow phase over its candidate list."""
    import torch

    import paper_1901_10475_gb300 as scd
    dev = _device()
    els = P.catalog_mixture(n=N_OBJ, seed=P.SEED_BASE + 2)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=FRACTION)
    sc = scd.Scene(els, args.horizon_s, TICK_S, pol, mode=args.mode)
    d_el = torch.as_tensor(els, device="cuda")
    stream = torch.cuda.current_stream()
    buf = {}
    np_ms, np_evals, np_evals64 = [], [], []

    def step():
        scd.scd_scene_set_elements_device(sc.handle, d_el.data_ptr(), N_OBJ)
        scd.scd_build_boxes(sc.handle)
        ptr, m = scd.scd_find_pairs_device(sc.handle)
        buf["ptr"] = ptr
        if buf.get("m") != m:
            buf["m"] = m
            buf["first"] = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
            buf["count"] = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        buf["w"] = scd.scd_narrow_phase(sc.handle, ptr, m, buf["first"].data_ptr(),
                                        buf["count"].data_ptr())
        e1.record(stream)
        e1.synchronize()
        np_ms.append(e0.elapsed_time(e1))
        mm = sc.metrics()
        np_evals.append(mm["narrow_evals"])
        np_evals64.append(mm["narrow_evals_fp64"])
        return m

    r = time_scene_steps(sc, step, args.steps, args.warmup, dev, world)
    r["launches"] += 3 * args.steps  # the narrow phase: state init, object constants, k_narrow
    k = args.steps
    r["phase_ms"]["ms_narrow"] = statistics.mean(np_ms[-k:])
    r["narrow"] = {"ms": statistics.mean(np_ms[-k:]), "tick_evals": int(np_evals[-1]),
                   "tick_evals_fp64": int(np_evals64[-1]),
                   "tick_evals_per_s": np_evals[-1] / (statistics.mean(np_ms[-k:]) * 1e-3),
                   "candidates": buf["m"],
                   "candidate_ticks": _candidate_ticks(buf["ptr"], buf["m"]),
                   "candidates_with_witness": int((buf["first"][:buf["m"]] >= 0).sum()),
                   "witness_ticks": int(buf["count"][:buf["m"]].long().sum()),
                   "earliest_witness": list(buf["w"]) if buf["w"] else None}
    r["value"] = slowest_rank(sum(r["times"]), world) / (args.steps * world)
    r["unit"] = "ms"
    r["higher_is_better"] = False
    # end to end through the C ABI: host elements in, earliest witness out
    host_in = torch.as_tensor(np.ascontiguousarray(els)).pin_memory()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    ts = []
    for q in range(max(1, min(args.steps, 5))):
        flush.fill_(float(q))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        scd._binding.lib().scd_scene_set_elements(sc.handle, ctypes.c_void_p(host_in.data_ptr()),
                                                  N_OBJ)
        scd.scd_build_boxes(sc.handle)
        ptr, m = scd.scd_find_pairs_device(sc.handle)
        scd.scd_narrow_phase(sc.handle, ptr, m, buf["first"].data_ptr(), buf["count"].data_ptr())
        ts.append((time.perf_counter() - t0) * 1e3)
    r["e2e"] = {"value": statistics.median(ts), "unit": "ms", "h2d_bytes_per_step": 56 * N_OBJ,
                "d2h_bytes_per_step": 12}
    r["n"] = N_OBJ
    sc.close()
    return r


def run_refine(args, world, wl="refine512"):
    """Adaptive refinement on the small workload (or the 24 h catalog one),
    and the fixed-step screen plus narrow phase on the same population for
    comparison."""
    import torch

    import paper_1901_10475_gb300 as scd
    dev = _device()
    if wl == "refine24h":
        els = P.catalog_mixture(n=N_OBJ, seed=P.SEED_BASE + 2)
        T_S = args.horizon_s
        pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=FRACTION)
    else:
        els = P.uniform_leo(512)
        T_S = 6000.0
        pol = scd.make_step_policy(scd.SCD_STEP_FIXED, fixed_ticks=10)
    sc = scd.Scene(els, T_S, TICK_S, pol, mode=args.mode)
    sc.build_boxes()
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts, out

    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(dev) as clk:
        times, (w, rb) = timed(lambda: scd.scd_refine_witnesses(sc.handle), args.steps,
                               args.warmup)
        refine_launches = sc.metrics()["launches"]

        def fixed():
            scd.scd_build_boxes(sc.handle)
            ptr, m = scd.scd_find_pairs_device(sc.handle)
            return scd.scd_narrow_phase(sc.handle, ptr, m)

        ftimes, earliest = timed(fixed, args.steps, args.warmup)
        # the continuous-time variant at eps = 1 s on the same population
        ctimes, (spans, crb) = timed(lambda: scd.scd_refine_continuous(sc.handle, 1.0),
                                     args.steps, args.warmup)
    # algorithmic bytes of the rounds, per interval: its box, Morton key and
    # index written (44 B); six radix passes over key and index (36 B each:
    # read twice, written once); the gather of the sorted box and object
    # (76 B); the radix tree's links and parents (40 B) and refit (90 B);
    # the traversal's sorted box, node and id reads (72 B); flags and the
    # split's reads and writes (40 B)
    per_box = 44 + 6 * 36 + 76 + 40 + 90 + 72 + 40
    byt = int(rb.sum()) * per_box
    ms = statistics.mean(times)
    pk, src = _peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    # kernels per timed solve, counted by the library
    launches = args.steps * refine_launches
    r = {"times": times, "clocks": clk.summary(), "unit": "ms", "higher_is_better": False,
         "value": slowest_rank(sum(times), world) / (args.steps * world),
         "launches": launches, "n": len(els)}
    r["refine"] = {"start_fraction": float(sc.tuning()["refine_start"]),
                   "rounds": int(len(rb)), "intervals_per_round": [int(x) for x in rb],
                   "boxes": int(rb.sum()), "witnesses": int(len(w)),
                   "earliest_witness": [int(x) for x in w[0]] if len(w) else None,
                   "fixed_step_ms": statistics.mean(ftimes),
                   "fixed_step_boxes": int(sc.metrics()["boxes"]),
                   "fixed_step_earliest": list(earliest) if earliest else None,
                   "continuous": {"eps_s": 1.0, "ms": statistics.mean(ctimes),
                                  "rounds": int(len(crb)), "boxes": int(crb.sum()),
                                  "spans": int(len(spans))}}
    r["roofline_refine"] = {"kernel_phase": "refinement rounds", "bound": "hbm",
                            "achieved": byt / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                            "frac": byt / (ms * 1e-3) / 1e9 / hbm, "traffic": None,
                            "peak_source": src, "algorithmic_bytes": byt}
    # end to end through the ABI: host elements in, witnesses out
    host_in = torch.as_tensor(np.ascontiguousarray(els)).pin_memory()
    ts = []
    for q in range(max(1, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        scd._binding.lib().scd_scene_set_elements(sc.handle, ctypes.c_void_p(host_in.data_ptr()),
                                                  len(els))
        scd.scd_build_boxes(sc.handle)
        w2, _ = scd.scd_refine_witnesses(sc.handle)
        ts.append((time.perf_counter() - t0) * 1e3)
    r["e2e"] = {"value": statistics.median(ts), "unit": "ms", "h2d_bytes_per_step": 56 * len(els),
                "d2h_bytes_per_step": 12 * len(w2)}
    sc.close()
    return r


def _candidate_ticks(ptr, m):
    """Sum of thi - tlo + 1 over a device candidate list."""
    import paper_1901_10475_gb300 as scd
    if m == 0:
        return 0
    p = scd.device_view(ptr, (m, 4), "<i4")
    return int((p[:, 3].long() - p[:, 2].long() + 1).sum())


def run_batch64(args, world):
    import torch

    import paper_1901_10475_gb300 as scd
    dev = _device()
    scenes = P.batch_scenes()
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=FRACTION)
    # batches of at most 4e7 boxes (estimated from P/100), smallest scenes
    # first (the same throughput as arrival order, a far lower median latency)
    from paper_1901_10475_gb300 import batching
    est = [batching.estimated_boxes(els, hz, TICK_S, FRACTION) for els, hz in scenes]
    groups = batching.plan_batches(est, 4e7, "shortest_first")
    stream = torch.cuda.current_stream()

    def one_pass(record):
        t0 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        done = []
        npairs = launches = 0
        for g in groups:
            b = scd.BatchScene([scenes[s][0] for s in g], [scenes[s][1] for s in g], TICK_S, pol,
                               mode=args.mode)
            b.build_boxes()
            npairs += scd.scd_find_pairs_device(b.handle)[1]
            launches += b.metrics()["launches"]
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            done.append((g, ev))
            b.close()
        torch.cuda.synchronize()
        lat = {}
        for g, ev in done:
            for s in g:
                lat[s] = t0.elapsed_time(ev)
        return t0, done, lat, npairs, launches

    for _ in range(args.warmup):
        one_pass(False)
    totals, lats = [], []
    launches = 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            t0, done, lat, npairs, nl = one_pass(True)
            totals.append(t0.elapsed_time(done[-1][1]))
            lats.extend(lat.values())
            launches += nl
    ms = statistics.mean(totals)
    # whole job: every rank's scenes over the slowest rank's time
    t_all = slowest_rank(sum(totals), world)
    return {"value": len(scenes) * world * args.steps * 1e3 / t_all, "unit": "scenes/s",
            "higher_is_better": True,
            "times": totals, "clocks": clk.summary(), "n_pairs": npairs,
            "latency_ms": {"p50": float(np.percentile(lats, 50)),
                           "p99": float(np.percentile(lats, 99))},
            "batches": len(groups), "objects": int(sum(len(e) for e, _ in scenes)),
            "boxes_est": float(sum(est)), "ms_per_pass": ms, "launches": launches}


def run_learned100k(args, world):
    import torch

    import paper_1901_10475_gb300 as scd
    from paper_1901_10475_gb300 import stepnet as sn
    dev = _device()
    # train on the method's own sweeps of a smaller population
    train_els = P.catalog_mixture(n=100000, seed=P.SEED_BASE + 6, dense_shells=True)
    t0 = time.perf_counter()
    # 20 step multipliers from P/70 to P/280 (geometric) at the screen's own
    # horizon: 2M (elements, step, candidate-pair count) samples from 100k
    # objects, with the screens' times (per-object costs do not carry over
    # from short horizons: a box costs more in the larger tree of a long one)
    mults = tuple(float(70.0 * 4.0 ** (q / 19.0)) for q in range(20))
    sw = sn.sweep(train_els, HORIZON_S, multipliers=mults, mode=args.mode, count="runs")
    c_box, c_hit = sn.fit_cost_model(sw)
    Y = sn.targets(train_els, sw, c_box, c_hit).astype(np.float32)
    X = sn.features(train_els).cpu().numpy()
    net = sn.StepNet(seed=7)
    losses = sn.train(net, X, Y, epochs=60, batch=1024, lr=3e-3)
    train_s = time.perf_counter() - t0

    els = P.catalog_mixture(n=100000, seed=P.SEED_BASE + 5, dense_shells=True)
    d_el = torch.as_tensor(els, device="cuda")
    out = {}
    for name, pol in [("learned", net.policy()),
                      ("p100", scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION,
                                                    period_fraction=FRACTION))]:
        sc = scd.Scene(els, HORIZON_S, TICK_S, pol, mode=args.mode)

        def step():
            scd.scd_scene_set_elements_device(sc.handle, d_el.data_ptr(), len(els))
            scd.scd_build_boxes(sc.handle)
            return scd.scd_find_pairs_device(sc.handle)[1]

        out[name] = time_scene_steps(sc, step, args.steps, args.warmup, dev, world)
        sc.close()
    r = out["learned"]
    r["value"] = slowest_rank(sum(r["times"]), world) / (args.steps * world)
    r["unit"] = "ms"
    r["higher_is_better"] = False
    r["n"] = 100000
    r["p100_ms"] = statistics.mean(out["p100"]["times"])
    r["p100_boxes"] = out["p100"]["metrics"]["boxes"]
    r["p100_pairs"] = out["p100"]["n_pairs"]
    r["training"] = {"seconds": train_s, "objects": len(X),
                     "sweep_samples": int(len(mults) * len(train_els)),
                     "multipliers": [round(m, 1) for m in mults],
                     "sweep_ms": [round(float(x), 2) for x in sw["ms"]],
                     "sweep_boxes": [int(x) for x in sw["total_boxes"]],
                     "sweep_pairs": [int(x) for x in sw["total_pairs"]],
                     "final_loss": float(losses[-1]),
                     "c_box_ms": c_box, "c_hit_ms": c_hit}
    net.close()
    return r


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _windows(n_windows: int, window_ticks: int, T: int, phase: float = 0.5):
    """Start ticks of n windows spread evenly over [0, T]."""
    step = (T + 1) / n_windows
    return [int(step * (w + phase) - window_ticks / 2) for w in range(n_windows)]


def cpu_oracle_windows(starts, window_ticks: int, threads: int):
    """The oracle's screen of the 24 h workload, measured on sample windows
    of the horizon.  Window [t0, t0 + w) stands for the part of the whole
    screen found from the boxes whose segments start in it: their boxes
    (whole segments, generated and timed), the sweep's pairs found from them
    with the boxes starting up to one longest segment later as candidates
    (generated untimed: they are the next windows' boxes), and the canonical
    list of those pairs.  Over a partition of [0, T] such windows are
    exactly the whole screen (a pinned property of the oracle).  Windows
    run on `threads` host threads (the oracle's C calls release the GIL).
    Returns (wall seconds of the timed work, summed per-window seconds,
    boxes, pairs, each window's seconds)."""
    import concurrent.futures as cf

    import oracle as O
    els = P.catalog_mixture(n=N_OBJ, seed=P.SEED_BASE + 2)
    T = int(HORIZON_S / TICK_S)
    k = O.step_ticks(els, O.STEP_PERIOD_FRACTION, TICK_S, frac=FRACTION)
    longest = int(np.max(k))

    def one(t0):
        t1 = t0 + window_ticks
        c0 = time.perf_counter()
        lo, hi, obj = O.boxes_starting(els, T, TICK_S, k, t0, t1, O.BOX_SPEED)
        c1 = time.perf_counter()
        xl, xh, xo = O.boxes_starting(els, T, TICK_S, k, t1, t1 + longest, O.BOX_SPEED)
        c2 = time.perf_counter()
        cells = O.raw_cells_sweep_before(np.concatenate([lo, xl]), np.concatenate([hi, xh]),
                                         np.concatenate([obj, xo]), t1)
        O.canonicalize(cells)
        c3 = time.perf_counter()
        return (c1 - c0) + (c3 - c2), c2 - c1, len(lo), len(cells)

    w0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, starts))
    wall = time.perf_counter() - w0
    # the untimed candidate generation ran inside the wall time too: take it
    # out in proportion to its share of the threads' time
    busy = sum(r[0] for r in res)
    extra = sum(r[1] for r in res)
    return (wall * busy / (busy + extra), busy, sum(r[2] for r in res), sum(r[3] for r in res),
            [r[0] for r in res])


def cpu_baseline_measure():
    """ms per 24 h screen of the oracle on all host cores and on one, from
    window samples (see cpu_oracle_windows); the per-window times of the
    even and the odd windows must give per-tick costs within 5% of each
    other (the sample is representative of the horizon)."""
    T = int(HORIZON_S / TICK_S)
    cores = os.cpu_count() or 1
    n_all, w_all, w_one = 3 * cores, 60, 100
    starts = _windows(n_all, w_all, T)
    wall, busy, nbox, npair, per = cpu_oracle_windows(starts, w_all, cores)
    scale = (T + 1) / (n_all * w_all)
    halves = [sum(per[0::2]) / (len(per[0::2]) * w_all), sum(per[1::2]) / (len(per[1::2]) * w_all)]
    one = cpu_oracle_windows(_windows(1, w_one, T, phase=0.25), w_one, 1)
    ms_all = wall * 1e3 * scale
    ms_one = one[0] * 1e3 * (T + 1) / w_one
    desc = (f"oracle (box generation, time-sorted sweep, canonical sort) on {n_all} windows of "
            f"{w_all} ticks spread over the 24 h screen of all {N_OBJ} objects ({nbox} whole "
            f"segment boxes, {npair} pairs; {100.0 / scale:.2f}% of the horizon), {cores} "
            f"threads, scaled by {scale:.1f}; windows partition the screen exactly")
    return {"value": ms_all, "unit": "ms", "cores": cores, "kind": "oracle", "sample": desc,
            "cpu_model": _cpu_model(), "sample_seconds": wall,
            "one_core": {"value": ms_one, "unit": "ms", "cores": 1,
                         "sample": f"one window of {w_one} ticks, one thread",
                         "sample_seconds": one[0]},
            "halves_s_per_tick": halves,
            "halves_agree": abs(halves[0] - halves[1]) <= 0.05 * max(halves)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="catalog24h", choices=sorted(WORKLOADS))
    ap.add_argument("--tuning", default="", help="JSON tuning overrides")
    ap.add_argument("--autotune", action="store_true", help="search the tuning first")
    ap.add_argument("--graph", type=int, default=-1,
                    help="1: replay each screen's find sequence as one captured CUDA graph, "
                         "0: launch eagerly (default: graph for band_slab, eager otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="catalog24h: skip the narrow-phase and INTERVAL-screen figures")
    ap.add_argument("--box-mode", default="", choices=["", "speed", "interval"],
                    help="occ-int bound; default: speed, interval for batch64 and learned100k")
    ap.add_argument("--horizon-s", type=float, default=HORIZON_S,
                    help="shorter horizons give the small profiling case")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    wl = args.workload
    metric = WORKLOADS[wl]["metric"]
    desc = WORKLOADS[wl]["desc"]
    if not args.box_mode:
        args.box_mode = "interval" if wl in ("batch64", "learned100k") else "speed"
    args.mode = 1 if args.box_mode == "interval" else 0
    desc += ("; INTERVAL boxes (interval evaluation over the eccentric-anomaly range)"
             if args.mode else "; SPEED boxes")
    if args.horizon_s != HORIZON_S:
        desc = desc.replace("24 h", f"{args.horizon_s:.0f} s")
    if wl in ("catalog24h", "band_slab") and (
            args.graph == 1 or (args.graph < 0 and wl == "band_slab")):
        desc += "; the find sequence replayed as one captured CUDA graph"


    if args.impl == "reference":
        if rank != 0:
            return
        # one step = the oracle's 24 h screen measured on a window sample on
        # all host cores (a bounded share of the horizon, scaled up)
        T = int(HORIZON_S / TICK_S)
        cores = os.cpu_count() or 1
        n_w, w_t = 2 * cores, 60
        vals, sdesc = [], ""
        for _ in range(args.warmup):  # warm-up steps: one short window
            cpu_oracle_windows(_windows(1, 10, T), 10, 1)
        for q in range(args.steps):
            starts = _windows(n_w, w_t, T, phase=(q * 0.37) % 1.0)
            wall = cpu_oracle_windows(starts, w_t, cores)[0]
            scale = (T + 1) / (n_w * w_t)
            vals.append(wall * 1e3 * scale)
            sdesc = (f"oracle (box generation, time-sorted sweep, canonical sort) on {n_w} "
                     f"windows of {w_t} ticks per step, spread over the 24 h screen of all "
                     f"{N_OBJ} objects (whole-segment boxes; windows partition the screen "
                     f"exactly), {cores} threads, scaled by {scale:.1f}")
        v = statistics.mean(vals)
        print(json.dumps({
            "impl": "reference", "metric": WORKLOADS["catalog24h"]["metric"], "value": v,
            "unit": "ms", "higher_is_better": False, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64/f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["catalog24h"]["desc"], "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": sdesc, "cpu_model": _cpu_model()},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "step_times_ms": vals,
        }))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if wl in ("catalog24h", "band_slab"):
        r = run_single(args, world, wl)
    elif wl == "narrow24h":
        r = run_narrow(args, world)
    elif wl in ("refine512", "refine24h"):
        r = run_refine(args, world, wl)
    elif wl == "batch64":
        r = run_batch64(args, world)
    else:
        r = run_learned100k(args, world)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank != 0:
        return

    line = {
        "metric": metric, "value": r["value"], "unit": r["unit"], "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(r["times"]), "higher_is_better": r["higher_is_better"],
        "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32", "data": "synthetic",
        "config": {"workload": desc,
                   "l2": ("flushed between steps (writes 2x L2)" if wl == "refine512" else
                          "flushed between steps (writes 2x L2); working set > 1 GB")},
    }
    pk, src = _peaks()
    if "metrics" in r:
        m = r["metrics"]
        line["config"].update({"boxes": m["boxes"], "pairs": r["n_pairs"],
                               "records": m["records"], "open_runs": m["open_runs"],
                               "leaf_size": m["leaf_size"],
                               "morton_bits": m["morton_bits"], "stack_depth": m["stack_depth"],
                               "block_threads": m["block_threads"]})
        line["box_pair_tests_per_s"] = r["tests"] / (sum(r["times"]) * 1e-3)
        line["node_tests"] = m["node_tests"]
        line["leaf_tests"] = m["leaf_tests"]
        ph = r["phase_ms"]
        byt = algorithmic_bytes(m, r["n"])
        # the dominant phase of the screen (the narrow phase of narrow24h is
        # reported on its own, under "narrow")
        dom = max((k for k in ph if k != "ms_narrow"), key=ph.get)
        name = dom[3:]
        hbm = pk.get("hbm_gbs", 6800.0)
        achieved = byt[name] / (ph[dom] * 1e-3) / 1e9
        # the committed capture is of the default configuration only
        default_cfg = (args.horizon_s == HORIZON_S and not args.mode and not args.tuning
                       and not args.autotune)
        traffic = measured_traffic(wl) if name == "traverse" and default_cfg else None
        line["roofline"] = {"kernel_phase": name, "bound": "hbm", "achieved": achieved,
                            "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                            "traffic": traffic,
                            "traffic_source": ("committed ncu capture of these sources "
                                               "(profiles/k_traverse2_catalog16848_24h.md)"
                                               if traffic is not None else None),
                            "peak_source": src, "phase_ms": ph,
                            "algorithmic_bytes": byt[name]}
        if "phase_ms_source" in r:
            line["roofline"]["phase_ms_source"] = r["phase_ms_source"]
        line["gpu_launches"] = r["launches"]
    if wl == "catalog24h":
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline_measure()
        line["cpu_baseline"] = cpu
    if "e2e" in r:
        line["e2e"] = r["e2e"]
    if "gpu_launches" not in line and r.get("launches") is not None:
        line["gpu_launches"] = r["launches"]
    if "roofline_refine" in r:
        line["roofline"] = r["roofline_refine"]
    for k in ("latency_ms", "batches", "objects", "boxes_est", "ms_per_pass", "p100_ms",
              "p100_boxes", "p100_pairs", "training", "tuning", "narrow", "refine",
              "interval_screen"):
        if k in r and r[k] is not None:
            line[k] = r[k]
    line["clocks"] = r["clocks"]
    line["step_times_ms"] = r["times"]
    print(json.dumps(line))


if __name__ == "__main__":
    main()

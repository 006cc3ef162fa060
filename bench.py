"""Benchmark: one 24 h screen of a 16,848-object catalog-shaped population.

A step is one pass of the whole hot path from device-resident elements to
the device-resident canonical pair list: per-object steps (P/100), FP64
propagation, FP32 boxes and Morton keys, radix sort, hierarchy, refit,
traversal with merged emission, canonical sort.  The JSON line's ``value``
is milliseconds per screen (whole job: all ranks' screens over the max-rank
time); ``e2e`` is the same through the C ABI with host buffers (elements
copied in, pairs copied out inside the timed region).

--impl reference times the CPU oracle on a bounded sample of the same
workload (a time window of the horizon) and scales it to a 24 h screen.
"""
from __future__ import annotations

import argparse
import json
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

METRIC = "ms per 24h screen at n=16848"
N_OBJ = 16848
HORIZON_S = 86400.0
TICK_S = 1.0
FRACTION = 100.0
L2_BYTES = 129 * 1024 * 1024
WORKLOAD = ("catalog-shaped synthetic mixture n=16848 (72% LEO, 8% MEO, 10% GEO, 10% HEO, "
            "0.1% seeded crossing pairs), 24 h horizon, 1 s ticks, per-object step P/100, "
            "SPEED boxes, plain 4D LBVH")


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
    """Algorithmic HBM bytes of one screen by phase (each array read or
    written once per pass it needs)."""
    N = m["boxes"]
    L = m["leaf_size"]
    M = (N + L - 1) // L
    runs = m["records"]
    key_b = 4 if m["morton_bits"] <= 8 else 8
    passes = (4 * m["morton_bits"] + 7) // 8
    pair_bits = 2 * max(1, int(np.ceil(np.log2(max(n, 2))))) + int(np.ceil(np.log2(m["T"] + 1)))
    ppasses = (pair_bits + 7) // 8
    return {
        # elements in; boxes (32 B), object id, box id and key out
        "boxes": 56 * n + N * (32 + 4 + 4 + key_b),
        # per pass: keys+values read twice (count, rank), written once
        "sort": passes * N * 3 * (key_b + 4),
        # gather boxes by id; leaf keys; hierarchy nodes and refit
        "build": N * (4 + 32 + 4 + 32 + 4) + M * (key_b + 80 + 32 + 32 + 16),
        # every sorted box and node read at least once; records written
        "traverse": N * (32 + 8) + (M - 1) * 80 + 2 * runs * 8,
        # two key-only sorts of the run records, then the output pairs
        "canon": 2 * ppasses * runs * 8 * 3 + runs * (16 + 16),
    }


def run_ours(args, rank, world):
    import torch

    import paper_1901_10475_gb300 as scd

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    els = P.catalog_mixture(n=N_OBJ, seed=P.SEED_BASE + 2)
    pol = scd.make_step_policy(scd.SCD_STEP_PERIOD_FRACTION, period_fraction=FRACTION)
    sc = scd.Scene(els, args.horizon_s, TICK_S, pol, stream=stream)
    if args.tuning:
        sc.set_tuning(json.loads(args.tuning))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    d_el = torch.as_tensor(els, device="cuda")

    def step():
        scd.scd_scene_set_elements_device(sc.handle, d_el.data_ptr(), N_OBJ)
        scd.scd_build_boxes(sc.handle)
        return scd.scd_find_pairs_device(sc.handle)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    times, phase = [], {k: [] for k in ("ms_boxes", "ms_sort", "ms_build", "ms_traverse", "ms_canon")}
    tests = 0
    launches = 0
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    n_pairs = 0
    with ClockSampler(dev) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))  # evict L2 between steps (outside the timed events)
            ev0[k].record(stream)
            _, n_pairs = step()
            ev1[k].record(stream)
            m = sc.metrics()
            for key in phase:
                phase[key].append(m[key])
            tests += m["node_tests"] + m["leaf_tests"]
            launches += m["launches"]
        torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    t_total = sum(times)
    if world > 1:
        t = torch.tensor([t_total], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_total = float(t.item())
    ms_per_screen = t_total / (args.steps * world)
    m = sc.metrics()

    # end to end through the C ABI with host buffers
    host_in = torch.as_tensor(els).pin_memory()
    host_out = np.zeros(max(2 * n_pairs, 1), scd.PAIR_DTYPE)
    import ctypes
    out_pinned = torch.empty(host_out.nbytes, dtype=torch.uint8).pin_memory()
    out_np = out_pinned.numpy().view(scd.PAIR_DTYPE)
    e2e_times = []
    e2e_steps = max(1, min(args.steps, 5))
    for k in range(e2e_steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        scd._binding.lib().scd_scene_set_elements(sc.handle, ctypes.c_void_p(host_in.data_ptr()),
                                                  N_OBJ)
        scd.scd_build_boxes(sc.handle)
        n_host = scd.scd_find_pairs_into(sc.handle, out_np)
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = statistics.median(e2e_times)

    byt = algorithmic_bytes(m, N_OBJ)
    phase_ms = {k: statistics.mean(v) for k, v in phase.items()}
    pk, src = _peaks()
    return {
        "ms_per_screen": ms_per_screen, "times": times, "phase_ms": phase_ms, "tests": tests,
        "launches": launches, "metrics": m, "bytes": byt, "n_pairs": n_pairs, "clocks": clk.summary(),
        "e2e_ms": e2e_ms, "e2e_pairs": n_host, "peaks": pk, "peak_src": src,
    }


def cpu_oracle_sample(window_ticks: int = 600):
    """The oracle on a bounded sample: every object's boxes whose segments
    start inside [0, window] of the 24 h screen, their overlap set and
    canonical list.  Returns (seconds, sample description, ms per 24 h)."""
    import oracle as O
    els = P.catalog_mixture(n=N_OBJ, seed=P.SEED_BASE + 2)
    t0 = time.perf_counter()
    k = O.step_ticks(els, O.STEP_PERIOD_FRACTION, TICK_S, frac=FRACTION)
    lo, hi, obj = O.boxes(els, window_ticks, TICK_S, k, O.BOX_SPEED)
    cells = O.canonicalize(O.raw_cells_sweep(lo, hi, obj))
    sec = time.perf_counter() - t0
    scale = (HORIZON_S / TICK_S + 1) / (window_ticks + 1)
    desc = (f"oracle (1 thread) on the first {window_ticks + 1} ticks of the 24 h screen, all "
            f"{N_OBJ} objects ({len(lo)} boxes, {len(cells)} pairs), scaled by {scale:.1f}")
    return sec, desc, sec * 1e3 * scale


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tuning", default="")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--horizon-s", type=float, default=HORIZON_S,
                    help="shorter horizons give the small profiling case")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        for _ in range(args.warmup):
            cpu_oracle_sample(120)
        desc = ""
        for _ in range(args.steps):
            sec, desc, ms = cpu_oracle_sample(120)
            vals.append(ms)
        v = statistics.mean(vals)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "ms",
            "higher_is_better": False, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64/f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    m = r["metrics"]
    byt = r["bytes"]
    ph = r["phase_ms"]
    # dominant phase and its roofline
    dom = max(ph, key=ph.get)
    name = dom[3:]
    hbm = r["peaks"].get("hbm_gbs", 6800.0)
    achieved = byt[name] / (ph[dom] * 1e-3) / 1e9
    roof = {"kernel_phase": name, "bound": "hbm", "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
            "peak_source": r["peak_src"], "phase_ms": ph,
            "algorithmic_bytes": byt[name]}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        sec, desc, ms = cpu_oracle_sample(600)
        cpu = {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle", "sample": desc,
               "sample_seconds": sec}
    ms = r["ms_per_screen"]
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.horizon_s == HORIZON_S else
                   WORKLOAD.replace("24 h horizon", f"{args.horizon_s:.0f} s horizon"),
                   "boxes": m["boxes"], "pairs": r["n_pairs"],
                   "records": m["records"], "leaf_size": m["leaf_size"],
                   "morton_bits": m["morton_bits"], "stack_depth": m["stack_depth"],
                   "block_threads": m["block_threads"],
                   "l2": "flushed between steps (writes 2x L2); working set > 1 GB"},
        "box_pair_tests_per_s": r["tests"] / (sum(r["times"]) * 1e-3),
        "node_tests": m["node_tests"], "leaf_tests": m["leaf_tests"],
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": r["e2e_ms"], "unit": "ms", "h2d_bytes_per_step": 56 * N_OBJ,
                "d2h_bytes_per_step": 16 * r["e2e_pairs"]},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "step_times_ms": r["times"],
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()

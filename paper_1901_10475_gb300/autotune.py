"""Autotuner for the screen's tree and traversal parameters.

Times whole screens (boxes through the canonical list) with CUDA events on
the scene's stream for candidate tunings, keeps the fastest, and caches the
choice in a JSON file keyed by GPU name, a hash of the workload and log2 of
the box count.  A staged search: leaf size x Morton bits x space warp
first, then the time weight, the stack depth, the size split of the key and
the block shape (leaves of several boxes) or the nodes per traversal step
and the node width (one box per leaf) around the winner.
"""
from __future__ import annotations

import hashlib
import json
import math
import os

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib",
                             "autotune_cache.json")

STAGE1 = [dict(leaf_size=L, morton_bits=b, space_warp=w)
          for L in (1, 2, 4) for b in (8, 10, 12, 16) for w in (0, 1)]


def _time_screen(scene, reps: int, decomp=None) -> float:
    import torch
    from . import _binding as B
    st = torch.cuda.current_stream()
    best = float("inf")
    for r in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        B.scd_build_boxes(scene.handle)
        B.scd_find_pairs_device(scene.handle, decomp)
        e1.record(st)
        e1.synchronize()
        if r > 0:  # the first run sizes buffers
            best = min(best, e0.elapsed_time(e1))
    return best


def workload_key(elements, horizon_s: float, tick_s: float, step_desc: str, nboxes: int) -> str:
    import numpy as np
    import torch
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(elements, dtype=np.float64).tobytes())
    h.update(f"{horizon_s}:{tick_s}:{step_desc}".encode())
    name = torch.cuda.get_device_name()
    return f"{name}|{h.hexdigest()[:16]}|log2N={int(math.log2(max(nboxes, 1)))}"


STAGE1_DECOMPOSED = [dict(leaf_size=1, morton_bits=b, space_warp=w)
                     for b in (8, 10, 12) for w in (0, 1)]


def tune(scene, reps: int = 2, verbose: bool = False, decomp=None):
    """Search the tuning space on `scene` (boxes are rebuilt for every
    candidate; `decomp` as for scd_find_pairs).  Returns (best tuning dict,
    list of (tuning, ms))."""
    from . import _binding as B
    base = {f: getattr(B.scd_default_tuning(), f) for f, _ in B.scd_tuning._fields_}
    results = []

    def run(cand):
        t = dict(base)
        t.update(cand)
        scene.set_tuning(t)
        ms = _time_screen(scene, reps, decomp)
        results.append((t, ms))
        if verbose:
            print(f"autotune {cand} -> {ms:.3f} ms", flush=True)
        return ms

    best, best_ms = None, float("inf")
    for cand in (STAGE1 if decomp is None else STAGE1_DECOMPOSED):
        ms = run(cand)
        if ms < best_ms:
            best, best_ms = dict(cand), ms
    stage2 = [dict(best, time_scale=ts) for ts in (1.0, 4.0, 8.0, 16.0) if ts != base["time_scale"]]
    stage2 += [dict(best, stack_depth=sd) for sd in (32, 128)]
    # the size split: off, a finer and a coarser threshold than the default
    stage2 += [dict(best, split_km=sk) for sk in (0.0, -500.0, -1000.0, -2000.0)
               if sk != base["split_km"]]
    if best["leaf_size"] > 1:
        stage2 += [dict(best, block_threads=bt) for bt in (64, 256)]
    else:
        stage2 += [dict(best, nodes_per_step=1), dict(best, node_width=4)]
    for cand in stage2:
        ms = run(cand)
        if ms < best_ms:
            best, best_ms = dict(cand), ms
    full = dict(base)
    full.update(best)
    scene.set_tuning(full)
    return full, results


def load_or_tune(scene, key: str, cache_path: str = DEFAULT_CACHE, reps: int = 2,
                 verbose: bool = False, decomp=None):
    """The cached tuning for `key`, or a fresh search whose result is cached."""
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        scene.set_tuning(cache[key]["tuning"])
        return cache[key]["tuning"], None
    best, results = tune(scene, reps=reps, verbose=verbose, decomp=decomp)
    cache[key] = {"tuning": best, "ms": min(ms for _, ms in results)}
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return best, results

"""GB300-native broad-phase n-to-n screening over 4D space-time boxes
(Bak & Hobbs, "Efficient n-to-n Collision Detection for Space Debris using
4D AABB Trees").

The work runs in libscd.so (hand-written sm_103a CUDA behind the C ABI of
include/scd.h); this package marshals arguments and uses PyTorch only for
device memory (its caching allocator) and streams.
"""
from __future__ import annotations

import json

import numpy as np

from . import _binding as B
from ._binding import (PAIR_DTYPE, SCD_BOX_INTERVAL, SCD_BOX_SPEED, SCD_DECOMP_ALT_BANDS,
                       SCD_DECOMP_NONE, SCD_DECOMP_SLAB_OCT, SCD_STEP_BAND_TABLE, SCD_STEP_FIXED,
                       SCD_STEP_LEARNED, SCD_STEP_PERIOD_FRACTION, ScdError, make_step_policy,
                       scd_batch_find_pairs, scd_build_boxes, scd_default_tuning,
                       scd_find_pairs, scd_find_pairs_device, scd_find_pairs_into,
                       scd_find_raw_cells_device,
                       WITNESS_DTYPE, scd_get_boxes, scd_get_steps, scd_last_metrics,
                       scd_narrow_phase, scd_refine_continuous, scd_refine_trace,
                       scd_refine_witnesses,
                       SPAN_DTYPE,
                       scd_propagate,
                       scd_propagate_noalloc,
                       scd_scene_create, scd_scene_destroy, scd_scene_set_elements,
                       scd_scene_get_tuning, scd_scene_set_elements_device,
                       scd_scene_set_tuning, scd_status_string, scd_tuning)

for _n in dir(B):  # every entry point and constant under its C name
    if _n.startswith("scd_") or _n.startswith("SCD_"):
        globals()[_n] = getattr(B, _n)

__all__ = [n for n in dir(B) if n.startswith("scd_") or n.startswith("SCD_")] + [
    "Scene", "device_view", "PAIR_DTYPE", "WITNESS_DTYPE", "SPAN_DTYPE", "ScdError",
    "make_step_policy"]


class _CudaArray:
    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def device_view(ptr: int, shape, typestr: str):
    """A torch tensor viewing device memory owned by the library (no copy)."""
    import torch
    if int(np.prod(shape)) == 0:
        dt = {"<f4": torch.float32, "<u4": torch.int32, "<i4": torch.int32,
              "<f8": torch.float64}[typestr]
        return torch.empty(tuple(shape), dtype=dt, device="cuda")
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")


class Scene:
    """One screening problem: n objects over [0, horizon] in ticks of tick_s."""

    def __init__(self, elements, horizon_s: float, tick_s: float = 1.0, step=None,
                 mode: int = SCD_BOX_SPEED, stream=None, tuning=None):
        import torch
        B.use_torch_allocator()
        if step is None:
            step = make_step_policy(SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        self.n = len(elements)
        self.handle = scd_scene_create(elements, horizon_s, tick_s, step, mode,
                                       int(stream.cuda_stream))
        if tuning is not None:
            self.set_tuning(tuning)

    def set_tuning(self, t):
        if isinstance(t, dict):
            x = scd_default_tuning()
            for k, v in t.items():
                setattr(x, k, v)
            t = x
        scd_scene_set_tuning(self.handle, t)

    def tuning(self) -> dict:
        t = scd_scene_get_tuning(self.handle)
        return {f: getattr(t, f) for f, _ in scd_tuning._fields_}

    def set_elements(self, elements):
        scd_scene_set_elements(self.handle, elements)

    def build_boxes(self):
        scd_build_boxes(self.handle)
        return self

    def find_pairs(self, decomp=None) -> np.ndarray:
        return scd_find_pairs(self.handle, decomp)

    def find_pairs_device(self, decomp=None):
        ptr, n = scd_find_pairs_device(self.handle, decomp)
        return device_view(ptr, (n, 4), "<i4")

    def find_raw_cells_device(self):
        ptr, n = scd_find_raw_cells_device(self.handle)
        return device_view(ptr, (n, 4), "<i4")

    def narrow_phase(self, pairs):
        """Collision witnesses inside a device candidate list (an (m, 4) int32
        tensor of scd_pair records, e.g. find_pairs_device()): per candidate
        the first witness tick (-1: none) and the witness count, as device
        tensors, and the earliest witness (i, j, t) in Alg 1's order, or
        None."""
        import torch
        m = int(pairs.shape[0])
        first = torch.empty(m, dtype=torch.int32, device=pairs.device)
        count = torch.empty(m, dtype=torch.int32, device=pairs.device)
        w = scd_narrow_phase(self.handle, pairs.data_ptr() if m else 0, m,
                             first.data_ptr() if m else 0, count.data_ptr() if m else 0)
        return first, count, w

    def refine_witnesses(self):
        """Every collision witness (i, j, t) by adaptive refinement, in Alg
        1's order, and the active intervals of each round (needs
        build_boxes)."""
        return scd_refine_witnesses(self.handle)

    def refine_continuous(self, eps_s: float):
        """Spans (i, j, t0, t1) of the continuous-time refinement down to
        intervals of eps_s seconds, and the active intervals per round."""
        return scd_refine_continuous(self.handle, eps_s)

    def boxes(self):
        lo, hi, obj, n = scd_get_boxes(self.handle)
        return (device_view(lo, (n, 4), "<f4"), device_view(hi, (n, 4), "<f4"),
                device_view(obj, (n,), "<i4"))

    def steps(self):
        return device_view(scd_get_steps(self.handle), (self.n,), "<i4")

    def metrics(self) -> dict:
        return json.loads(scd_last_metrics(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            scd_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchScene(Scene):
    """Many independent scenes (own elements and horizons) screened in one
    build, one sort, one tree and one persistent traversal."""

    def __init__(self, elements_list, horizons_s, tick_s: float = 1.0, step=None,
                 mode: int = SCD_BOX_SPEED, stream=None, tuning=None):
        import torch
        B.use_torch_allocator()
        if step is None:
            step = make_step_policy(SCD_STEP_PERIOD_FRACTION, period_fraction=100.0)
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        self.n_scenes = len(elements_list)
        self.handle, self.scene_off = B.scd_batch_scene_create(
            elements_list, horizons_s, tick_s, step, mode, int(stream.cuda_stream))
        self.n = int(self.scene_off[-1])
        if tuning is not None:
            self.set_tuning(tuning)

    def find_pairs_per_scene(self):
        """One array per scene, object indices local to the scene."""
        allp = self.find_pairs()
        off = B.scd_batch_scene_offsets(self.handle, self.n_scenes)
        out = []
        for k in range(self.n_scenes):
            p = allp[off[k]:off[k + 1]].copy()
            p["i"] -= np.uint32(self.scene_off[k])
            p["j"] -= np.uint32(self.scene_off[k])
            out.append(p)
        return out


def pairs_from_device(t) -> np.ndarray:
    """Copy an (n, 4) int32 device view of scd_pair records to numpy."""
    a = t.cpu().numpy()
    out = np.zeros(len(a), PAIR_DTYPE)
    out["i"] = a[:, 0].view(np.uint32)
    out["j"] = a[:, 1].view(np.uint32)
    out["tlo"] = a[:, 2]
    out["thi"] = a[:, 3]
    return out

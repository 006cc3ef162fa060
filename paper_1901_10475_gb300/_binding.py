"""ctypes binding of libscd (include/scd.h): argument marshalling only.

Every name here is the C entry point of the same name.  The library is the
compiled CUDA path; there is no CPU fallback.  If the shared library cannot
be built or loaded, importing fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SCD_OK = 0
SCD_ERR_INVALID_ARG = -1
SCD_ERR_OOM = -2
SCD_ERR_BUFFER_TOO_SMALL = -3
SCD_ERR_CUDA = -4
SCD_ERR_KEPLER_NOCONV = -5
SCD_ERR_TIMEOUT = -6
SCD_ERR_INTERNAL = -7
SCD_ERR_STATE = -8
SCD_ERR_CAPACITY = -9
SCD_NOALLOC_MAX_OBJECTS = 32768

SCD_STEP_FIXED, SCD_STEP_PERIOD_FRACTION, SCD_STEP_BAND_TABLE, SCD_STEP_LEARNED = 0, 1, 2, 3
SCD_BOX_SPEED, SCD_BOX_INTERVAL = 0, 1
SCD_DECOMP_NONE, SCD_DECOMP_ALT_BANDS, SCD_DECOMP_SLAB_OCT = 0, 1, 2


class scd_element(ctypes.Structure):
    _fields_ = [("a_km", ctypes.c_double), ("e", ctypes.c_double), ("inc_rad", ctypes.c_double),
                ("raan_rad", ctypes.c_double), ("argp_rad", ctypes.c_double),
                ("M0_rad", ctypes.c_double), ("radius_km", ctypes.c_double)]


class scd_step_policy(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("fixed_ticks", ctypes.c_uint32),
                ("period_fraction", ctypes.c_double),
                ("band_edges_km", ctypes.POINTER(ctypes.c_double)),
                ("band_fractions", ctypes.POINTER(ctypes.c_double)),
                ("n_bands", ctypes.c_int), ("stepnet", ctypes.c_void_p)]


class scd_decomp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p_bands", ctypes.c_int), ("n_slabs", ctypes.c_int)]


class scd_pair(ctypes.Structure):
    _fields_ = [("i", ctypes.c_uint32), ("j", ctypes.c_uint32), ("tlo", ctypes.c_int32),
                ("thi", ctypes.c_int32)]


class scd_tuning(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("stack_depth", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("morton_bits", ctypes.c_int),
                ("time_scale", ctypes.c_float), ("use_graph", ctypes.c_int),
                ("space_warp", ctypes.c_int), ("nodes_per_step", ctypes.c_int),
                ("node_width", ctypes.c_int), ("split_km", ctypes.c_float),
                ("refine_start", ctypes.c_float)]


class scd_witness(ctypes.Structure):
    _fields_ = [("i", ctypes.c_uint32), ("j", ctypes.c_uint32), ("t", ctypes.c_int32)]


PAIR_DTYPE = np.dtype([("i", "<u4"), ("j", "<u4"), ("tlo", "<i4"), ("thi", "<i4")])

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None


class ScdError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def lib() -> ctypes.CDLL:
    """Load libscd.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        P = ctypes.POINTER
        sigs = {
            "scd_set_allocator": (i32, [ALLOC_FN, FREE_FN, vp]),
            "scd_scene_create": (i32, [vp, i64, d, d, P(scd_step_policy), i32, vp, P(vp)]),
            "scd_scene_set_elements": (i32, [vp, vp, i64]),
            "scd_scene_set_elements_device": (i32, [vp, vp, i64]),
            "scd_scene_set_tuning": (i32, [vp, P(scd_tuning)]),
            "scd_default_tuning": (i32, [P(scd_tuning)]),
            "scd_scene_get_tuning": (i32, [vp, P(scd_tuning)]),
            "scd_build_boxes": (i32, [vp]),
            "scd_find_pairs": (i32, [vp, P(scd_decomp), vp, i64, P(i64)]),
            "scd_find_pairs_device": (i32, [vp, P(scd_decomp), P(vp), P(i64)]),
            "scd_find_raw_cells_device": (i32, [vp, P(vp), P(i64)]),
            "scd_get_boxes": (i32, [vp, P(vp), P(vp), P(vp), P(i64)]),
            "scd_narrow_phase": (i32, [vp, vp, i64, vp, vp, P(scd_witness)]),
            "scd_refine_witnesses": (i32, [vp, vp, i64, P(i64), vp, P(i32)]),
            "scd_refine_continuous": (i32, [vp, d, vp, i64, P(i64), vp, P(i32)]),
            "scd_refine_trace": (i32, [vp, d, vp, vp, vp, i64, P(i64), vp, P(i32)]),
            "scd_get_steps": (i32, [vp, P(vp)]),
            "scd_propagate": (i32, [vp, i64, vp, vp, i64, vp, vp]),
            "scd_propagate_noalloc": (i32, [vp, i64, vp, vp, i64, vp, vp]),
            "scd_batch_find_pairs": (i32, [P(vp), i32, P(scd_decomp), P(vp), P(i64), P(i64)]),
            "scd_last_metrics": (i32, [vp, ctypes.c_char_p, ctypes.c_size_t]),
            "scd_stepnet_create": (i32, [vp, ctypes.c_uint64, P(vp)]),
            "scd_stepnet_set_params": (i32, [vp, vp, i64]),
            "scd_stepnet_get_params": (i32, [vp, vp, i64]),
            "scd_stepnet_features": (i32, [vp, i64, vp, vp]),
            "scd_stepnet_forward": (i32, [vp, vp, i64, vp]),
            "scd_stepnet_grad": (i32, [vp, vp, vp, i64, vp, P(ctypes.c_float)]),
            "scd_stepnet_train_step": (i32, [vp, vp, vp, i64, ctypes.c_float, ctypes.c_float,
                                             P(ctypes.c_float)]),
            "scd_stepnet_save": (i32, [vp, ctypes.c_char_p]),
            "scd_stepnet_load": (i32, [vp, ctypes.c_char_p]),
            "scd_stepnet_destroy": (None, [vp]),
            "scd_count_pairs_per_object": (i32, [vp, i64, i64, vp, vp]),
            "scd_batch_scene_create": (i32, [vp, vp, vp, i32, d, P(scd_step_policy), i32, vp,
                                             P(vp)]),
            "scd_batch_scene_offsets": (i32, [vp, vp]),
            "scd_scene_destroy": (None, [vp]),
            "scd_status_string": (ctypes.c_char_p, [i32]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def status_string(status: int) -> str:
    return lib().scd_status_string(int(status)).decode()


def check(status: int, what: str) -> None:
    if status != SCD_OK:
        raise ScdError(status, what)


# --- torch caching allocator as the device allocator ----------------------

_torch_hooks = None


def use_torch_allocator() -> None:
    """Route libscd's device allocations through torch's caching allocator."""
    global _torch_hooks
    if _torch_hooks is not None:
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:  # out of memory: the library reports SCD_ERR_OOM
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    check(lib().scd_set_allocator(hooks[0], hooks[1], None), "scd_set_allocator")
    _torch_hooks = hooks


# --- entry points with the C names ----------------------------------------

def _elems(els) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(els, dtype=np.float64))
    if a.ndim != 2 or a.shape[1] != 7:
        raise ValueError("elements must be an (n, 7) float64 array")
    return a


def make_step_policy(kind: int = SCD_STEP_PERIOD_FRACTION, fixed_ticks: int = 1,
                     period_fraction: float = 100.0, band_edges_km=(), band_fractions=(),
                     stepnet: int = 0):
    pol = scd_step_policy()
    pol.kind = kind
    pol.stepnet = stepnet or None
    pol.fixed_ticks = int(fixed_ticks)
    pol.period_fraction = float(period_fraction)
    keep = []
    if kind == SCD_STEP_BAND_TABLE:
        e = np.ascontiguousarray(np.asarray(band_edges_km, np.float64).reshape(-1))
        f = np.ascontiguousarray(np.asarray(band_fractions, np.float64).reshape(-1))
        keep = [e, f]
        pol.band_edges_km = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        pol.band_fractions = f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        pol.n_bands = len(f)
    pol._keep = keep  # the arrays must outlive the create call
    return pol


def scd_scene_create(els, horizon_s: float, tick_s: float, policy: scd_step_policy,
                     mode: int = SCD_BOX_SPEED, stream: int = 0) -> int:
    a = _elems(els)
    out = ctypes.c_void_p()
    check(lib().scd_scene_create(a.ctypes.data, len(a), float(horizon_s), float(tick_s),
                                 ctypes.byref(policy), int(mode), ctypes.c_void_p(stream),
                                 ctypes.byref(out)), "scd_scene_create")
    return out.value


def scd_scene_set_elements(scene: int, els) -> None:
    a = _elems(els)
    check(lib().scd_scene_set_elements(scene, a.ctypes.data, len(a)), "scd_scene_set_elements")


def scd_scene_set_elements_device(scene: int, d_ptr: int, n: int) -> None:
    check(lib().scd_scene_set_elements_device(scene, d_ptr, n), "scd_scene_set_elements_device")


def scd_default_tuning() -> scd_tuning:
    t = scd_tuning()
    check(lib().scd_default_tuning(ctypes.byref(t)), "scd_default_tuning")
    return t


def scd_scene_set_tuning(scene: int, t: scd_tuning) -> None:
    check(lib().scd_scene_set_tuning(scene, ctypes.byref(t)), "scd_scene_set_tuning")


def scd_scene_get_tuning(scene: int) -> scd_tuning:
    t = scd_tuning()
    check(lib().scd_scene_get_tuning(scene, ctypes.byref(t)), "scd_scene_get_tuning")
    return t


def scd_build_boxes(scene: int) -> None:
    check(lib().scd_build_boxes(scene), "scd_build_boxes")


def _decomp(d):
    if d is None:
        return None
    if isinstance(d, scd_decomp):
        return ctypes.byref(d)
    x = scd_decomp()
    x.kind, x.p_bands, x.n_slabs = d
    return ctypes.byref(x)


def scd_find_pairs(scene: int, decomp=None, cap: int | None = None) -> np.ndarray:
    """Canonical pair list copied to host memory (a numpy PAIR_DTYPE array)."""
    n = ctypes.c_int64(0)
    if cap is None:
        cap = 1 << 16
    while True:
        out = np.zeros(max(cap, 1), PAIR_DTYPE)
        rc = lib().scd_find_pairs(scene, _decomp(decomp), out.ctypes.data, cap, ctypes.byref(n))
        if rc == SCD_ERR_BUFFER_TOO_SMALL:
            cap = int(n.value)
            continue
        check(rc, "scd_find_pairs")
        return out[:n.value]


def scd_find_pairs_into(scene: int, host_out: np.ndarray, decomp=None) -> int:
    """Fill a caller-owned (pinned) host array; returns the pair count."""
    n = ctypes.c_int64(0)
    rc = lib().scd_find_pairs(scene, _decomp(decomp), host_out.ctypes.data, len(host_out),
                              ctypes.byref(n))
    check(rc, "scd_find_pairs")
    return int(n.value)


def scd_find_pairs_device(scene: int, decomp=None):
    """(device pointer, count) of the canonical list, owned by the scene."""
    p, n = ctypes.c_void_p(), ctypes.c_int64(0)
    check(lib().scd_find_pairs_device(scene, _decomp(decomp), ctypes.byref(p), ctypes.byref(n)),
          "scd_find_pairs_device")
    return p.value, int(n.value)


def scd_find_raw_cells_device(scene: int):
    p, n = ctypes.c_void_p(), ctypes.c_int64(0)
    check(lib().scd_find_raw_cells_device(scene, ctypes.byref(p), ctypes.byref(n)),
          "scd_find_raw_cells_device")
    return p.value, int(n.value)


def scd_narrow_phase(scene: int, d_pairs: int, n_pairs: int, d_first: int = 0,
                     d_count: int = 0):
    """Narrow phase over n_pairs device candidates: fills the device arrays
    d_first (int32) and d_count (uint32) when given; returns the earliest
    witness (i, j, t) in Alg 1's order, or None."""
    w = scd_witness()
    check(lib().scd_narrow_phase(scene, d_pairs or None, int(n_pairs), d_first or None,
                                 d_count or None, ctypes.byref(w)), "scd_narrow_phase")
    return None if w.t < 0 else (int(w.i), int(w.j), int(w.t))


WITNESS_DTYPE = np.dtype([("i", "<u4"), ("j", "<u4"), ("t", "<i4")])


def scd_refine_witnesses(scene: int, cap: int = 1 << 16):
    """Every collision witness of the scene by adaptive refinement, in Alg
    1's order (a numpy WITNESS_DTYPE array), and the active intervals of
    each round."""
    n = ctypes.c_int64(0)
    rounds = ctypes.c_int(0)
    rb = np.zeros(64, np.int64)
    while True:
        out = np.zeros(max(cap, 1), WITNESS_DTYPE)
        rc = lib().scd_refine_witnesses(scene, out.ctypes.data, cap, ctypes.byref(n),
                                        rb.ctypes.data, ctypes.byref(rounds))
        if rc == SCD_ERR_BUFFER_TOO_SMALL:
            cap = int(n.value)
            continue
        check(rc, "scd_refine_witnesses")
        return out[:n.value].copy(), rb[:rounds.value].copy()


SPAN_DTYPE = np.dtype([("i", "<u4"), ("j", "<u4"), ("t0", "<f8"), ("t1", "<f8")])


def scd_refine_continuous(scene: int, eps_s: float, cap: int = 1 << 16):
    """The continuous-time refinement's spans (i, j, t0, t1) at resolution
    eps_s (a numpy SPAN_DTYPE array), and the active intervals per round."""
    n = ctypes.c_int64(0)
    rounds = ctypes.c_int(0)
    rb = np.zeros(64, np.int64)
    while True:
        out = np.zeros(max(cap, 1), SPAN_DTYPE)
        rc = lib().scd_refine_continuous(scene, float(eps_s), out.ctypes.data, cap,
                                         ctypes.byref(n), rb.ctypes.data, ctypes.byref(rounds))
        if rc == SCD_ERR_BUFFER_TOO_SMALL:
            cap = int(n.value)
            continue
        check(rc, "scd_refine_continuous")
        return out[:n.value].copy(), rb[:rounds.value].copy()


def scd_refine_trace(scene: int, eps_s: float = 0.0, cap: int = 1 << 20):
    """Every round's boxes of the refinement (discrete when eps_s <= 0, else
    the continuous variant at eps_s): a list with, per round, (lo4, hi4,
    obj) numpy arrays."""
    n = ctypes.c_int64(0)
    rounds = ctypes.c_int(0)
    rb = np.zeros(64, np.int64)
    while True:
        lo = np.zeros((max(cap, 1), 4), np.float32)
        hi = np.zeros((max(cap, 1), 4), np.float32)
        obj = np.zeros(max(cap, 1), np.uint32)
        rc = lib().scd_refine_trace(scene, float(eps_s), lo.ctypes.data, hi.ctypes.data,
                                    obj.ctypes.data, cap, ctypes.byref(n), rb.ctypes.data,
                                    ctypes.byref(rounds))
        if rc == SCD_ERR_BUFFER_TOO_SMALL:
            cap = int(n.value)
            continue
        check(rc, "scd_refine_trace")
        out, off = [], 0
        for m in rb[:rounds.value]:
            out.append((lo[off:off + m].copy(), hi[off:off + m].copy(), obj[off:off + m].copy()))
            off += int(m)
        return out


def scd_get_boxes(scene: int):
    lo, hi, obj, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64(0)
    check(lib().scd_get_boxes(scene, ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(obj),
                              ctypes.byref(n)), "scd_get_boxes")
    return lo.value, hi.value, obj.value, int(n.value)


def scd_get_steps(scene: int) -> int:
    p = ctypes.c_void_p()
    check(lib().scd_get_steps(scene, ctypes.byref(p)), "scd_get_steps")
    return p.value


def scd_propagate(d_elems: int, n: int, d_obj: int, d_t: int, m: int, d_out: int,
                  stream: int = 0) -> None:
    check(lib().scd_propagate(d_elems, n, d_obj, d_t, m, d_out, ctypes.c_void_p(stream)),
          "scd_propagate")


def scd_propagate_noalloc(d_elems: int, n: int, d_obj: int, d_t: int, m: int, d_out: int,
                          stream: int = 0) -> None:
    """scd_propagate for callers that cannot allocate device memory: the
    scratch lives in a fixed device array of SCD_NOALLOC_MAX_OBJECTS entries,
    shared by all calls (serialise calls that could overlap on the GPU)."""
    check(lib().scd_propagate_noalloc(d_elems, n, d_obj, d_t, m, d_out, ctypes.c_void_p(stream)),
          "scd_propagate_noalloc")


def scd_batch_find_pairs(scenes, decomp=None, caps=None):
    k = len(scenes)
    arr = (ctypes.c_void_p * k)(*scenes)
    caps = list(caps) if caps is not None else [1 << 16] * k
    while True:
        outs = [np.zeros(max(c, 1), PAIR_DTYPE) for c in caps]
        optr = (ctypes.c_void_p * k)(*[o.ctypes.data for o in outs])
        c_caps = (ctypes.c_int64 * k)(*caps)
        n_outs = (ctypes.c_int64 * k)()
        rc = lib().scd_batch_find_pairs(arr, k, _decomp(decomp), optr, c_caps, n_outs)
        if rc == SCD_ERR_BUFFER_TOO_SMALL:
            caps = [max(caps[q], int(n_outs[q])) for q in range(k)]
            continue
        check(rc, "scd_batch_find_pairs")
        return [outs[q][:n_outs[q]] for q in range(k)]


def scd_last_metrics(scene: int) -> str:
    buf = ctypes.create_string_buffer(4096)
    check(lib().scd_last_metrics(scene, buf, len(buf)), "scd_last_metrics")
    return buf.value.decode()


SCD_STEPNET_IN, SCD_STEPNET_HIDDEN, SCD_STEPNET_PARAMS = 8, 64, 4801


def scd_stepnet_create(stream: int = 0, seed: int = 1) -> int:
    out = ctypes.c_void_p()
    check(lib().scd_stepnet_create(ctypes.c_void_p(stream), int(seed), ctypes.byref(out)),
          "scd_stepnet_create")
    return out.value


def scd_stepnet_set_params(net: int, params) -> None:
    a = np.ascontiguousarray(np.asarray(params, np.float32).reshape(-1))
    check(lib().scd_stepnet_set_params(net, a.ctypes.data, len(a)), "scd_stepnet_set_params")


def scd_stepnet_get_params(net: int) -> np.ndarray:
    a = np.zeros(SCD_STEPNET_PARAMS, np.float32)
    check(lib().scd_stepnet_get_params(net, a.ctypes.data, len(a)), "scd_stepnet_get_params")
    return a


def scd_stepnet_features(d_elems: int, n: int, d_feat: int, stream: int = 0) -> None:
    check(lib().scd_stepnet_features(d_elems, n, d_feat, ctypes.c_void_p(stream)),
          "scd_stepnet_features")


def scd_stepnet_forward(net: int, d_x: int, n: int, d_y: int) -> None:
    check(lib().scd_stepnet_forward(net, d_x, n, d_y), "scd_stepnet_forward")


def scd_stepnet_grad(net: int, d_x: int, d_t: int, n: int, d_grad: int) -> float:
    loss = ctypes.c_float(0)
    check(lib().scd_stepnet_grad(net, d_x, d_t, n, d_grad, ctypes.byref(loss)), "scd_stepnet_grad")
    return float(loss.value)


def scd_stepnet_train_step(net: int, d_x: int, d_t: int, n: int, lr: float,
                           weight_decay: float = 0.0) -> float:
    loss = ctypes.c_float(0)
    check(lib().scd_stepnet_train_step(net, d_x, d_t, n, float(lr), float(weight_decay),
                                       ctypes.byref(loss)), "scd_stepnet_train_step")
    return float(loss.value)


def scd_stepnet_save(net: int, path: str) -> None:
    check(lib().scd_stepnet_save(net, path.encode()), "scd_stepnet_save")


def scd_stepnet_load(net: int, path: str) -> None:
    check(lib().scd_stepnet_load(net, path.encode()), "scd_stepnet_load")


def scd_stepnet_destroy(net: int) -> None:
    if net:
        lib().scd_stepnet_destroy(net)


def scd_count_pairs_per_object(d_pairs: int, n_pairs: int, n_objects: int, d_counts: int,
                               stream: int = 0) -> None:
    check(lib().scd_count_pairs_per_object(d_pairs, n_pairs, n_objects, d_counts,
                                           ctypes.c_void_p(stream)), "scd_count_pairs_per_object")


def scd_batch_scene_create(elements_list, horizons_s, tick_s: float, policy,
                           mode: int = SCD_BOX_SPEED, stream: int = 0):
    """One scene holding a batch of independent scenes; returns (handle,
    scene offsets)."""
    els = np.ascontiguousarray(np.concatenate([_elems(e) for e in elements_list]))
    off = np.zeros(len(elements_list) + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in elements_list])
    hz = np.ascontiguousarray(np.asarray(horizons_s, np.float64))
    out = ctypes.c_void_p()
    check(lib().scd_batch_scene_create(els.ctypes.data, off.ctypes.data, hz.ctypes.data,
                                       len(elements_list), float(tick_s), ctypes.byref(policy),
                                       int(mode), ctypes.c_void_p(stream), ctypes.byref(out)),
          "scd_batch_scene_create")
    return out.value, off


def scd_batch_scene_offsets(scene: int, n_scenes: int) -> np.ndarray:
    off = np.zeros(n_scenes + 1, np.int64)
    check(lib().scd_batch_scene_offsets(scene, off.ctypes.data), "scd_batch_scene_offsets")
    return off


def scd_scene_destroy(scene: int) -> None:
    if scene:
        lib().scd_scene_destroy(scene)


def scd_status_string(status: int) -> str:
    return status_string(status)

"""Plain FP64 CPU oracle for 4D space-time box screening (Bak & Hobbs,
"Efficient n-to-n Collision Detection for Space Debris using 4D AABB Trees").

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library: the C part (``oracle.c``) is compiled by ``build()``
below with gcc and driven through ctypes; the step-network part is numpy.

Element arrays are float64 with shape (n, 7): a [km], e, i, RAAN, argument of
perigee, mean anomaly at t=0 [rad], radius [km].  Time is integer ticks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "lib", "liboracle.so")
_lock = threading.Lock()
_lib = None

CELL_DTYPE = np.dtype([("i", "<u4"), ("j", "<u4"), ("tlo", "<i4"), ("thi", "<i4")])
WITNESS_DTYPE = np.dtype([("i", "<u4"), ("j", "<u4"), ("t", "<i4")])

STEP_FIXED, STEP_PERIOD_FRACTION, STEP_BAND_TABLE = 0, 1, 2
BOX_SPEED, BOX_INTERVAL = 0, 1
MU = 398600.4418
RE = 6378.137
EPS_KM = 1e-6


def build(force: bool = False) -> str:
    """Compile oracle.c into lib/liboracle.so (gcc, FP contraction off so
    that a*b+c is never fused: the same decisions on x86 and Arm)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src),
                                                   os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            d, i64, i32, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            sig = {
                "or_mean_motion": (d, [vp]), "or_period": (d, [vp]), "or_max_speed": (d, [vp]),
                "or_solve_kepler": (d, [d, d, vp]),
                "or_true_anomaly": (d, [vp, d]),
                "or_position": (None, [vp, d, vp]),
                "or_position_from_nu": (None, [vp, d, vp]),
                "or_velocity_fd": (None, [vp, d, d, vp]),
                "or_nu_rk4": (d, [vp, d, d]),
                "or_step_ticks": (i64, [vp, i32, i64, d, vp, vp, i32, d]),
                "or_iv_add": (None, [vp, vp, vp]), "or_iv_mul": (None, [vp, vp, vp]),
                "or_iv_scale": (None, [d, vp, vp]),
                "or_iv_cos": (None, [vp, vp]), "or_iv_sin": (None, [vp, vp]),
                "or_box": (None, [vp, i32, i64, i64, d, vp, vp, vp, vp]),
                "or_boxes": (i64, [vp, i64, i64, d, vp, i32, vp, vp, vp, i64]),
                "or_raw_cells_bruteforce": (i64, [vp, vp, vp, i64, vp, i64]),
                "or_raw_cells_sweep": (i64, [vp, vp, vp, i64, vp, i64]),
                "or_raw_cells_sweep_before": (i64, [vp, vp, vp, i64, i64, vp, i64]),
                "or_boxes_starting": (i64, [vp, i64, i64, d, vp, i32, i64, i64, vp, vp, vp, i64]),
                "or_raw_cells_selected": (i64, [vp, vp, vp, i64, vp, vp, i64]),
                "or_canonicalize": (i64, [vp, i64]),
                "or_alg1_witnesses": (i64, [vp, i64, i64, d, vp, i64]),
                "or_alg1_sweep": (i64, [vp, i64, i64, i64, d, vp, vp, i64]),
                "or_raw_cells_tree": (i64, [vp, vp, vp, i64, vp, i64]),
                "or_alg3": (i32, [vp, i64, i64, d, i32, i64, vp, vp, vp, vp]),
                "or_narrow_phase": (i64, [vp, i64, vp, i64, d, vp, vp, vp, vp, i64]),
                "or_refine_discrete": (i64, [vp, i64, i64, d, i32, d, vp, i64, vp, vp, vp]),
                "or_refine_start_ticks": (i64, [vp, i64, d, d]),
                "or_refine_continuous": (i64, [vp, i64, d, d, i32, vp, i64, vp, vp]),
                "or_refine_round": (i64, [vp, vp, vp, i64, i32, vp, vp, vp, i64]),
                "or_radial_range": (None, [vp, vp]),
                "or_band_edges": (None, [vp, i64, i32, vp]),
                "or_band_counts": (None, [vp, i64, i32, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _els(els) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(els, dtype=np.float64))
    if a.ndim == 1:
        a = a.reshape(1, 7)
    assert a.shape[1] == 7
    return a


# --- dynamics (Sec. 6.1, Eq. 1) -------------------------------------------

def mean_motion(el) -> float:
    return lib().or_mean_motion(_p(_els(el)))


def period(el) -> float:
    return lib().or_period(_p(_els(el)))


def max_speed(el) -> float:
    return lib().or_max_speed(_p(_els(el)))


def solve_kepler(M: float, e: float):
    it = ctypes.c_int(0)
    E = lib().or_solve_kepler(M, e, ctypes.byref(it))
    return E, it.value


def true_anomaly(el, t_s: float) -> float:
    return lib().or_true_anomaly(_p(_els(el)), float(t_s))


def position(el, t_s: float) -> np.ndarray:
    out = np.zeros(3)
    lib().or_position(_p(_els(el)), float(t_s), _p(out))
    return out


def position_from_nu(el, nu: float) -> np.ndarray:
    out = np.zeros(3)
    lib().or_position_from_nu(_p(_els(el)), float(nu), _p(out))
    return out


def positions(els, obj_idx, t_s) -> np.ndarray:
    """FP64 positions of objects obj_idx[q] at times t_s[q] (seconds)."""
    E = _els(els)
    obj_idx = np.asarray(obj_idx)
    t_s = np.asarray(t_s, dtype=np.float64)
    out = np.zeros((len(obj_idx), 3))
    L = lib()
    tmp = np.zeros(3)
    for q in range(len(obj_idx)):
        L.or_position(_p(E[int(obj_idx[q])]), float(t_s[q]), _p(tmp))
        out[q] = tmp
    return out


def velocity_fd(el, t_s: float, h_s: float = 1e-3) -> np.ndarray:
    out = np.zeros(3)
    lib().or_velocity_fd(_p(_els(el)), float(t_s), float(h_s), _p(out))
    return out


def nu_rk4(el, t_s: float, h_s: float) -> float:
    return lib().or_nu_rk4(_p(_els(el)), float(t_s), float(h_s))


# --- step policy -----------------------------------------------------------

def step_ticks(els, kind: int, tick_s: float, fixed_ticks: int = 1, frac: float = 100.0,
               band_edges_km=(), band_fracs=(100.0,)) -> np.ndarray:
    E = _els(els)
    be = np.ascontiguousarray(np.asarray(band_edges_km, dtype=np.float64).reshape(-1))
    bf = np.ascontiguousarray(np.asarray(band_fracs, dtype=np.float64).reshape(-1))
    if be.size == 0:
        be = np.zeros(1)
    L = lib()
    return np.array([L.or_step_ticks(_p(E[i]), kind, int(fixed_ticks), float(frac), _p(be), _p(bf),
                                     int(len(bf)), float(tick_s)) for i in range(len(E))],
                    dtype=np.int64)


# --- interval arithmetic (Sec. 4.5) -----------------------------------------

def _iv2(fn, *args):
    out = np.zeros(2)
    keep, conv = [], []  # arrays stay referenced until the call returns
    for a in args:
        if isinstance(a, (list, tuple, np.ndarray)):
            keep.append(np.ascontiguousarray(a, dtype=np.float64))
            conv.append(_p(keep[-1]))
        else:
            conv.append(float(a))
    fn(*conv, _p(out))
    return out


def iv_add(a, b):
    return _iv2(lib().or_iv_add, a, b)


def iv_mul(a, b):
    return _iv2(lib().or_iv_mul, a, b)


def iv_scale(k, a):
    return _iv2(lib().or_iv_scale, k, a)


def iv_cos(x):
    return _iv2(lib().or_iv_cos, x)


def iv_sin(x):
    return _iv2(lib().or_iv_sin, x)


# --- boxes (Defs 7-8) ------------------------------------------------------

def box(el, mode: int, tlo: int, thi: int, tick_s: float):
    lo = np.zeros(4, np.float32)
    hi = np.zeros(4, np.float32)
    c = np.zeros(3)
    hw = np.zeros(1)
    lib().or_box(_p(_els(el)), mode, int(tlo), int(thi), float(tick_s), _p(lo), _p(hi), _p(c), _p(hw))
    return lo, hi, c, float(hw[0])


def boxes(els, T: int, tick_s: float, k, mode: int = BOX_SPEED):
    """All boxes, object-major then segment order: (lo4, hi4, obj)."""
    E = _els(els)
    k = np.ascontiguousarray(np.asarray(k, dtype=np.int64))
    N = int(np.sum((T + 1 + k - 1) // k))
    lo = np.zeros((N, 4), np.float32)
    hi = np.zeros((N, 4), np.float32)
    obj = np.zeros(N, np.uint32)
    got = lib().or_boxes(_p(E), len(E), int(T), float(tick_s), _p(k), mode, _p(lo), _p(hi), _p(obj), N)
    assert got == N
    return lo, hi, obj


def boxes_starting(els, T: int, tick_s: float, k, t0: int, t1: int, mode: int = BOX_SPEED):
    """The boxes of `boxes` whose segments start at a tick in [t0, t1), in
    the same order: whole segments of the horizon [0, T]."""
    E = _els(els)
    k = np.ascontiguousarray(np.asarray(k, dtype=np.int64))
    f = lib().or_boxes_starting
    n = f(_p(E), len(E), int(T), float(tick_s), _p(k), mode, int(t0), int(t1), None, None,
          None, 0)
    lo = np.zeros((n, 4), np.float32)
    hi = np.zeros((n, 4), np.float32)
    obj = np.zeros(n, np.uint32)
    got = f(_p(E), len(E), int(T), float(tick_s), _p(k), mode, int(t0), int(t1), _p(lo), _p(hi),
            _p(obj), n)
    assert got == n
    return lo, hi, obj


# --- pair sets -------------------------------------------------------------

def _cells_call(fn, *args):
    cap = 1 << 16
    while True:
        out = np.zeros(cap, CELL_DTYPE)
        n = fn(*args, _p(out), cap)
        if n <= cap:
            return out[:n].copy()
        cap = int(n)


def raw_cells_bruteforce(lo4, hi4, obj):
    lo4 = np.ascontiguousarray(lo4, np.float32)
    hi4 = np.ascontiguousarray(hi4, np.float32)
    obj = np.ascontiguousarray(obj, np.uint32)
    return _cells_call(lib().or_raw_cells_bruteforce, _p(lo4), _p(hi4), _p(obj), len(obj))


def raw_cells_tree(lo4, hi4, obj):
    """Every overlapping box pair of different objects, through the paper's
    incrementally built AABB tree (Sec. 3.2)."""
    lo4 = np.ascontiguousarray(lo4, np.float32)
    hi4 = np.ascontiguousarray(hi4, np.float32)
    obj = np.ascontiguousarray(obj, np.uint32)
    return _cells_call(lib().or_raw_cells_tree, _p(lo4), _p(hi4), _p(obj), len(obj))


def raw_cells_sweep(lo4, hi4, obj):
    lo4 = np.ascontiguousarray(lo4, np.float32)
    hi4 = np.ascontiguousarray(hi4, np.float32)
    obj = np.ascontiguousarray(obj, np.uint32)
    return _cells_call(lib().or_raw_cells_sweep, _p(lo4), _p(hi4), _p(obj), len(obj))


def raw_cells_sweep_before(lo4, hi4, obj, t_end: int):
    """The sweep's pairs whose earlier box (by lower tick, then index)
    starts before tick t_end."""
    lo4 = np.ascontiguousarray(lo4, np.float32)
    hi4 = np.ascontiguousarray(hi4, np.float32)
    obj = np.ascontiguousarray(obj, np.uint32)
    return _cells_call(lib().or_raw_cells_sweep_before, _p(lo4), _p(hi4), _p(obj), len(obj),
                       int(t_end))


def raw_cells_selected(lo4, hi4, obj, sel):
    lo4 = np.ascontiguousarray(lo4, np.float32)
    hi4 = np.ascontiguousarray(hi4, np.float32)
    obj = np.ascontiguousarray(obj, np.uint32)
    sel = np.ascontiguousarray(sel, np.uint8)
    return _cells_call(lib().or_raw_cells_selected, _p(lo4), _p(hi4), _p(obj), len(obj), _p(sel))


def canonicalize(cells) -> np.ndarray:
    c = np.ascontiguousarray(np.array(cells, dtype=CELL_DTYPE, copy=True))
    n = lib().or_canonicalize(_p(c), len(c))
    return c[:n].copy()


def screen(els, T: int, tick_s: float, k, mode: int = BOX_SPEED):
    """The whole method on the CPU: boxes, every overlapping box pair, then
    the canonical sorted and merged list."""
    lo, hi, obj = boxes(els, T, tick_s, k, mode)
    return canonicalize(raw_cells_sweep(lo, hi, obj))


# --- the paper's algorithms ------------------------------------------------

def alg1_witnesses(els, T: int, tick_s: float) -> np.ndarray:
    E = _els(els)
    return _cells_call_w(lib().or_alg1_witnesses, _p(E), len(E), int(T), float(tick_s))


APPROACH_DTYPE = np.dtype([("i", "<u4"), ("j", "<u4"), ("t", "<i4"), ("dist", "<f8")])


def alg1_sweep(els, t0: int, t1: int, tick_s: float) -> np.ndarray:
    """Alg 1 witnesses on ticks t0..t1 (pairs found by an x sweep, same
    predicate), each with the Euclidean distance of the two centres."""
    E = _els(els)
    cap = 1 << 12
    while True:
        w = np.zeros(cap, WITNESS_DTYPE)
        dist = np.zeros(cap)
        n = lib().or_alg1_sweep(_p(E), len(E), int(t0), int(t1), float(tick_s), _p(w), _p(dist),
                                cap)
        if n <= cap:
            out = np.zeros(n, APPROACH_DTYPE)
            out["i"], out["j"], out["t"], out["dist"] = w["i"][:n], w["j"][:n], w["t"][:n], dist[:n]
            return out
        cap = int(n)


def _alg1_chunk(args):
    els, t0, t1, tick_s = args
    return alg1_sweep(els, t0, t1, tick_s)


def close_approaches(els, T: int, tick_s: float, d_km: float, processes: int = 0) -> np.ndarray:
    """Every (i < j, tick) with the two centres closer than d_km (Euclidean)
    at a tick of 0..T: the Alg 1 witnesses (cube contact, a superset when
    d_km <= r_i + r_j) filtered by distance.  Tick ranges run in a pool of
    processes started with spawn (safe after a GPU context exists)."""
    import multiprocessing as mp
    E = _els(els)
    n_proc = processes or min(32, os.cpu_count() or 1)
    edges = np.linspace(0, T + 1, 4 * n_proc + 1).astype(np.int64)
    jobs = [(E, int(a), int(b) - 1, float(tick_s)) for a, b in zip(edges[:-1], edges[1:]) if b > a]
    if n_proc > 1 and len(jobs) > 1:
        with mp.get_context("spawn").Pool(n_proc) as pool:
            parts = pool.map(_alg1_chunk, jobs)
    else:
        parts = [_alg1_chunk(j) for j in jobs]
    w = np.concatenate(parts) if parts else np.zeros(0, APPROACH_DTYPE)
    return w[w["dist"] < d_km]


def _cells_call_w(fn, *args):
    cap = 1 << 12
    while True:
        out = np.zeros(cap, WITNESS_DTYPE)
        n = fn(*args, _p(out), cap)
        if n <= cap:
            return out[:n].copy()
        cap = int(n)


def alg3(els, T: int, tick_s: float, mode: int = BOX_SPEED, t_first: int = -1):
    """Serial Alg 3.  Returns (rc, (i, j, t) or None, iterations)."""
    E = _els(els)
    wi, wj = ctypes.c_uint32(0), ctypes.c_uint32(0)
    wt, it = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib().or_alg3(_p(E), len(E), int(T), float(tick_s), mode, int(t_first), ctypes.byref(wi),
                       ctypes.byref(wj), ctypes.byref(wt), ctypes.byref(it))
    w = (wi.value, wj.value, wt.value) if rc == 1 else None
    return rc, w, it.value


def narrow_phase(els, cands, tick_s: float, witnesses: bool = True):
    """Narrow phase over a candidate list (CELL_DTYPE rows i < j, [tlo, thi]):
    every tick of every candidate interval tested with Alg 1's predicate
    (Defs 2-4).  Returns (first, count, margin, witness list): per candidate
    the first witness tick (-1: none), the number of witness ticks and the
    smallest |d_inf - (r_i + r_j)| over its ticks; the witnesses in
    candidate order (empty if witnesses is False)."""
    E = _els(els)
    C = np.ascontiguousarray(np.asarray(cands, dtype=CELL_DTYPE))
    m = len(C)
    first = np.zeros(m, np.int32)
    count = np.zeros(m, np.uint32)
    margin = np.zeros(m, np.float64)
    cap = 1 << 12 if witnesses else 0
    while True:
        out = np.zeros(max(cap, 1), WITNESS_DTYPE)
        k = lib().or_narrow_phase(_p(E), len(E), _p(C), m, float(tick_s), _p(first), _p(count),
                                  _p(margin), _p(out) if witnesses else None, cap)
        if k < 0:
            raise ValueError("candidate with an object index >= n or an empty tick interval")
        if not witnesses or k <= cap:
            return first, count, margin, out[:min(k, cap)].copy()
        cap = int(k)


def earliest_witness(wit):
    """The first witness in Alg 1's order (tick, then i, then j) of a witness
    list, or None."""
    if len(wit) == 0:
        return None
    o = np.lexsort((wit["j"], wit["i"], wit["t"]))[0]
    return int(wit["i"][o]), int(wit["j"][o]), int(wit["t"][o])


SPAN_DTYPE = np.dtype([("i", "<u4"), ("j", "<u4"), ("t0", "<f8"), ("t1", "<f8")])


def refine_start_ticks(el, T: int, tick_s: float, fraction: float) -> int:
    """First-interval length (ticks) for the start fraction f: the largest
    power of two not above max(1, floor(P / (f tick_s))), or T + 1 when
    longer or f = 0."""
    return int(lib().or_refine_start_ticks(_p(_els([el])), int(T), float(tick_s),
                                           float(fraction)))


def refine_discrete(els, T: int, tick_s: float, mode: int = BOX_SPEED,
                    start_fraction: float = 0.0):
    """Adaptive refinement in bulk-synchronous rounds (Alg 5-6 taken top-down
    over all objects, each starting from [0, T] (start_fraction 0) or from
    intervals of refine_start_ticks): returns (witnesses in Alg 1's order, active
    intervals per round, distinct tick candidates)."""
    E = _els(els)
    rb = np.zeros(64, np.int64)
    rounds = ctypes.c_int(0)
    ntc = ctypes.c_int64(0)
    cap = 1 << 12
    while True:
        out = np.zeros(cap, WITNESS_DTYPE)
        k = lib().or_refine_discrete(_p(E), len(E), int(T), float(tick_s), int(mode),
                                     float(start_fraction), _p(out), cap,
                                     _p(rb), ctypes.byref(rounds), ctypes.byref(ntc))
        if k <= cap:
            return out[:k].copy(), rb[:rounds.value].copy(), int(ntc.value)
        cap = int(k)


def refine_continuous(els, T_s: float, eps_s: float, mode: int = BOX_SPEED):
    """The continuous-time variant (Sec. 4.6): returns (spans (i, j, t0, t1)
    at resolution eps_s, active intervals per round)."""
    E = _els(els)
    rb = np.zeros(64, np.int64)
    rounds = ctypes.c_int(0)
    cap = 1 << 12
    while True:
        out = np.zeros(cap, SPAN_DTYPE)
        k = lib().or_refine_continuous(_p(E), len(E), float(T_s), float(eps_s), int(mode),
                                       _p(out), cap, _p(rb), ctypes.byref(rounds))
        if k <= cap:
            return out[:k].copy(), rb[:rounds.value].copy()
        cap = int(k)


# --- decomposition (Sec. 5, Sec. 6.1) ----------------------------------------

def radial_range(el) -> np.ndarray:
    out = np.zeros(2)
    lib().or_radial_range(_p(_els(el)), _p(out))
    return out


def band_edges(els, p: int) -> np.ndarray:
    E = _els(els)
    out = np.zeros(max(p - 1, 1))
    lib().or_band_edges(_p(E), len(E), int(p), _p(out))
    return out[:p - 1]


def band_counts(els, p: int) -> np.ndarray:
    E = _els(els)
    out = np.zeros(p, np.int64)
    lib().or_band_counts(_p(E), len(E), int(p), _p(out))
    return out


def potential_collision_filter(els, cells) -> np.ndarray:
    """Keep the cells whose objects share an edge of the potential-collision
    graph (Def 9): padded radial ranges that intersect."""
    E = _els(els)
    rr = np.array([radial_range(E[i]) for i in range(len(E))])
    i = cells["i"].astype(np.int64)
    j = cells["j"].astype(np.int64)
    keep = np.maximum(rr[i, 0], rr[j, 0]) <= np.minimum(rr[i, 1], rr[j, 1])
    return cells[keep]


def refine_round(lo4, hi4, obj, cont: bool = False) -> np.ndarray:
    """One refinement round on the given FP32 boxes (first and last unit of
    each interval in the w lane): the next round's intervals as an (m, 3)
    int64 array of (object, t0, t1), in input order."""
    lo4 = np.ascontiguousarray(lo4, np.float32)
    hi4 = np.ascontiguousarray(hi4, np.float32)
    obj = np.ascontiguousarray(obj, np.uint32)
    m = len(obj)
    cap = 2 * m + 1
    nobj = np.zeros(cap, np.uint32)
    nt0 = np.zeros(cap, np.int32)
    nt1 = np.zeros(cap, np.int32)
    k = lib().or_refine_round(_p(lo4), _p(hi4), _p(obj), m, int(cont), _p(nobj), _p(nt0),
                              _p(nt1), cap)
    return np.stack([nobj[:k].astype(np.int64), nt0[:k], nt1[:k]], 1)

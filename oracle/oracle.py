"""ctypes wrapper around the FP64 oracle in ``oracle.cpp`` (test infrastructure only).

The oracle is built with plain g++ (no CUDA) and shares no code with the CUDA
sources.  Functions take numpy arrays and return numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (g++, -O2, IEEE-exact: no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-ffp-contract=off",
               _SRC, "-o", _LIB + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Surface(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32),
                ("px", C.c_void_p), ("py", C.c_void_p), ("pz", C.c_void_p),
                ("nx", C.c_void_p), ("ny", C.c_void_p), ("nz", C.c_void_p),
                ("i0", C.c_void_p), ("i1", C.c_void_p), ("i2", C.c_void_p),
                ("kind", C.c_int32), ("eta", C.c_float)]


class Receiver(C.Structure):
    _fields_ = [("p0", C.c_float * 3), ("e1", C.c_float * 3), ("e2", C.c_float * 3)]


class Emitters(C.Structure):
    _fields_ = [("n", C.c_int32), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("intensity", C.c_void_p)]


class Record(C.Structure):
    _fields_ = [("emitter", C.c_int32), ("tri0", C.c_int32), ("tri1", C.c_int32),
                ("cell", C.c_uint32), ("flags", C.c_uint32), ("pad", C.c_int32),
                ("u_lo", C.c_double), ("u_hi", C.c_double), ("v_lo", C.c_double), ("v_hi", C.c_double),
                ("e_lo", C.c_double), ("e_hi", C.c_double), ("q_cond", C.c_double), ("m_cond", C.c_double)]


RECORD_DTYPE = np.dtype([("emitter", np.int32), ("tri0", np.int32), ("tri1", np.int32),
                         ("cell", np.uint32), ("flags", np.uint32), ("pad", np.int32),
                         ("u_lo", np.float64), ("u_hi", np.float64), ("v_lo", np.float64),
                         ("v_hi", np.float64), ("e_lo", np.float64), ("e_hi", np.float64),
                         ("q_cond", np.float64), ("m_cond", np.float64)])
assert RECORD_DTYPE.itemsize == C.sizeof(Record)

# Cell flags (the documented interface values; the CUDA path uses the same numbers).
LIVE, SPLIT, CULL_BEHIND, CULL_EMPTY, FOLD, POS_UNBOUNDED, QSIGN_FP64, TIR = 1, 2, 4, 8, 16, 32, 64, 128
DEPTH_SHIFT = 24


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            vp, i32, i64, u64, f32, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float, C.c_double
            L.orc_bb_size.restype = C.c_int
            L.orc_bb_eval.restype = f64
            L.orc_philox_uniform.restype = f32
            L.orc_philox_uniform.argtypes = [u64, i64, u64]
            L.orc_bound.argtypes = [vp, vp, vp, i32, i32, i32, vp, i64, vp, i64, vp, i32, i32, f32, f32]
            L.orc_index.argtypes = [vp] * 9 + [i64, i32, f32, vp, vp, vp, i64, vp]
            L.orc_sample.argtypes = [vp, vp, vp, i32, vp, vp, i64, f32, u64, vp, vp, vp, i64, vp, vp, i32, vp]
            L.orc_solve.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp, vp, i32, i32, f64, vp, vp, vp, vp, i32, i32, u64,
                                    vp]
            L.orc_roots.argtypes = [vp, vp, vp, i32, i32, f64, f64, i32, i32, i32, f64, vp, vp]
            L.orc_eval_path.argtypes = [vp, vp, vp, i32, i32, vp, vp, i64, vp, vp, vp, vp]
            L.orc_eval_direct.argtypes = [vp, vp, vp, i32, i32, vp, vp, i64, vp, vp, vp, vp]
            L.orc_bb_mul.argtypes = [C.c_int, C.c_int, vp, C.c_int, vp, vp]
            L.orc_bb_elevate.argtypes = [C.c_int, C.c_int, vp, vp]
            L.orc_bb_deriv.argtypes = [C.c_int, vp, C.c_int, vp]
            L.orc_bb_eval.argtypes = [C.c_int, C.c_int, vp, f64, f64]
            L.orc_chord_inv32.argtypes = [f64, f64, vp]
            L.orc_chord_sqrt.argtypes = [f64, f64, vp]
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_cell_corners.argtypes = [C.c_uint32, C.c_int, vp]
            L.orc_pair_candidates.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, i64, vp, i32]
            L.orc_pair_gap.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, i64, vp]
            L.orc_bound_pairs.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, i64, vp, i32]
            L.orc_bound_pairs_diag.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, i64, vp, vp]
            L.orc_pair_diag_size.restype = i32
            L.orc_chain_irradiance.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, i64, vp, vp, i32]
            L.orc_chain_box.argtypes = [vp, vp, vp, vp, i32, i32, i32, f64, f64, f64, f64, vp]
            L.orc_eval_pair.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp, vp, i64, vp]
            L.orc_solve_pair.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, i32, i32, f64, vp, vp, vp, vp, i32]
            L.orc_implicit_bound.argtypes = [vp, vp, vp, i64] + [vp] * 10 + [i32, i32]
            L.orc_implicit_eval.argtypes = [vp, vp, vp, i32, i32, C.c_uint32, i32, f64, f64, f64, f64, i32, i64,
                                            vp, vp, vp, vp, vp]
            L.orc_implicit_bound_pairs.argtypes = [vp, vp, vp, vp, i64] + [vp] * 11 + [i32, i32]
            L.orc_implicit_eval_pair.argtypes = [vp, vp, vp, vp, i32, i32, C.c_uint32, i32, i32, f64, f64, f64, f64,
                                                 i32, i64, vp, vp, vp, vp, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


class _SceneViews:
    """Keeps the contiguous arrays alive while ctypes structs point at them."""

    def __init__(self, scene):
        self.keep = []

        def c(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self.keep.append(a)
            return _p(a)

        def surface(s):
            return Surface(s.n_verts, s.n_tris, c(s.px, np.float32), c(s.py, np.float32), c(s.pz, np.float32),
                           c(s.nx, np.float32), c(s.ny, np.float32), c(s.nz, np.float32),
                           c(s.i0, np.int32), c(s.i1, np.int32), c(s.i2, np.int32), s.kind, s.eta)

        self.surf = surface(scene.s1)
        self.surf2 = surface(scene.s2) if scene.s2 is not None else None
        r = scene.receiver
        self.rec = Receiver((C.c_float * 3)(*r.p0), (C.c_float * 3)(*r.e1), (C.c_float * 3)(*r.e2))
        e = scene.emitters
        self.em = Emitters(e.n, c(e.x, np.float32), c(e.y, np.float32), c(e.z, np.float32),
                           c(e.intensity, np.float32))


# ------------------------------------------------------------------ Bernstein helpers
def bb_mul(dim: int, m: int, p, n: int, q) -> np.ndarray:
    L = lib()
    p = np.ascontiguousarray(p, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    out = np.zeros(L.orc_bb_size(dim, m + n))
    L.orc_bb_mul(dim, m, _p(p), n, _p(q), _p(out))
    return out


def bb_elevate(dim: int, n: int, p) -> np.ndarray:
    L = lib()
    p = np.ascontiguousarray(p, np.float64)
    out = np.zeros(L.orc_bb_size(dim, n + 1))
    L.orc_bb_elevate(dim, n, _p(p), _p(out))
    return out


def bb_deriv(n: int, p, j: int) -> np.ndarray:
    L = lib()
    p = np.ascontiguousarray(p, np.float64)
    out = np.zeros(L.orc_bb_size(2, n - 1))
    L.orc_bb_deriv(n, _p(p), j, _p(out))
    return out


def bb_eval(dim: int, n: int, p, m1: float, m2: float = 0.0) -> float:
    p = np.ascontiguousarray(p, np.float64)
    return lib().orc_bb_eval(dim, n, _p(p), m1, m2)


def bb_index(n: int):
    """(g0, g1, g2) multi-indices in coefficient order for the 2-simplex."""
    out = []
    for g1 in range(n + 1):
        for g2 in range(n - g1 + 1):
            out.append((n - g1 - g2, g1, g2))
    return out


def chord_inv32(s_lo: float, s_hi: float):
    out = np.zeros(4)
    lib().orc_chord_inv32(s_lo, s_hi, _p(out))
    return tuple(out)


def chord_sqrt(lo: float, hi: float):
    """Chord a*beta + b of sqrt on [lo, hi] and the range [dlo, dhi] of sqrt - chord."""
    out = np.zeros(4)
    lib().orc_chord_sqrt(lo, hi, _p(out))
    return tuple(out)


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def philox_uniform(seed: int, point: int, key: int) -> float:
    return lib().orc_philox_uniform(seed, point, key)


def cell_corners(cell_id: int, depth: int) -> np.ndarray:
    out = np.zeros(6)
    lib().orc_cell_corners(cell_id, depth, _p(out))
    return out.reshape(3, 2)


# ------------------------------------------------------------------ pipeline stages
def bound(scene, depth: Optional[int] = None, max_extra_split: int = 4, irradiance: bool = True,
          work: Optional[np.ndarray] = None, n_threads: int = 1, adapt_depth: int = 0, sigma: float = 0.0,
          alpha: float = 0.0) -> np.ndarray:
    """Cell records (structured array, RECORD_DTYPE) for all base cells or the given work items.
    adapt_depth > depth: adaptive subdivision (Sec. 6.1) down to adapt_depth, stopping at box area
    < sigma or E_hi < alpha E_lo."""
    L = lib()
    V = _SceneViews(scene)
    d = scene.depth if depth is None else depth
    if work is not None:
        work = np.ascontiguousarray(work, np.int64)
        n_work = work.shape[0]
        wp = _p(work)
    else:
        n_work, wp = 0, None
    cap = max(16, (n_work if work is not None else scene.emitters.n * scene.s1.n_tris * 4 ** d) * 2)
    while True:
        out = np.zeros(cap, RECORD_DTYPE)
        n_out = np.zeros(1, np.int64)
        rc = L.orc_bound(C.byref(V.surf), C.byref(V.rec), C.byref(V.em), d, max_extra_split, int(irradiance),
                         wp, n_work, _p(out), cap, _p(n_out), n_threads, adapt_depth, sigma, alpha)
        if rc == -2:
            cap = int(n_out[0])
            continue
        if rc != 0:
            raise RuntimeError(f"orc_bound failed: {rc}")
        return out[: int(n_out[0])]


def records_to_f32(rec: np.ndarray):
    """Round the oracle's float64 boxes outward to float32 (lo down, hi up)."""
    def down(x):
        f = x.astype(np.float32)
        bad = f.astype(np.float64) > x
        f[bad] = np.nextafter(f[bad], np.float32(-np.inf))
        return f

    def up(x):
        f = x.astype(np.float32)
        bad = f.astype(np.float64) < x
        f[bad] = np.nextafter(f[bad], np.float32(np.inf))
        return f

    return dict(u_lo=down(rec["u_lo"]), u_hi=up(rec["u_hi"]), v_lo=down(rec["v_lo"]), v_hi=up(rec["v_hi"]),
                e_lo=down(rec["e_lo"]), e_hi=up(rec["e_hi"]), emitter=rec["emitter"].astype(np.int32),
                tri0=rec["tri0"].astype(np.int32), tri1=rec["tri1"].astype(np.int32),
                flags=rec["flags"].astype(np.uint32))


def index(u_lo, u_hi, v_lo, v_hi, e_hi, emitter, tri0, tri1, flags, grid_res: int = 512, m: float = 1.0):
    """CSR (offsets[G*G+1], key u64, etilde f32) sorted by key within each grid cell."""
    L = lib()
    arrs = [np.ascontiguousarray(a, dt) for a, dt in
            [(u_lo, np.float32), (u_hi, np.float32), (v_lo, np.float32), (v_hi, np.float32), (e_hi, np.float32),
             (emitter, np.int32), (tri0, np.int32), (tri1, np.int32), (flags, np.uint32)]]
    n = arrs[0].shape[0]
    G = grid_res
    offsets = np.zeros(G * G + 1, np.int64)
    cap = max(16, 4 * n)
    while True:
        key = np.zeros(cap, np.uint64)
        et = np.zeros(cap, np.float32)
        n_out = np.zeros(1, np.int64)
        rc = L.orc_index(*[_p(a) for a in arrs], n, G, m, _p(offsets), _p(key), _p(et), cap, _p(n_out))
        if rc == -2:
            cap = int(n_out[0])
            continue
        return offsets, key[: int(n_out[0])], et[: int(n_out[0])]


def sample(offsets, key, etilde, grid_res: int, su, sv, gamma: float, seed: int, bins: bool = False,
           with_bins: bool = False):
    """Worklist (point, key, P) in (point, key) order, and |U| summed over points.  bins: the
    bin-packed selection (one draw per bin of Sec. 5.3) instead of one draw per tuple; with_bins
    also returns |B| summed over points."""
    L = lib()
    offsets = np.ascontiguousarray(offsets, np.int64)
    key = np.ascontiguousarray(key, np.uint64)
    etilde = np.ascontiguousarray(etilde, np.float32)
    su = np.ascontiguousarray(su, np.float32)
    sv = np.ascontiguousarray(sv, np.float32)
    cap = max(16, key.shape[0])
    while True:
        wp = np.zeros(cap, np.int64)
        wk = np.zeros(cap, np.uint64)
        wP = np.zeros(cap, np.float32)
        n_out = np.zeros(1, np.int64)
        n_u = np.zeros(1, np.int64)
        n_b = np.zeros(1, np.int64)
        rc = L.orc_sample(_p(offsets), _p(key), _p(etilde), grid_res, _p(su), _p(sv), su.shape[0], gamma, seed,
                          _p(wp), _p(wk), _p(wP), cap, _p(n_out), _p(n_u), int(bins), _p(n_b))
        if rc == -2:
            cap = int(n_out[0])
            continue
        k = int(n_out[0])
        if with_bins:
            return wp[:k], wk[:k], wP[:k], int(n_u[0]), int(n_b[0])
        return wp[:k], wk[:k], wP[:k], int(n_u[0])


def solve(scene, wl_point, wl_key, wl_p, newton_iters: int = 16, polish_iters: int = 1, tol: float = 1e-5,
          n_threads: int = 1, stoc_trials: int = 0, seed: int = 0, with_trials: bool = False):
    """Per worklist entry: contribution E/P (float64), root (u, v) and status (1 = root).
    stoc_trials > 0: stochastic starts with the reciprocal weighting (Sec. 6.1 "Stoc"), capped at
    stoc_trials; with_trials also returns the weight N of each entry."""
    L = lib()
    V = _SceneViews(scene)
    wl_point = np.ascontiguousarray(wl_point, np.int64)
    wl_key = np.ascontiguousarray(wl_key, np.uint64)
    wl_p = np.ascontiguousarray(wl_p, np.float32)
    su = np.ascontiguousarray(scene.su, np.float32)
    sv = np.ascontiguousarray(scene.sv, np.float32)
    n = wl_point.shape[0]
    contrib = np.zeros(n)
    ru = np.zeros(n)
    rv = np.zeros(n)
    st = np.zeros(n, np.int32)
    tr = np.zeros(n, np.int32)
    L.orc_solve(C.byref(V.surf), C.byref(V.rec), C.byref(V.em), _p(wl_point), _p(wl_key), _p(wl_p), n, _p(su),
                _p(sv), newton_iters, polish_iters, tol, _p(contrib), _p(ru), _p(rv), _p(st), n_threads,
                stoc_trials, seed, _p(tr))
    if with_trials:
        return contrib, ru, rv, st, tr
    return contrib, ru, rv, st


def roots(scene, emitter: int, tri: int, tu: float, tv: float, n: int = 24, newton_iters: int = 16,
          polish_iters: int = 1, tol: float = 1e-5):
    """Sum of E over every distinct root of one tuple at one target (Newton from an n x n grid of
    starts), and the number of roots."""
    L = lib()
    V = _SceneViews(scene)
    s = np.zeros(1)
    k = np.zeros(1, np.int32)
    L.orc_roots(C.byref(V.surf), C.byref(V.rec), C.byref(V.em), emitter, tri, tu, tv, n, newton_iters, polish_iters,
                tol, _p(s), _p(k))
    return float(s[0]), int(k[0])


def accumulate(n_points: int, wl_point, contrib) -> np.ndarray:
    """Per-point estimate: sum of contributions (worklist in point order), float64."""
    E = np.zeros(n_points)
    np.add.at(E, np.asarray(wl_point, np.int64), contrib)
    return E


def eval_path(scene, emitter: int, tri: int, u, v, direct: bool = False):
    L = lib()
    V = _SceneViews(scene)
    u = np.ascontiguousarray(u, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    n = u.shape[0]
    uk, vk, E, t = (np.zeros(n) for _ in range(4))
    fn = L.orc_eval_direct if direct else L.orc_eval_path
    fn(C.byref(V.surf), C.byref(V.rec), C.byref(V.em), emitter, tri, _p(u), _p(v), n, _p(uk), _p(vk), _p(E), _p(t))
    return uk, vk, E, t


def implicit_bound(scene, emitter, tri0, cell, depth, u_lo, u_hi, v_lo, v_hi, n_threads: int = 1, b_mask: int = 3):
    """Implicit-differentiation irradiance bounds (Sec. 4.4) of single-refraction records given by
    (emitter, tri0, cell id, depth, position box): (e_lo, e_hi) float64 arrays.  b_mask: 1 = b
    (1,0,0) only, 2 = (0,1,0) only, 3 = the tighter of both."""
    L = lib()
    V = _SceneViews(scene)
    a = [np.ascontiguousarray(x, dt) for x, dt in [(emitter, np.int32), (tri0, np.int32), (cell, np.uint32),
                                                   (depth, np.int32), (u_lo, np.float64), (u_hi, np.float64),
                                                   (v_lo, np.float64), (v_hi, np.float64)]]
    n = a[0].shape[0]
    lo, hi = np.zeros(n), np.zeros(n)
    rc = L.orc_implicit_bound(C.byref(V.surf), C.byref(V.rec), C.byref(V.em), n, *[_p(x) for x in a], _p(lo),
                              _p(hi), n_threads, b_mask)
    if rc != 0:
        raise RuntimeError(f"orc_implicit_bound failed: {rc}")
    return lo, hi


def implicit_eval(scene, emitter: int, tri0: int, cell: int, depth: int, box, which_b: int, l1, l2, s, t) -> dict:
    """The implicit forms F, G, det A, det B and |d0|^2 of one record at cell barycentrics (l1, l2)
    and box coordinates (s, t) in [0, 1]^2, for b = (1,0,0) (which_b 0) or (0,1,0) (1)."""
    L = lib()
    V = _SceneViews(scene)
    l1, l2, s, t = (np.ascontiguousarray(x, np.float64) for x in (l1, l2, s, t))
    n = l1.shape[0]
    out = np.zeros((n, 5))
    rc = L.orc_implicit_eval(C.byref(V.surf), C.byref(V.rec), C.byref(V.em), emitter, tri0, cell, depth, *map(float, box),
                             which_b, n, _p(l1), _p(l2), _p(s), _p(t), _p(out))
    if rc != 0:
        raise RuntimeError(f"orc_implicit_eval failed: {rc}")
    return dict(F=out[:, 0], G=out[:, 1], detA=out[:, 2], detB=out[:, 3], L0=out[:, 4])


def implicit_bound_pairs(scene, emitter, tri0, cell, depth, tri1, u_lo, u_hi, v_lo, v_hi, n_threads: int = 1,
                         b_mask: int = 3):
    """Implicit-differentiation irradiance bounds (Sec. 4.4) of chain records whose first vertex
    reflects: (e_lo, e_hi) float64 arrays.  b_mask as in implicit_bound."""
    L = lib()
    V = _SceneViews(scene)
    a = [np.ascontiguousarray(x, dt) for x, dt in [(emitter, np.int32), (tri0, np.int32), (cell, np.uint32),
                                                   (depth, np.int32), (tri1, np.int32), (u_lo, np.float64),
                                                   (u_hi, np.float64), (v_lo, np.float64), (v_hi, np.float64)]]
    n = a[0].shape[0]
    lo, hi = np.zeros(n), np.zeros(n)
    rc = L.orc_implicit_bound_pairs(C.byref(V.surf), C.byref(V.surf2), C.byref(V.rec), C.byref(V.em), n,
                                    *[_p(x) for x in a], _p(lo), _p(hi), n_threads, b_mask)
    if rc != 0:
        raise RuntimeError(f"orc_implicit_bound_pairs failed: {rc}")
    return lo, hi


def implicit_eval_pair(scene, emitter: int, tri0: int, cell: int, depth: int, tri1: int, box, which_b: int, l1, l2,
                       s, t) -> dict:
    """The chain forms F~, G~ and the implicit irradiance of one reflecting-first chain record at
    cell barycentrics (l1, l2) and box coordinates (s, t)."""
    L = lib()
    V = _SceneViews(scene)
    l1, l2, s, t = (np.ascontiguousarray(x, np.float64) for x in (l1, l2, s, t))
    n = l1.shape[0]
    out = np.zeros((n, 3))
    rc = L.orc_implicit_eval_pair(C.byref(V.surf), C.byref(V.surf2), C.byref(V.rec), C.byref(V.em), emitter, tri0,
                                  cell, depth, tri1, *map(float, box), which_b, n, _p(l1), _p(l2), _p(s), _p(t),
                                  _p(out))
    if rc != 0:
        raise RuntimeError(f"orc_implicit_eval_pair failed: {rc}")
    return dict(F=out[:, 0], G=out[:, 1], E=out[:, 2])


def tuple_key(emitter, tri0, tri1=-1):
    return (np.uint64(emitter) << np.uint64(48)) | (np.uint64(tri1 + 1) << np.uint64(24)) | np.uint64(tri0)


def render(scene, gamma: float, seed: int, depth: Optional[int] = None, max_extra_split: int = 4,
           newton_iters: int = 16, polish_iters: int = 1, tol: float = 1e-5, n_threads: int = 1,
           bins: bool = False):
    """Whole path on the CPU: bound -> index -> Algorithm 1 (or its bin-packed form) -> Newton ->
    per-point estimate."""
    rec = bound(scene, depth=depth, max_extra_split=max_extra_split, n_threads=n_threads)
    f = records_to_f32(rec)
    off, key, et = index(f["u_lo"], f["u_hi"], f["v_lo"], f["v_hi"], f["e_hi"], f["emitter"], f["tri0"],
                         f["tri1"], f["flags"], scene.grid_res)
    wp, wk, wP, n_u = sample(off, key, et, scene.grid_res, scene.su, scene.sv, gamma, seed, bins=bins)
    contrib, ru, rv, st = solve(scene, wp, wk, wP, newton_iters, polish_iters, tol, n_threads)
    E = accumulate(scene.su.shape[0], wp, contrib)
    return dict(records=rec, offsets=off, key=key, etilde=et, wl_point=wp, wl_key=wk, wl_p=wP, n_U=n_u,
                contrib=contrib, root_u=ru, root_v=rv, status=st, E=E)


# ------------------------------------------------------------------ two specular vertices (pairs)
def pair_candidates(scene, depth: Optional[int] = None, n_threads: int = 1):
    """(emitter, tri0, cell, tri1) items whose footprint meets T2 (brute force over every T2)."""
    L = lib()
    V = _SceneViews(scene)
    d = scene.depth if depth is None else depth
    cap = max(1024, scene.emitters.n * scene.s1.n_tris * 4 ** d * 4)
    while True:
        e, t1, t2 = (np.zeros(cap, np.int32) for _ in range(3))
        cell = np.zeros(cap, np.uint32)
        n_out = np.zeros(1, np.int64)
        rc = L.orc_pair_candidates(C.byref(V.surf), C.byref(V.surf2), C.byref(V.em), d, _p(e), _p(t1), _p(cell),
                                   _p(t2), cap, _p(n_out), n_threads)
        if rc == -2:
            cap = int(n_out[0])
            continue
        if rc != 0:
            raise RuntimeError(f"orc_pair_candidates failed: {rc}")
        n = int(n_out[0])
        return e[:n], t1[:n], cell[:n], t2[:n]


def pair_gap(scene, e, t1, cell, t2, depth: Optional[int] = None):
    """Distance by which T2's xy box misses the cell's footprint (<= 0: candidate)."""
    L = lib()
    V = _SceneViews(scene)
    d = scene.depth if depth is None else depth
    arr = [np.ascontiguousarray(a, dt) for a, dt in ((e, np.int32), (t1, np.int32), (cell, np.uint32), (t2, np.int32))]
    gap = np.zeros(arr[0].shape[0])
    L.orc_pair_gap(C.byref(V.surf), C.byref(V.surf2), C.byref(V.em), d, *[_p(a) for a in arr], arr[0].shape[0],
                   _p(gap))
    return gap


def bound_pairs(scene, e, t1, cell, t2, depth: Optional[int] = None, n_threads: int = 1) -> np.ndarray:
    """Records (RECORD_DTYPE) of the given pair items."""
    L = lib()
    V = _SceneViews(scene)
    d = scene.depth if depth is None else depth
    arr = [np.ascontiguousarray(a, dt) for a, dt in ((e, np.int32), (t1, np.int32), (cell, np.uint32), (t2, np.int32))]
    n = arr[0].shape[0]
    out = np.zeros(n, RECORD_DTYPE)
    rc = L.orc_bound_pairs(C.byref(V.surf), C.byref(V.surf2), C.byref(V.rec), C.byref(V.em), d,
                           *[_p(a) for a in arr], n, _p(out), n_threads)
    if rc != 0:
        raise RuntimeError(f"orc_bound_pairs failed: {rc}")
    return out


# Intermediate quantities of a pair record (the oracle's PairDiag): the chord of sqrt(beta) at each
# vertex (a, b, delta_lo, delta_hi), the direction-ratio bounds of tuple construction, the u2 box,
# the degree-1 interpolant of u2 at the cell corners and its remainder ranges, the receiver forms'
# expansion point, and how far the record's computation got (stage 3: complete).
PAIR_DIAG_DTYPE = np.dtype([("chord1", np.float64, 4), ("rx", np.float64, 2), ("ry", np.float64, 2),
                            ("u2box", np.float64, 4), ("lu", np.float64, 3), ("lv", np.float64, 3),
                            ("rho", np.float64, 4), ("chord2", np.float64, 4), ("uc", np.float64),
                            ("vc", np.float64), ("stage", np.int32), ("pad", np.int32)])


def bound_pairs_diag(scene, e, t1, cell, t2, depth: Optional[int] = None):
    """Records (RECORD_DTYPE) of the given pair items and their intermediates (PAIR_DIAG_DTYPE)."""
    L = lib()
    assert PAIR_DIAG_DTYPE.itemsize == L.orc_pair_diag_size()
    V = _SceneViews(scene)
    d = scene.depth if depth is None else depth
    arr = [np.ascontiguousarray(a, dt) for a, dt in ((e, np.int32), (t1, np.int32), (cell, np.uint32), (t2, np.int32))]
    n = arr[0].shape[0]
    out = np.zeros(n, RECORD_DTYPE)
    diag = np.zeros(n, PAIR_DIAG_DTYPE)
    rc = L.orc_bound_pairs_diag(C.byref(V.surf), C.byref(V.surf2), C.byref(V.rec), C.byref(V.em), d,
                                *[_p(a) for a in arr], n, _p(out), _p(diag))
    if rc != 0:
        raise RuntimeError(f"orc_bound_pairs_diag failed: {rc}")
    return out, diag


def chain_irradiance(scene, e, t1, cell, t2, depth: Optional[int] = None, n_threads: int = 1):
    """Irradiance bounds (e_lo, e_hi) of the given pair items: the chain map in interval arithmetic
    with forward-mode derivatives over the cell (e_hi = +inf when not certified)."""
    L = lib()
    V = _SceneViews(scene)
    d = scene.depth if depth is None else depth
    arr = [np.ascontiguousarray(a, dt) for a, dt in ((e, np.int32), (t1, np.int32), (cell, np.uint32), (t2, np.int32))]
    n = arr[0].shape[0]
    lo, hi = np.zeros(n), np.zeros(n)
    rc = L.orc_chain_irradiance(C.byref(V.surf), C.byref(V.surf2), C.byref(V.rec), C.byref(V.em), d,
                                *[_p(a) for a in arr], n, _p(lo), _p(hi), n_threads)
    if rc != 0:
        raise RuntimeError(f"orc_chain_irradiance failed: {rc}")
    return lo, hi


def chain_box(scene, emitter: int, tri0: int, tri1: int, u0: float, u1: float, v0: float, v1: float) -> dict:
    """One box of the chain irradiance bound with its factors: rc (0 certified, 1 no chain, 2 not
    certified), the intervals of s = |x1 - x0|^2 and det du_k/du1 over the box, and [e_lo, e_hi]."""
    L = lib()
    V = _SceneViews(scene)
    out = np.zeros(7)
    L.orc_chain_box(C.byref(V.surf), C.byref(V.surf2), C.byref(V.rec), C.byref(V.em), emitter, tri0, tri1, u0, u1,
                    v0, v1, _p(out))
    return dict(rc=int(out[0]), s=(out[1], out[2]), det=(out[3], out[4]), e_lo=out[5], e_hi=out[6])


def bound_pair_scene(scene, depth: Optional[int] = None, n_threads: int = 1,
                     irradiance: bool = False) -> np.ndarray:
    """Candidates then their records, in candidate order.  irradiance: live records receive the chain
    irradiance bounds (chain_irradiance); otherwise e_hi = +inf (P = 1 in Algorithm 1)."""
    e, t1, cell, t2 = pair_candidates(scene, depth, n_threads)
    rec = bound_pairs(scene, e, t1, cell, t2, depth, n_threads)
    if irradiance and rec.shape[0]:
        live = (rec["flags"] & LIVE) != 0
        lo, hi = chain_irradiance(scene, rec["emitter"][live], rec["tri0"][live], rec["cell"][live],
                                  rec["tri1"][live], depth, n_threads)
        rec["e_lo"][live] = lo
        rec["e_hi"][live] = hi
    return rec


def eval_pair(scene, emitter: int, tri0: int, tri1: int, u, v) -> dict:
    """Direct chain evaluation: uk, vk, E, u2, v2, t1, t2, detJ per (u1, v1) (NaN: no refracted path)."""
    L = lib()
    V = _SceneViews(scene)
    u = np.ascontiguousarray(u, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    out = np.zeros((u.shape[0], 8))
    L.orc_eval_pair(C.byref(V.surf), C.byref(V.surf2), C.byref(V.rec), C.byref(V.em), emitter, tri0, tri1, _p(u),
                    _p(v), u.shape[0], _p(out))
    return {k: out[:, i] for i, k in enumerate(("uk", "vk", "E", "u2", "v2", "t1", "t2", "detJ"))}


def solve_pair(scene, wl_point, wl_key, wl_p, newton_iters: int = 16, polish_iters: int = 1, tol: float = 1e-5,
               n_threads: int = 1):
    """Pair-tuple Newton: contribution E/P, root (u1, v1), status (1 = root) per worklist entry."""
    L = lib()
    V = _SceneViews(scene)
    wl_point = np.ascontiguousarray(wl_point, np.int64)
    wl_key = np.ascontiguousarray(wl_key, np.uint64)
    wl_p = np.ascontiguousarray(wl_p, np.float32)
    su = np.ascontiguousarray(scene.su, np.float32)
    sv = np.ascontiguousarray(scene.sv, np.float32)
    n = wl_point.shape[0]
    contrib, ru, rv = np.zeros(n), np.zeros(n), np.zeros(n)
    st = np.zeros(n, np.int32)
    L.orc_solve_pair(C.byref(V.surf), C.byref(V.surf2), C.byref(V.rec), C.byref(V.em), _p(wl_point), _p(wl_key),
                     _p(wl_p), n, _p(su), _p(sv), newton_iters, polish_iters, tol, _p(contrib), _p(ru), _p(rv),
                     _p(st), n_threads)
    return contrib, ru, rv, st


def render_pairs(scene, gamma: float, seed: int, depth: Optional[int] = None, newton_iters: int = 16,
                 polish_iters: int = 1, tol: float = 1e-5, n_threads: int = 1, irradiance: bool = False):
    """Whole two-vertex path on the CPU: candidates -> pair bounds (irradiance: with the chain
    irradiance bounds) -> index -> Algorithm 1 -> Newton."""
    rec = bound_pair_scene(scene, depth, n_threads, irradiance)
    f = records_to_f32(rec)
    off, key, et = index(f["u_lo"], f["u_hi"], f["v_lo"], f["v_hi"], f["e_hi"], f["emitter"], f["tri0"],
                         f["tri1"], f["flags"], scene.grid_res)
    wp, wk, wP, n_u = sample(off, key, et, scene.grid_res, scene.su, scene.sv, gamma, seed)
    contrib, ru, rv, st = solve_pair(scene, wp, wk, wP, newton_iters, polish_iters, tol, n_threads)
    E = accumulate(scene.su.shape[0], wp, contrib)
    return dict(records=rec, offsets=off, key=key, etilde=et, wl_point=wp, wl_key=wk, wl_p=wP, n_U=n_u,
                contrib=contrib, root_u=ru, root_v=rv, status=st, E=E)

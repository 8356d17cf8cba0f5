"""Python binding of libbnb (include/bnb.h): argument marshalling only.

The C entry points keep their names (``bnb_bound_tuples``, ``bnb_build_index``,
``bnb_sample_and_solve`` and the ``*_ws`` queries).  Torch tensors provide the
device memory and the CUDA stream; every step of the path runs in libbnb's
kernels.  There is no CPU fallback: importing the library fails loudly when
``libbnb.so`` has not been built.

Higher-level helpers (``DeviceScene``, ``bound_tuples``, ``build_index``,
``sample_and_solve``) allocate outputs and workspaces as torch tensors, zero
the device status words, call the C function, and re-call once with larger
buffers when the device reports BNB_ERR_CAPACITY.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbnb.so")

BNB_OK, BNB_ERR_INVALID, BNB_ERR_CAPACITY, BNB_ERR_CUDA, BNB_ERR_UNSUPPORTED, BNB_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
BNB_REFLECT, BNB_REFRACT = 0, 1
LIVE, SPLIT, CULL_BEHIND, CULL_EMPTY, FOLD, POS_UNBOUNDED, QSIGN_FP64, TIR = 1, 2, 4, 8, 16, 32, 64, 128
DEPTH_SHIFT = 24

vp, i32, i64, u64, f32, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float, C.c_size_t


class bnb_surface(C.Structure):
    _fields_ = [("n_verts", i32), ("n_tris", i32), ("px", vp), ("py", vp), ("pz", vp), ("nx", vp), ("ny", vp),
                ("nz", vp), ("i0", vp), ("i1", vp), ("i2", vp), ("kind", i32), ("eta", f32)]


class bnb_receiver(C.Structure):
    _fields_ = [("p0", f32 * 3), ("e1", f32 * 3), ("e2", f32 * 3)]


class bnb_emitters(C.Structure):
    _fields_ = [("n", i32), ("x", vp), ("y", vp), ("z", vp), ("intensity", vp)]


class bnb_bound_cfg(C.Structure):
    _fields_ = [("depth", i32), ("max_extra_split", i32), ("irradiance", i32), ("fp64", i32), ("adapt_depth", i32),
                ("sigma", f32), ("alpha", f32), ("block_threads", i32), ("split_capacity", i64)]


class bnb_cell_bounds(C.Structure):
    _fields_ = [("capacity", i64), ("count", vp), ("status", vp), ("u_lo", vp), ("u_hi", vp), ("v_lo", vp),
                ("v_hi", vp), ("e_hi", vp), ("e_lo", vp), ("emitter", vp), ("tri0", vp), ("tri1", vp),
                ("cell", vp), ("flags", vp), ("e_hi_min", vp), ("n_base", i64), ("depth", i32), ("n_emitters", i32),
                ("n_tris", i32)]


class bnb_index(C.Structure):
    _fields_ = [("grid_res", i32), ("capacity", i64), ("count", vp), ("status", vp), ("offsets", vp),
                ("key", vp), ("etilde", vp)]


class bnb_sample_cfg(C.Structure):
    _fields_ = [("gamma", f32), ("seed", u64), ("newton_iters", i32), ("polish_iters", i32), ("tol", f32),
                ("worklist_capacity", i64), ("bins", i32), ("stoc_trials", i32)]


class bnb_sample_stats(C.Structure):
    _fields_ = [("counters", vp), ("status", vp), ("sel_count", vp), ("sel_point", vp), ("sel_key", vp),
                ("root_u1", vp)]


class bnb_job(C.Structure):
    _fields_ = [("packed_tris", vp), ("n_tris", i32), ("n_emitters", i32), ("ex", vp), ("ey", vp), ("ez", vp),
                ("ei", vp), ("emitter_on", vp), ("rp0", f32 * 3), ("re1", f32 * 3), ("re2", f32 * 3),
                ("grid_res", i32), ("kind", i32), ("eta", f32), ("reserved0", i32), ("offsets", vp), ("key", vp), ("etilde", vp), ("index_capacity", i64),
                ("su", vp), ("sv", vp), ("n_points", i64), ("gamma", f32), ("reserved", C.c_uint32), ("seed", u64),
                ("E_out", vp)]


class bnb_bound_job(C.Structure):
    _fields_ = [("packed_tris", vp), ("ex", vp), ("ey", vp), ("ez", vp), ("ei", vp), ("n_tris", i32),
                ("n_emitters", i32), ("kind", i32), ("depth", i32), ("eta", f32), ("irradiance", i32),
                ("rp0", f32 * 3), ("re1", f32 * 3), ("re2", f32 * 3), ("reserved", i32), ("capacity", i64),
                ("count", vp), ("status", vp), ("u_lo", vp), ("u_hi", vp), ("v_lo", vp), ("v_hi", vp), ("e_hi", vp),
                ("e_lo", vp), ("emitter", vp), ("tri0", vp), ("tri1", vp), ("cell", vp), ("flags", vp)]


class bnb_batch_cfg(C.Structure):
    _fields_ = [("max_jobs", i32), ("newton_iters", i32), ("max_points", i64), ("worklist_capacity", i64),
                ("polish_iters", i32), ("tol", f32), ("block_threads", i32), ("blocks_per_sm", i32)]


_lib = None
EXPORTS = ["bnb_bound_tuples", "bnb_bound_tuples_ws", "bnb_bound_tuples_noalloc", "bnb_build_index",
           "bnb_build_index_ws", "bnb_sample_and_solve", "bnb_sample_and_solve_ws", "bnb_status_string",
           "bnb_abi_version", "bnb_pack_surface", "bnb_pack_surface_bytes", "bnb_sample_and_solve_batched",
           "bnb_sample_and_solve_batched_ws", "bnb_bound_tuples_batched", "bnb_bound_tuples_batched_ws",
           "bnb_implicit_irradiance", "bnb_stream_status", "bnb_gamma_for_target", "bnb_gamma_for_target_ws",
           "bnb_ffma_probe"]


def lib():
    """Load libbnb.so (raises when it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbnb.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        L.bnb_bound_tuples.restype = i32
        L.bnb_bound_tuples.argtypes = [P(bnb_surface), P(bnb_surface), P(bnb_receiver), P(bnb_emitters),
                                       P(bnb_bound_cfg), P(bnb_cell_bounds), vp, sz, vp]
        L.bnb_bound_tuples_ws.restype = sz
        L.bnb_bound_tuples_ws.argtypes = [P(bnb_surface), P(bnb_surface), P(bnb_emitters), P(bnb_bound_cfg)]
        L.bnb_bound_tuples_noalloc.restype = i32
        L.bnb_bound_tuples_noalloc.argtypes = [P(bnb_surface), P(bnb_surface), P(bnb_receiver), P(bnb_emitters),
                                               P(bnb_bound_cfg), P(bnb_cell_bounds), vp]
        L.bnb_build_index.restype = i32
        L.bnb_build_index.argtypes = [P(bnb_cell_bounds), f32, i64, P(bnb_index), vp, sz, vp]
        L.bnb_build_index_ws.restype = sz
        L.bnb_build_index_ws.argtypes = [P(bnb_cell_bounds), i32, i64]
        L.bnb_sample_and_solve.restype = i32
        L.bnb_sample_and_solve.argtypes = [P(bnb_surface), P(bnb_surface), P(bnb_receiver), P(bnb_emitters),
                                           P(bnb_index), vp, vp, i64, P(bnb_sample_cfg), vp, P(bnb_sample_stats),
                                           vp, sz, vp]
        L.bnb_sample_and_solve_ws.restype = sz
        L.bnb_sample_and_solve_ws.argtypes = [P(bnb_surface), P(bnb_surface), i64, i64]
        L.bnb_implicit_irradiance.restype = i32
        L.bnb_implicit_irradiance.argtypes = [P(bnb_surface), P(bnb_receiver), P(bnb_emitters), P(bnb_cell_bounds),
                                              i64, i32, vp]
        L.bnb_gamma_for_target.restype = i32
        L.bnb_gamma_for_target.argtypes = [P(bnb_index), vp, vp, i64, C.c_double, vp, vp, sz, vp]
        L.bnb_gamma_for_target_ws.restype = sz
        L.bnb_gamma_for_target_ws.argtypes = [i32]
        L.bnb_ffma_probe.restype = i32
        L.bnb_ffma_probe.argtypes = [i32, i32, i32, i32, vp, vp]
        L.bnb_stream_status.restype = i32
        L.bnb_stream_status.argtypes = [vp]
        L.bnb_status_string.restype = C.c_char_p
        L.bnb_status_string.argtypes = [i32]
        L.bnb_abi_version.restype = i32
        L.bnb_pack_surface_bytes.restype = sz
        L.bnb_pack_surface_bytes.argtypes = [P(bnb_surface)]
        L.bnb_pack_surface.restype = i32
        L.bnb_pack_surface.argtypes = [P(bnb_surface), vp, sz, vp]
        L.bnb_sample_and_solve_batched.restype = i32
        L.bnb_sample_and_solve_batched.argtypes = [vp, vp, P(bnb_batch_cfg), P(bnb_sample_stats), vp, sz, vp]
        L.bnb_bound_tuples_batched.restype = i32
        L.bnb_bound_tuples_batched.argtypes = [vp, vp, i32, vp, sz, vp]
        L.bnb_bound_tuples_batched_ws.restype = sz
        L.bnb_bound_tuples_batched_ws.argtypes = [i32]
        L.bnb_sample_and_solve_batched_ws.restype = sz
        L.bnb_sample_and_solve_batched_ws.argtypes = [P(bnb_batch_cfg)]
        _lib = L
    return _lib


# Raw entry points with the C names (argument marshalling only).
def bnb_bound_tuples(*a):
    return lib().bnb_bound_tuples(*a)


def bnb_bound_tuples_ws(*a):
    return lib().bnb_bound_tuples_ws(*a)


def bnb_bound_tuples_noalloc(*a):
    return lib().bnb_bound_tuples_noalloc(*a)


def bnb_build_index(*a):
    return lib().bnb_build_index(*a)


def bnb_build_index_ws(*a):
    return lib().bnb_build_index_ws(*a)


def bnb_sample_and_solve(*a):
    return lib().bnb_sample_and_solve(*a)


def bnb_sample_and_solve_ws(*a):
    return lib().bnb_sample_and_solve_ws(*a)


def bnb_pack_surface(*a):
    return lib().bnb_pack_surface(*a)


def bnb_pack_surface_bytes(*a):
    return lib().bnb_pack_surface_bytes(*a)


def bnb_sample_and_solve_batched(*a):
    return lib().bnb_sample_and_solve_batched(*a)


def bnb_sample_and_solve_batched_ws(*a):
    return lib().bnb_sample_and_solve_batched_ws(*a)


def bnb_bound_tuples_batched(*a):
    return lib().bnb_bound_tuples_batched(*a)


def bnb_bound_tuples_batched_ws(*a):
    return lib().bnb_bound_tuples_batched_ws(*a)


def bnb_implicit_irradiance(*a):
    return lib().bnb_implicit_irradiance(*a)


def bnb_gamma_for_target(*a):
    return lib().bnb_gamma_for_target(*a)


def bnb_gamma_for_target_ws(*a):
    return lib().bnb_gamma_for_target_ws(*a)


def gamma_for_target(index: "Index", target: float, su: Optional[torch.Tensor] = None,
                     sv: Optional[torch.Tensor] = None, stream=None, out: Optional[torch.Tensor] = None,
                     ws: Optional[torch.Tensor] = None) -> torch.Tensor:
    """gamma whose expected |S| per shading point is `target` (Sec. 5.4), computed by
    bnb_gamma_for_target on the device; returns a one-element device float tensor (not synchronized).
    su, sv: the shading points that weigh the grid cells (None: every grid cell once)."""
    dev = index.offsets.device
    out = out if out is not None else torch.empty(1, dtype=torch.float32, device=dev)
    need = bnb_gamma_for_target_ws(index.grid_res)
    if ws is None or ws.numel() < need + 256:
        ws = _ws(need, dev)
    n = 0 if su is None else int(su.shape[0])
    rc = bnb_gamma_for_target(C.byref(index.c), _ptr(su), _ptr(sv), n, float(target), _ptr(out), _align(ws),
                              C.c_size_t(need), _stream(stream))
    _check(rc, "bnb_gamma_for_target")
    return out


def bnb_ffma_probe(*a):
    return lib().bnb_ffma_probe(*a)


def fp32_fma_peak(device=None, seconds: float = 1.0, stream=None) -> dict:
    """Measured FP32 FMA throughput (TFLOP/s) of this GPU with bnb_ffma_probe: scalar FFMA and paired
    FFMA2, a resident grid (8 blocks of 256 threads per SM), timed with CUDA events on the stream
    over about `seconds` per form after a warm-up; returns both rates and the larger as "peak"."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = sms * 8, 256
    sink = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    out = {"blocks": blocks, "threads": threads}
    for paired in (0, 1):
        iters = 4096
        flops = lambda it: blocks * threads * it * 32 * (2 if paired else 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):  # warm-up, and grow iters until one launch takes ~20 ms
            e0.record(st)
            _check(bnb_ffma_probe(blocks, threads, iters, paired, _ptr(sink), _stream(st)), "bnb_ffma_probe")
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            iters = max(1, min(1 << 22, int(iters * 20.0 / max(ms, 1e-3))))
        reps = max(3, int(seconds * 1e3 / 20.0))
        e0.record(st)
        for _ in range(reps):
            _check(bnb_ffma_probe(blocks, threads, iters, paired, _ptr(sink), _stream(st)), "bnb_ffma_probe")
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out["ffma2_tflops" if paired else "ffma_tflops"] = flops(iters) / (ms / 1e3) / 1e12
    if not bool(torch.isfinite(sink).all()):
        raise BnbError("bnb_ffma_probe: non-finite chain")
    out["peak"] = max(out["ffma_tflops"], out["ffma2_tflops"])
    return out


def bnb_stream_status(*a):
    return lib().bnb_stream_status(*a)


def stream_status(stream=None) -> int:
    """Synchronizes the stream and returns (and clears) the device error word: BNB_OK, or the first
    code a kernel raised since the last read."""
    return int(bnb_stream_status(_stream(stream)))


def bnb_status_string(s: int) -> str:
    return lib().bnb_status_string(s).decode()


class BnbError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != BNB_OK:
        raise BnbError(f"{what}: {bnb_status_string(rc)} ({rc})")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ws(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks; +256 keeps a zero-size request valid.
    return torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)


# ----------------------------------------------------------------------------- device scene
class DeviceScene:
    """A scene's inputs resident in device memory, with the C structs pointing at them."""

    def __init__(self, scene, device="cuda"):
        self.scene = scene
        self.device = torch.device(device)
        d = self.device
        s = scene.s1

        def t(a, dt):
            return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(d)

        self.t = dict(px=t(s.px, torch.float32), py=t(s.py, torch.float32), pz=t(s.pz, torch.float32),
                      nx=t(s.nx, torch.float32), ny=t(s.ny, torch.float32), nz=t(s.nz, torch.float32),
                      i0=t(s.i0, torch.int32), i1=t(s.i1, torch.int32), i2=t(s.i2, torch.int32),
                      ex=t(scene.emitters.x, torch.float32), ey=t(scene.emitters.y, torch.float32),
                      ez=t(scene.emitters.z, torch.float32), ei=t(scene.emitters.intensity, torch.float32),
                      su=t(scene.su, torch.float32), sv=t(scene.sv, torch.float32))
        s2 = scene.s2
        if s2 is not None:  # second specular surface (two-vertex chains)
            for k, a in (("px", s2.px), ("py", s2.py), ("pz", s2.pz), ("nx", s2.nx), ("ny", s2.ny), ("nz", s2.nz)):
                self.t["s2_" + k] = t(a, torch.float32)
            for k, a in (("i0", s2.i0), ("i1", s2.i1), ("i2", s2.i2)):
                self.t["s2_" + k] = t(a, torch.int32)
        T = self.t
        self.s1 = bnb_surface(s.n_verts, s.n_tris, _ptr(T["px"]), _ptr(T["py"]), _ptr(T["pz"]), _ptr(T["nx"]),
                              _ptr(T["ny"]), _ptr(T["nz"]), _ptr(T["i0"]), _ptr(T["i1"]), _ptr(T["i2"]), s.kind,
                              s.eta)
        self.s2 = None
        if s2 is not None:
            self.s2 = bnb_surface(s2.n_verts, s2.n_tris, *[_ptr(T["s2_" + k]) for k in
                                                           ("px", "py", "pz", "nx", "ny", "nz", "i0", "i1", "i2")],
                                  s2.kind, s2.eta)
        r = scene.receiver
        self.rec = bnb_receiver((f32 * 3)(*r.p0), (f32 * 3)(*r.e1), (f32 * 3)(*r.e2))
        self.em = bnb_emitters(scene.emitters.n, _ptr(T["ex"]), _ptr(T["ey"]), _ptr(T["ez"]), _ptr(T["ei"]))

    @property
    def n_points(self) -> int:
        return int(self.t["su"].shape[0])

    def s2_ref(self):
        """bnb_surface pointer of the second surface, or None (one specular vertex)."""
        return C.byref(self.s2) if self.s2 is not None else None

    def with_emitters(self, which) -> "DeviceScene":
        """The same resident mesh, receiver and points lit by the emitters `which` (indices into
        this scene's emitters, gathered into new device arrays)."""
        out = object.__new__(DeviceScene)
        out.device = self.device
        sel = np.asarray(which, dtype=np.int64)
        e = self.scene.emitters
        out.scene = dataclasses.replace(self.scene, emitters=dataclasses.replace(
            e, x=e.x[sel], y=e.y[sel], z=e.z[sel], intensity=e.intensity[sel]))
        idx = torch.as_tensor(sel, device=self.device)
        out.t = dict(self.t)
        for k in ("ex", "ey", "ez", "ei"):
            out.t[k] = self.t[k].index_select(0, idx)
        out.s1 = self.s1
        out.s2 = self.s2
        out.rec = self.rec
        T = out.t
        out.em = bnb_emitters(int(sel.shape[0]), _ptr(T["ex"]), _ptr(T["ey"]), _ptr(T["ez"]), _ptr(T["ei"]))
        return out


# ----------------------------------------------------------------------------- outputs
class CellBounds:
    """Cell records (SoA device tensors) plus their bnb_cell_bounds view."""

    def __init__(self, capacity: int, device, with_e_hi_min: bool = False, with_e_lo: bool = True):
        d = device
        self.capacity = int(capacity)
        f = lambda dt: torch.empty(self.capacity, dtype=dt, device=d)
        self.count = torch.zeros(1, dtype=torch.int64, device=d)
        self.status = torch.zeros(1, dtype=torch.int32, device=d)
        self.u_lo, self.u_hi, self.v_lo, self.v_hi = f(torch.float32), f(torch.float32), f(torch.float32), f(torch.float32)
        self.e_hi = f(torch.float32)
        self.e_lo = f(torch.float32) if with_e_lo else None
        self.emitter, self.tri0, self.tri1 = f(torch.int32), f(torch.int32), f(torch.int32)
        self.cell, self.flags = f(torch.int32), f(torch.int32)
        self.e_hi_min = f(torch.float32) if with_e_hi_min else None
        self.c = bnb_cell_bounds(self.capacity, _ptr(self.count), _ptr(self.status), _ptr(self.u_lo),
                                 _ptr(self.u_hi), _ptr(self.v_lo), _ptr(self.v_hi), _ptr(self.e_hi), _ptr(self.e_lo),
                                 _ptr(self.emitter), _ptr(self.tri0), _ptr(self.tri1), _ptr(self.cell),
                                 _ptr(self.flags), _ptr(self.e_hi_min), 0, 0, 0, 0)

    def reset(self):
        self.count.zero_()
        self.status.zero_()

    def n_records(self) -> int:
        return min(int(self.count.item()), self.capacity)

    def to_numpy(self) -> dict:
        n = self.n_records()
        g = lambda t: t[:n].cpu().numpy()
        out = dict(u_lo=g(self.u_lo), u_hi=g(self.u_hi), v_lo=g(self.v_lo), v_hi=g(self.v_hi),
                   e_lo=g(self.e_lo) if self.e_lo is not None else np.zeros(n, np.float32), e_hi=g(self.e_hi), emitter=g(self.emitter), tri0=g(self.tri0), tri1=g(self.tri1),
                   cell=g(self.cell).view(np.uint32), flags=g(self.flags).view(np.uint32))
        if self.e_hi_min is not None:
            out["e_hi_min"] = g(self.e_hi_min)
        return out


class Index:
    def __init__(self, grid_res: int, capacity: int, device):
        d = device
        self.grid_res = int(grid_res)
        self.capacity = int(capacity)
        self.count = torch.zeros(2, dtype=torch.int64, device=d)
        self.status = torch.zeros(1, dtype=torch.int32, device=d)
        self.offsets = torch.empty(self.grid_res * self.grid_res + 1, dtype=torch.int64, device=d)
        self.key = torch.empty(max(1, self.capacity), dtype=torch.int64, device=d)
        self.etilde = torch.empty(max(1, self.capacity), dtype=torch.float32, device=d)
        self.c = bnb_index(self.grid_res, self.capacity, _ptr(self.count), _ptr(self.status), _ptr(self.offsets),
                           _ptr(self.key), _ptr(self.etilde))

    def reset(self):
        self.count.zero_()
        self.status.zero_()

    def to_numpy(self):
        n = min(int(self.count[0].item()), self.capacity)
        return (self.offsets.cpu().numpy(), self.key[:n].cpu().numpy().view(np.uint64),
                self.etilde[:n].cpu().numpy())


# ----------------------------------------------------------------------------- high-level calls
def implicit_irradiance(ds: DeviceScene, cells: CellBounds, n: int = -1, mode: int = 0, stream=None) -> None:
    """Implicit-differentiation irradiance bounds (Sec. 4.4) of the live single-refraction records
    [0, n) of `cells` (n = -1: all the pass produced), in place: mode 0 writes them, mode 1
    intersects them with the stored bounds."""
    rc = bnb_implicit_irradiance(C.byref(ds.s1), C.byref(ds.rec), C.byref(ds.em), C.byref(cells.c), n, mode,
                                        _stream(stream))
    _check(rc, "bnb_implicit_irradiance")


def bound_tuples(ds: DeviceScene, depth: int, max_extra_split: int = 4, irradiance=True,
                 fp64: bool = False, capacity: Optional[int] = None, out: Optional[CellBounds] = None,
                 ws: Optional[torch.Tensor] = None, stream=None, sync_check: bool = True,
                 with_e_hi_min: bool = False, with_e_lo: bool = True, adapt_depth: int = 0, sigma: float = 0.0,
                 alpha: float = 0.0, split_capacity: int = 0, block_threads: int = 0) -> CellBounds:
    """Bound pass (one or two specular vertices).  adapt_depth > depth: adaptive subdivision
    (Sec. 6.1) down to adapt_depth, a cell stopping when its box area is below sigma or
    E_hi < alpha E_lo; split_capacity sizes the per-level split queue (0: the library default).
    irradiance: False / True, or 2 (single refraction) to intersect each bound with the
    implicit-differentiation bound (Sec. 4.4).  block_threads: block size of the float32 reflection
    pass (0: the library default; see batch.autotune_bound)."""
    n_base = ds.scene.emitters.n * ds.s1.n_tris * 4 ** depth
    adaptive = adapt_depth > depth
    if adaptive and split_capacity == 0:
        split_capacity = n_base + 4096
    if out is None:
        # pairs: one record per (cell, candidate T2), a few per cell; adaptive: the tree's cells;
        # the call reports the count
        default = n_base * 4 + 1024 if (ds.s2 is not None or adaptive) else n_base + n_base // 8 + 1024
        out = CellBounds(capacity if capacity is not None else default, ds.device, with_e_hi_min, with_e_lo)
    for _ in range(6):
        cfg = bnb_bound_cfg(depth, max_extra_split, int(irradiance), int(fp64), adapt_depth if adaptive else 0,
                            sigma, alpha, int(block_threads), split_capacity)
        need = bnb_bound_tuples_ws(C.byref(ds.s1), ds.s2_ref(), C.byref(ds.em), C.byref(cfg))
        if need == 0:
            raise BnbError("bnb_bound_tuples_ws: invalid configuration")
        if ws is None or ws.numel() < need + 256:
            ws = _ws(need, ds.device)
        out.reset()
        rc = bnb_bound_tuples(C.byref(ds.s1), ds.s2_ref(), C.byref(ds.rec), C.byref(ds.em), C.byref(cfg),
                              C.byref(out.c), _align(ws), C.c_size_t(need), _stream(stream))
        _check(rc, "bnb_bound_tuples")
        if not sync_check:
            return out
        if int(out.status.item()) == BNB_OK:
            return out
        count = int(out.count.item())
        if count > out.capacity:  # records: re-call with room for all of them
            out = CellBounds(count + count // 8 + 1024, ds.device, with_e_hi_min, with_e_lo)
        else:  # a split level overflowed its queue
            split_capacity = 2 * (split_capacity or (4096 + n_base // 32))
    raise BnbError("bnb_bound_tuples: capacity exceeded repeatedly")


def _align(ws: torch.Tensor):
    p = ws.data_ptr()
    return C.c_void_p((p + 255) // 256 * 256)


def build_index(cells: CellBounds, grid_res: int = 512, m: float = 1.0, pre_capacity: Optional[int] = None,
                capacity: Optional[int] = None, out: Optional[Index] = None, ws: Optional[torch.Tensor] = None,
                stream=None, sync_check: bool = True) -> Index:
    dev = cells.u_lo.device
    n_rec = cells.capacity
    pre = pre_capacity if pre_capacity is not None else max(4096, n_rec // 4)
    cap = capacity if capacity is not None else pre
    for _ in range(3):
        if out is None or out.capacity < cap:
            out = Index(grid_res, cap, dev)
        need = bnb_build_index_ws(C.byref(cells.c), grid_res, pre)
        if ws is None or ws.numel() < need + 256:
            ws = _ws(need, dev)
        out.reset()
        rc = bnb_build_index(C.byref(cells.c), m, pre, C.byref(out.c), _align(ws), C.c_size_t(need),
                             _stream(stream))
        _check(rc, "bnb_build_index")
        if not sync_check:
            return out
        if int(out.status.item()) == BNB_OK:
            return out
        pre = max(pre, int(out.count[1].item()) + 1024)
        cap = max(cap, int(out.count[0].item()) + 1024, pre)
        free, _ = torch.cuda.mem_get_info(dev)
        if (pre * 32 + cap * 12) > free:
            raise BnbError(f"bnb_build_index: needs {pre} pre-merge and {cap} index entries, more than the "
                           f"free device memory ({free} bytes)")
        out = None
    raise BnbError("bnb_build_index: capacity exceeded repeatedly")


@dataclasses.dataclass
class SampleResult:
    E: torch.Tensor
    counters: torch.Tensor
    status: torch.Tensor
    sel_count: Optional[torch.Tensor] = None
    sel_point: Optional[torch.Tensor] = None  # with_roots: per selection, worklist order
    sel_key: Optional[torch.Tensor] = None
    root_u1: Optional[torch.Tensor] = None    # with_roots: (n, 2) float64, NaN where no root

    def roots(self):
        """(point, key, u, v) of the selections, as numpy arrays (with_roots only)."""
        n = min(int(self.counters[1].item()), int(self.sel_point.shape[0]))
        return (self.sel_point[:n].cpu().numpy(), self.sel_key[:n].cpu().numpy().view(np.uint64),
                self.root_u1[:n].cpu().numpy())


def sample_and_solve(ds: DeviceScene, index: Index, gamma: float, seed: int, newton_iters: int = 16,
                     polish_iters: int = 1, tol: float = 1e-5, worklist_capacity: Optional[int] = None,
                     su: Optional[torch.Tensor] = None, sv: Optional[torch.Tensor] = None,
                     E_out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None, stream=None,
                     sync_check: bool = True, with_sel_count: bool = False, bins: bool = False,
                     stoc_trials: int = 0, with_roots: bool = False) -> SampleResult:
    """Rendering pass.  bins: the bin-packed selection (one draw per group of Sec. 5.3) instead of
    Algorithm 1's draw per tuple; counters[3] then holds |B|.  stoc_trials > 0: stochastic Newton
    starts with the reciprocal weighting (Sec. 6.1 "Stoc"), weights capped at stoc_trials.
    with_roots: also return, per selection, its point, key and the accepted root's barycentric
    coordinates in T1 (NaN where the selection has no root)."""
    su = ds.t["su"] if su is None else su
    sv = ds.t["sv"] if sv is None else sv
    n_points = int(su.shape[0])
    wl = worklist_capacity if worklist_capacity is not None else max(1024, 16 * n_points)
    counters = torch.zeros(4, dtype=torch.int64, device=ds.device)
    status = torch.zeros(1, dtype=torch.int32, device=ds.device)
    E = E_out if E_out is not None else torch.empty(n_points, dtype=torch.float32, device=ds.device)
    sel = torch.zeros(n_points, dtype=torch.int32, device=ds.device) if with_sel_count else None
    for _ in range(2):
        cfg = bnb_sample_cfg(gamma, seed, newton_iters, polish_iters, tol, wl, int(bins), int(stoc_trials))
        need = bnb_sample_and_solve_ws(C.byref(ds.s1), ds.s2_ref(), n_points, wl)
        if ws is None or ws.numel() < need + 256:
            ws = _ws(need, ds.device)
        counters.zero_()
        status.zero_()
        sp = sk = ru = None
        if with_roots:
            sp = torch.empty(max(1, wl), dtype=torch.int64, device=ds.device)
            sk = torch.empty(max(1, wl), dtype=torch.int64, device=ds.device)
            ru = torch.empty((max(1, wl), 2), dtype=torch.float64, device=ds.device)
        stats = bnb_sample_stats(_ptr(counters), _ptr(status), _ptr(sel), _ptr(sp), _ptr(sk), _ptr(ru))
        rc = bnb_sample_and_solve(C.byref(ds.s1), ds.s2_ref(), C.byref(ds.rec), C.byref(ds.em), C.byref(index.c),
                                  _ptr(su), _ptr(sv), n_points, C.byref(cfg), _ptr(E), C.byref(stats), _align(ws),
                                  C.c_size_t(need), _stream(stream))
        _check(rc, "bnb_sample_and_solve")
        if not sync_check or int(status.item()) == BNB_OK:
            return SampleResult(E, counters, status, sel, sp, sk, ru)
        wl = int(counters[1].item()) + 1024
    raise BnbError("bnb_sample_and_solve: worklist capacity exceeded twice")

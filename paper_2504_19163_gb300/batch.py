"""Batched rendering pass: resident scenes, a device job table replayed from a CUDA graph, and
the launch-shape autotuner.

A job is one request's shading points against one resident scene (packed triangles, emitters,
receiver and index already in device memory).  ``BatchRunner`` owns a pinned host copy of the
job table, its device copy, the device job count and the workspace of
``bnb_sample_and_solve_batched``.  Its launch sequence (job table and count copied host to
device, status cleared, the batched call, status and counters copied back) does not depend on
the jobs, so it is captured once in a CUDA graph and replayed for every batch: the host only
rewrites the pinned table between replays.

``autotune`` times candidate launch shapes (threads per block, resident blocks per SM) of the
batched kernels on a representative batch and caches the fastest per (device, size class) in a
JSON file.  Results do not depend on the launch shape (per point the draws, the solve and the
sum order are fixed), so the tuner only changes speed.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import json
import math
import os
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import bnb
from .bnb import _align, _check, _ptr, _stream

JOB_BYTES = C.sizeof(bnb.bnb_job)


def gamma_for_target(index: bnb.Index, target: float, su: Optional[torch.Tensor] = None,
                     sv: Optional[torch.Tensor] = None, stream=None) -> float:
    """gamma such that the mean over shading points of the expected number of selected tuples
    equals `target` (Sec. 5.4: gamma and E|S| are in one-to-one correspondence), computed on the
    device by bnb_gamma_for_target.  Points default to a uniform density over [0,1]^2 (every grid
    cell weighted equally).  Synchronizes the stream to return the value."""
    g = bnb.gamma_for_target(index, target, su, sv, stream=stream)
    return float(g.item())


class ResidentScene:
    """A scene kept in device memory for rendering: its inputs (``DeviceScene``), its specular
    triangles packed for the batched pass, its emitters and receiver, and its index."""

    def __init__(self, ds: bnb.DeviceScene, index: bnb.Index, gamma: float, stream=None):
        self.ds = ds
        self.index = index
        self.gamma = float(gamma)
        nbytes = int(bnb.bnb_pack_surface_bytes(C.byref(ds.s1)))
        self.packed = torch.empty(max(16, nbytes) // 4, dtype=torch.float32, device=ds.device)
        _check(bnb.bnb_pack_surface(C.byref(ds.s1), _ptr(self.packed), C.c_size_t(nbytes), _stream(stream)),
               "bnb_pack_surface")

    @property
    def n_emitters(self) -> int:
        return int(self.ds.em.n)

    def device_bytes(self) -> int:
        b = self.packed.numel() * 4
        b += sum(t.numel() * t.element_size() for k, t in self.ds.t.items() if k not in ("su", "sv"))
        ix = self.index
        b += ix.offsets.numel() * 8 + ix.key.numel() * 8 + ix.etilde.numel() * 4
        return int(b)

    def fill_job(self, job: bnb.bnb_job, su: torch.Tensor, sv: torch.Tensor, E_out: torch.Tensor, seed: int,
                 emitter_on: Optional[torch.Tensor] = None, gamma: Optional[float] = None):
        T = self.ds.t
        job.packed_tris = self.packed.data_ptr()
        job.n_tris = self.ds.s1.n_tris
        job.n_emitters = self.ds.em.n
        job.ex, job.ey, job.ez, job.ei = (T["ex"].data_ptr(), T["ey"].data_ptr(), T["ez"].data_ptr(),
                                          T["ei"].data_ptr())
        job.emitter_on = None if emitter_on is None else emitter_on.data_ptr()
        r = self.ds.rec
        for c in range(3):
            job.rp0[c], job.re1[c], job.re2[c] = r.p0[c], r.e1[c], r.e2[c]
        ix = self.index
        job.grid_res = ix.grid_res
        job.kind = self.ds.s1.kind
        job.eta = self.ds.s1.eta
        job.reserved0 = 0
        job.offsets, job.key, job.etilde = ix.offsets.data_ptr(), ix.key.data_ptr(), ix.etilde.data_ptr()
        job.index_capacity = ix.capacity
        job.su, job.sv = su.data_ptr(), sv.data_ptr()
        job.n_points = int(su.shape[0])
        job.gamma = self.gamma if gamma is None else float(gamma)
        job.reserved = 0
        job.seed = int(seed)
        job.E_out = E_out.data_ptr()


@dataclasses.dataclass
class Job:
    scene: ResidentScene
    su: torch.Tensor
    sv: torch.Tensor
    E_out: torch.Tensor
    seed: int
    emitter_on: Optional[torch.Tensor] = None
    gamma: Optional[float] = None

    @property
    def n_points(self) -> int:
        return int(self.su.shape[0])


class BatchRunner:
    """One batched launch sequence with fixed capacities, optionally captured in a CUDA graph.

    ``submit(jobs)`` writes the jobs into the pinned table and enqueues the sequence (graph replay
    after the first call) on the runner's stream; it returns an event that completes when the
    batch, including the copy of status and counters to pinned host memory, is done.  A runner
    holds one batch at a time: ``submit`` waits for the previous batch's event before rewriting
    the pinned table."""

    def __init__(self, max_jobs: int, max_points: int, worklist_capacity: int, newton_iters: int = 16,
                 polish_iters: int = 1, tol: float = 1e-5, block_threads: int = 0, blocks_per_sm: int = 0,
                 device="cuda", use_graph: bool = True, stream: Optional[torch.cuda.Stream] = None):
        self.device = torch.device(device)
        self.cfg = bnb.bnb_batch_cfg(int(max_jobs), int(newton_iters), int(max_points), int(worklist_capacity),
                                     int(polish_iters), float(tol), int(block_threads), int(blocks_per_sm))
        self.ws_bytes = int(bnb.bnb_sample_and_solve_batched_ws(C.byref(self.cfg)))
        if self.ws_bytes == 0:
            raise bnb.BnbError("bnb_sample_and_solve_batched_ws: invalid batch configuration")
        d = self.device
        self.host_jobs = torch.zeros(max_jobs * JOB_BYTES, dtype=torch.uint8).pin_memory()
        self.dev_jobs = torch.zeros(max_jobs * JOB_BYTES, dtype=torch.uint8, device=d)
        self.host_n = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.dev_n = torch.zeros(1, dtype=torch.int32, device=d)
        # device stats: int64 counters[4] then int32 status (+pad), copied back as one block
        self.dev_stat = torch.zeros(6, dtype=torch.int64, device=d)
        self.host_stat = torch.zeros(6, dtype=torch.int64).pin_memory()
        self.ws = bnb._ws(self.ws_bytes, d)
        self.stats = bnb.bnb_sample_stats(C.c_void_p(self.dev_stat.data_ptr()),
                                          C.c_void_p(self.dev_stat.data_ptr() + 32), None)
        self.table = (bnb.bnb_job * max_jobs).from_address(self.host_jobs.data_ptr())
        self.stream = stream if stream is not None else torch.cuda.Stream(device=d)
        self.use_graph = use_graph
        self.graph: Optional[torch.cuda.CUDAGraph] = None
        self.done = torch.cuda.Event()
        self.done.record(self.stream)
        self.jobs: List[Job] = []

    @property
    def max_jobs(self) -> int:
        return self.cfg.max_jobs

    @property
    def max_points(self) -> int:
        return self.cfg.max_points

    def _enqueue(self):
        s = self.stream
        self.dev_jobs.copy_(self.host_jobs, non_blocking=True)
        self.dev_n.copy_(self.host_n, non_blocking=True)
        self.dev_stat.zero_()
        rc = bnb.bnb_sample_and_solve_batched(C.c_void_p(self.dev_jobs.data_ptr()),
                                              C.c_void_p(self.dev_n.data_ptr()), C.byref(self.cfg),
                                              C.byref(self.stats), _align(self.ws), C.c_size_t(self.ws_bytes),
                                              C.c_void_p(s.cuda_stream))
        _check(rc, "bnb_sample_and_solve_batched")
        self.host_stat.copy_(self.dev_stat, non_blocking=True)

    def write_table(self, jobs: Sequence[Job]):
        if len(jobs) > self.max_jobs:
            raise ValueError(f"{len(jobs)} jobs > max_jobs {self.max_jobs}")
        if sum(j.n_points for j in jobs) > self.max_points:
            raise ValueError("batch exceeds max_points")
        for i, j in enumerate(jobs):
            j.scene.fill_job(self.table[i], j.su, j.sv, j.E_out, j.seed, j.emitter_on, j.gamma)
        self.host_n[0] = len(jobs)

    def submit(self, jobs: Sequence[Job]) -> torch.cuda.Event:
        self.done.synchronize()  # the previous batch has read the pinned table
        self.write_table(jobs)
        self.jobs = list(jobs)
        with torch.cuda.stream(self.stream):
            if self.use_graph:
                if self.graph is None:
                    self.graph = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
                        self._enqueue()
                self.graph.replay()
            else:
                self._enqueue()
            self.done.record(self.stream)
        return self.done

    def result(self) -> Tuple[int, List[int]]:
        """(status, counters[0:3]) of the last batch; waits for it."""
        self.done.synchronize()
        st = self.host_stat.tolist()
        status = int(C.c_int32(st[4] & 0xFFFFFFFF).value)
        return status, st[:3]


# ----------------------------------------------------------------------------- batched bound pass
BOUND_JOB_BYTES = C.sizeof(bnb.bnb_bound_job)


def bound_batched(items: Sequence[Tuple[bnb.DeviceScene, int, bnb.CellBounds]], irradiance: bool = True,
                  stream=None) -> List[bnb.CellBounds]:
    """Bound the base cells of several scenes in one persistent launch (bnb_bound_tuples_batched).
    items: (scene on the device, depth, output records); the outputs' count and status are zeroed
    here and their host fields (n_base, depth, ...) set for the index pass.  Returns the outputs."""
    if not items:
        return []
    dev = items[0][0].device
    n = len(items)
    host = torch.zeros(n * BOUND_JOB_BYTES, dtype=torch.uint8).pin_memory()
    table = (bnb.bnb_bound_job * n).from_address(host.data_ptr())
    keep = []
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.stream(s):
        for i, (ds, depth, out) in enumerate(items):
            nbytes = int(bnb.bnb_pack_surface_bytes(C.byref(ds.s1)))
            packed = torch.empty(max(16, nbytes) // 4, dtype=torch.float32, device=dev)
            _check(bnb.bnb_pack_surface(C.byref(ds.s1), _ptr(packed), C.c_size_t(nbytes), _stream(s)),
                   "bnb_pack_surface")
            keep.append(packed)
            out.reset()
            T = ds.t
            j = table[i]
            j.packed_tris = packed.data_ptr()
            j.ex, j.ey, j.ez, j.ei = T["ex"].data_ptr(), T["ey"].data_ptr(), T["ez"].data_ptr(), T["ei"].data_ptr()
            j.n_tris, j.n_emitters = ds.s1.n_tris, ds.em.n
            j.kind, j.depth, j.eta, j.irradiance = ds.s1.kind, int(depth), ds.s1.eta, int(irradiance)
            r = ds.rec
            for c in range(3):
                j.rp0[c], j.re1[c], j.re2[c] = r.p0[c], r.e1[c], r.e2[c]
            j.reserved = 0
            oc = out.c
            j.capacity = oc.capacity
            for f in ("count", "status", "u_lo", "u_hi", "v_lo", "v_hi", "e_hi", "e_lo", "emitter", "tri0", "tri1",
                      "cell", "flags"):
                setattr(j, f, getattr(oc, f))
            oc.n_base = ds.em.n * ds.s1.n_tris * 4 ** int(depth)
            oc.depth = int(depth)
            oc.n_emitters = ds.em.n
            oc.n_tris = ds.s1.n_tris
        dev_table = host.to(dev, non_blocking=True)
        n_jobs = torch.tensor([n], dtype=torch.int32).pin_memory().to(dev, non_blocking=True)
        ws_bytes = int(bnb.bnb_bound_tuples_batched_ws(n))
        ws = bnb._ws(ws_bytes, dev)
        rc = bnb.bnb_bound_tuples_batched(C.c_void_p(dev_table.data_ptr()), C.c_void_p(n_jobs.data_ptr()), n,
                                          _align(ws), C.c_size_t(ws_bytes), C.c_void_p(s.cuda_stream))
        _check(rc, "bnb_bound_tuples_batched")
    s.synchronize()  # the table, packed triangles and workspace are released on return
    del keep
    return [it[2] for it in items]


# ----------------------------------------------------------------------------- autotuner
CANDIDATES = [(t, b) for t in (128, 256, 512) for b in (2, 4, 8, 16) if t * b <= 4096]
_cache_lock = threading.Lock()


def _cache_path() -> str:
    p = os.environ.get("BNB_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "bnb_autotune.json")


def size_class(max_points: int) -> int:
    return max(0, int(math.ceil(math.log2(max(1, max_points)))))


def cache_key(device, max_points: int) -> str:
    name = torch.cuda.get_device_name(device).replace(" ", "_")
    return f"{name}|sample_and_solve_batched|points_2^{size_class(max_points)}"


def load_cache() -> Dict[str, dict]:
    p = _cache_path()
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(key: str, entry: dict):
    with _cache_lock:
        c = load_cache()
        c[key] = entry
        p = _cache_path()
        os.makedirs(os.path.dirname(p) or ".", exist_ok=True)
        tmp = p + ".tmp"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, p)


def autotune(jobs: Sequence[Job], worklist_capacity: int, reps: int = 3, device="cuda", use_cache: bool = True,
             candidates: Sequence[Tuple[int, int]] = CANDIDATES) -> dict:
    """Fastest (block_threads, blocks_per_sm) for batches like `jobs`; cached per (device, size class).

    Every candidate runs the same batch `reps` times (after one warm-up) without a graph; the
    median CUDA-event time of the whole batched sequence decides."""
    max_points = sum(j.n_points for j in jobs)
    key = cache_key(device, max_points)
    if use_cache:
        hit = load_cache().get(key)
        if hit is not None:
            return hit
    timings = []
    for bt, bps in candidates:
        r = BatchRunner(len(jobs), max_points, worklist_capacity, block_threads=bt, blocks_per_sm=bps,
                        device=device, use_graph=False)
        ts = []
        for k in range(reps + 1):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            r.done.synchronize()
            r.write_table(jobs)
            a.record(r.stream)
            with torch.cuda.stream(r.stream):
                r._enqueue()
            b.record(r.stream)
            r.done.record(r.stream)
            b.synchronize()
            if k > 0:
                ts.append(a.elapsed_time(b))
        status, _ = r.result()
        if status != bnb.BNB_OK:
            raise bnb.BnbError(f"autotune: batch status {bnb.bnb_status_string(status)}")
        ts.sort()
        timings.append((ts[len(ts) // 2], bt, bps))
        del r
    timings.sort()
    best = timings[0]
    entry = {"block_threads": best[1], "blocks_per_sm": best[2], "ms": best[0],
             "candidates": [[bt, bps, ms] for ms, bt, bps in sorted(timings, key=lambda x: (x[1], x[2]))]}
    if use_cache:
        store_cache(key, entry)
    return entry


BOUND_SCHEDULES = (256, 320, 384)       # block sizes the float32 reflection bound pass is compiled for
REFRACT_SCHEDULES = (128, 256)          # ... and the float32 refraction pass


def autotune_bound(ds: bnb.DeviceScene, depth: int, reps: int = 3, use_cache: bool = True,
                   candidates: Optional[Sequence[int]] = None, **bound_kw) -> dict:
    """Fastest block size of the bound pass for scenes like `ds` at `depth`; cached per (device,
    kind, size class = log2 of the base cells).  Every candidate bounds the scene `reps` times after
    one warm-up into the same outputs; the median CUDA-event time decides.  Only the float32
    one-vertex passes have schedules: the others return the default (0) without timing."""
    if ds.s2 is not None or bound_kw.get("fp64"):
        return {"block_threads": 0, "ms": None, "candidates": []}
    refract = ds.s1.kind == bnb.BNB_REFRACT
    if candidates is None:
        candidates = REFRACT_SCHEDULES if refract else BOUND_SCHEDULES
    n_base = ds.scene.emitters.n * ds.s1.n_tris * 4 ** depth
    name = torch.cuda.get_device_name(ds.device).replace(" ", "_")
    key = f"{name}|bound_tuples_{'refract' if refract else 'reflect'}|cells_2^{size_class(n_base)}"
    if use_cache:
        hit = load_cache().get(key)
        if hit is not None:
            return hit
    out = bnb.bound_tuples(ds, depth, **bound_kw)
    stream = torch.cuda.current_stream(ds.device)
    timings = []
    for bt in candidates:
        ts = []
        for k in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bnb.bound_tuples(ds, depth, out=out, sync_check=False, block_threads=bt, **bound_kw)
            b.record(stream)
            b.synchronize()
            if k > 0:
                ts.append(a.elapsed_time(b))
        if int(out.status.item()) != bnb.BNB_OK:
            raise bnb.BnbError("autotune_bound: bound pass status not OK")
        ts.sort()
        timings.append((ts[len(ts) // 2], bt))
    best = min(timings)
    entry = {"block_threads": best[1], "ms": best[0], "candidates": [[bt, ms] for ms, bt in sorted(timings, key=lambda x: x[1])]}
    if use_cache:
        store_cache(key, entry)
    return entry

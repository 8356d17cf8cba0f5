"""Benchmark: one step = the whole path (bound -> index -> sample -> solve) over one
synthetic area-lit mirror workload, timed on the GPU with CUDA events.

Workload (N=1): 256^2 mirror heightfield (131,072 triangles, 6 seeded sinusoids
+ U[-0.01,0.01] noise, face-averaged normals), a 0.2 x 0.2 quad light at z=2 as
16 stratified point samples, subdivision depth 3: 134,217,728 (emitter,
triangle, cell) bounds per step; 1024^2 jittered shading points on the receiver
z=+1, 512^2 grid.  Multi-GPU: replicas (each rank runs the same workload;
`value` sums the ranks' work over the slowest rank's time).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on
bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bounded cells/s; caustic shading samples/s at 1e-4 rel err; p50/p99 latency"
WORKLOAD = ("mirror256: 256^2 mirror heightfield (131,072 tris, 6 sinusoids + noise 0.01), area light "
            "0.2x0.2 at z=2 as 16 stratified samples, depth 3 (134,217,728 cells/step), 1024^2 shading "
            "points, grid 512, reflection, FP32 with outward rounding")


# ----------------------------------------------------------------------------- algorithmic work
def nc(n: int) -> int:
    return (n + 1) * (n + 2) // 2


def bound_fma_per_cell() -> int:
    """FMAs of the canonical scaled-Bernstein value chain of one reflection cell (products as
    convolutions: nc(M)*nc(N) FMAs), excluding error tracking and ratio logic."""
    f = 0
    f += 2 * 3 * nc(1) * nc(1)                          # n.n, d0.n
    f += 3 * 2 * nc(2) * nc(1)                          # d~ = (n.n) d0 - 2 (d0.n) n
    f += 2 * (3 * nc(1) * nc(0) + 3 * 2 * nc(1) * nc(0))  # D(n.n), D(d0.n) along 2 edges
    f += 2 * 3 * (2 * nc(1) * nc(1) + 2 * nc(2) * nc(0))  # D d~
    f += 3 * nc(3) + 2 * 3 * nc(2)                      # Q, DQ
    f += 2 * 3 * nc(3) * nc(1)                          # A, B
    f += 2 * 2 * 3 * (nc(2) * nc(1) + nc(3) * nc(0))    # DA, DB
    f += 2 * nc(3) * nc(3) + nc(3) * nc(6)              # X, Q X
    f += 2 * (2 * nc(3) * nc(2) + nc(4) * nc(5))        # Y, B Y, Z, A Z
    f += 3 * nc(1) * nc(1)                              # s = d0.d0
    f += nc(3) * nc(3) + nc(6) * nc(3)                  # Q^2, Q^3
    f += 3 * nc(9) * nc(2)                              # N0, N1 and the elevated M per output coefficient
    return f


BOUND_FLOP_PER_CELL = 2 * bound_fma_per_cell()


def pair_fma_per_record() -> int:
    """FMAs of the value chain of one two-vertex record (tuple construction's candidate, composite
    position bound with the degree reduction of u2), excluding error tracking and ratio logic."""
    def refract_faces():  # degree-1 n, d -> the two faces of d~ (degree 5)
        f = 3 * 3 * nc(1) * nc(1)               # n.n, d.n, d.d
        f += 2 * nc(2) * nc(2) + 2 * nc(4)      # beta
        f += 3 * 2 * nc(2) * nc(1) + 3 * nc(3)  # eta' ((n.n) d - (d.n) n)
        f += 2 * (nc(4) + 3 * nc(4) * nc(1))    # W_j = a beta + b_j, d~ = T - W_j n
        return f
    f = refract_faces()                         # first vertex
    f += 2 * 3 * 2 * nc(1)                      # e22 x w2, w2 x e21
    f += 2 * (3 * nc(5) + 2 * 3 * nc(5) * nc(1))  # Q2, A2, B2 on both xi1 faces
    f += 2 * 2 * nc(1) * nc(5)                  # remainder numerators P2 - l Q2
    f += 3 * 2 * 2 * nc(1) + 3 * nc(1)          # x2, n2 from (u2, v2); d1 = x2 - x1
    f += refract_faces()                        # second vertex
    f += 2 * 3 * 2 * nc(1)                      # receiver h_u, h_v
    f += 2 * (3 * nc(5) + 2 * 3 * nc(5) * nc(1))  # Q3, A3, B3 on both xi2 faces
    return f


PAIR_FLOP_PER_RECORD = 2 * pair_fma_per_record()


def refract_fma_per_cell():
    """(position, irradiance) FMAs of the value chain of one single-refraction cell, in the kernel's
    order (products as convolutions: nc(M)*nc(N) FMAs; a pair p0 + W p1 with W^2 -> beta costs the
    four cross products plus the beta product), excluding error tracking and ratio logic.  Every
    cell not in total internal reflection pays the position part; live cells pay the irradiance
    part (the derivative-aware degree-17 bound over four faces)."""
    mac = lambda m, n: nc(m) * nc(n)

    def wp(m, n):
        return mac(m, n) + mac(m - 2, n - 2) + mac(m + n - 4, 4) + mac(m, n - 2) + mac(m - 2, n)
    pos = 3 * 3 * mac(1, 1) + 2 * mac(2, 2) + 2 * nc(4)             # n.n, d0.n, d0.d0, beta
    pos += 3 * (2 * mac(2, 1) + nc(3))                              # eta' ((n.n) d0 - (d0.n) n)
    pos += 3 * 4 * nc(1)                                            # receiver h_u, h_v
    pos += 2 * (nc(4) + 3 * (mac(4, 1) + nc(5) + 2 * mac(5, 1)))    # both faces: W_j, d~, Q, A, B
    pos += 3 * nc(1)                                                # forward cull
    per_edge = 3 * 4 * nc(1) + 2 * mac(1, 2) + nc(3) + mac(2, 1) + nc(3)
    per_edge += 3 * (2 * mac(1, 1) + 2 * mac(2, 0) + nc(2) + mac(3, 1) + nc(4))  # 2W-scaled d d~
    irr = 2 * per_edge
    irr += 3 * (nc(3) + nc(1) + 2 * (mac(3, 1) + mac(1, 1)))        # Q, A, B as pairs
    irr += 2 * 3 * (nc(4) + nc(2) + 2 * (mac(4, 1) + mac(2, 1)) + nc(1) + 2 * nc(1) + 2 * mac(1, 4) + 2 * nc(3))
    irr += 2 * wp(5, 5) + wp(3, 10) + 2 * wp(5, 4) + wp(4, 9) + 2 * wp(4, 5) + wp(4, 9)  # M'
    irr += wp(3, 3) + wp(6, 3) + 2 * nc(2)                          # Q^3, s^-3/2 chord faces
    irr += 2 * (nc(4) + mac(4, 11) + mac(4, 7) + mac(11, 4) + 2 * mac(15, 2))  # W faces, N, den
    return pos, irr


REFRACT_FMA_POS, REFRACT_FMA_IRR = refract_fma_per_cell()


# Algorithmic bytes of the HBM-bound stages: the index reads a live cell's box, E_hi and flags
# (24 B; 4 B of flags for the others), a tuple's key once (12 B), and writes 12 B (key, E~) per
# (grid cell, tuple) entry plus the offsets; the sampling pass reads 12 B per listed entry and
# writes 16 B per selection (point, key, P), the solve reads 72 B of geometry + 12 B of emitter per
# selection and writes 4 B; per point 8 B of coordinates + 4 B of estimate.
INDEX_BYTES_LIVE, INDEX_BYTES_TUPLE, INDEX_BYTES_ENTRY = 24, 12, 12
SAMPLE_BYTES_LISTED, SOLVE_BYTES_SELECTED, SAMPLE_BYTES_POINT = 12, 16 + 72 + 12 + 4, 12


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    return sms * 128 * 2 * mhz * 1e6 / 1e12


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.rows.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------- reference arm (oracle)
# Per-point work of the workload: mean |U| (listed tuples) and |S| (selected, gamma calibrated to
# E|S| = 4) per shading point, as measured by the GPU arm on this workload; used to extrapolate the
# oracle's per-draw and per-solve costs to a full step.
U_PER_POINT = 144.0
S_PER_POINT = 4.0


def oracle_step_sample(sc, cells: int, points: int, seed: int, n_threads: int):
    """One bounded sample of the workload through the FP64 oracle: `cells` contiguous base cells
    (bound + index) and up to `points` shading points whose grid cells list sampled tuples
    (Algorithm 1 draws over their lists + Newton on every listed tuple).
    Returns (s per cell, s per draw, s per solve, description)."""
    import copy

    import oracle
    rng = np.random.default_rng(seed)
    per = 4 ** sc.depth
    n_base = sc.emitters.n * sc.s1.n_tris * per
    t0_tuple = int(rng.integers(0, n_base // per - cells // per))
    work = np.arange(t0_tuple * per, t0_tuple * per + cells, dtype=np.int64)
    t0 = time.perf_counter()
    rec = oracle.bound(sc, work=work, n_threads=n_threads)
    f = oracle.records_to_f32(rec)
    off, key, et = oracle.index(f["u_lo"], f["u_hi"], f["v_lo"], f["v_hi"], f["e_hi"], f["emitter"], f["tri0"],
                                f["tri1"], f["flags"], sc.grid_res)
    t1 = time.perf_counter()
    G = sc.grid_res
    g = np.clip(np.floor(sc.sv * np.float32(G)), 0, G - 1).astype(np.int64) * G + \
        np.clip(np.floor(sc.su * np.float32(G)), 0, G - 1).astype(np.int64)
    pick = np.nonzero(np.diff(off)[g] > 0)[0][:points]
    su, sv = sc.su[pick], sc.sv[pick]
    t2 = time.perf_counter()
    wp, wk, wP, n_u = oracle.sample(off, key, et, G, su, sv, 1e30, seed)
    t3 = time.perf_counter()
    sc2 = copy.copy(sc)
    sc2.su, sc2.sv = su, sv
    oracle.solve(sc2, wp, wk, wP, n_threads=n_threads)
    t4 = time.perf_counter()
    return ((t1 - t0) / cells, (t3 - t2) / max(1, n_u), (t4 - t3) / max(1, wp.shape[0]),
            f"{cells} contiguous base cells (bound+index, {t1 - t0:.2f} s), {n_u} draws over {len(pick)} points "
            f"({t3 - t2:.3f} s), {wp.shape[0]} Newton solves ({t4 - t3:.2f} s)")


def oracle_step_seconds(sc, t_cell, t_draw, t_solve, u_per_point=U_PER_POINT, s_per_point=S_PER_POINT):
    n_cells = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
    n_points = sc.su.shape[0]
    return n_cells * t_cell + n_points * (u_per_point * t_draw + s_per_point * t_solve)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2504_19163_gb300 import scenes as S
    oracle.build()
    sc = S.config("mirror256")
    n_threads = os.cpu_count() or 1
    n_cells_full = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
    n_points_full = sc.su.shape[0]
    per = 4 ** sc.depth
    cells = -(-n_cells_full // 100 // per) * per  # >= 1% of the cells per step, whole tuples
    points = 1024
    for i in range(args.warmup):
        oracle_step_sample(sc, cells, points, 100 + i, n_threads)
    acc = np.zeros(3)
    desc = ""
    for i in range(args.steps):
        a, b, c, desc = oracle_step_sample(sc, cells, points, 1000 + i, n_threads)
        acc += (a, b, c)
    t_cell, t_draw, t_solve = acc / args.steps
    step_s = oracle_step_seconds(sc, t_cell, t_draw, t_solve)
    value = n_cells_full / step_s
    line = {"impl": "reference", "extrapolated": True,
            "extrapolation": f"each step times the oracle on {cells} seeded contiguous base cells ({cells / n_cells_full:.2%} "
                             f"of the workload) and on the draws and solves of {points} points; the step time is "
                             f"extrapolated to all {n_cells_full} cells and {n_points_full} points",
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": n_threads, "kind": "oracle",
                             "sample": f"per step: {desc}; extrapolated to {n_cells_full} cells and "
                                       f"{n_points_full} points x ({U_PER_POINT} draws + {S_PER_POINT} solves)"},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "shading_samples_per_s": n_points_full / step_s}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    from paper_2504_19163_gb300 import bnb, build
    from paper_2504_19163_gb300 import scenes as S

    from paper_2504_19163_gb300 import replicas as RP
    rank, local, world = RP.rank_env()
    torch.cuda.set_device(local)
    dist = RP.init("nccl", torch.device("cuda", local))
    build.build()
    dev = torch.device("cuda", local)
    sc = S.config("mirror256")
    if args.emitters and args.emitters < sc.emitters.n:
        # smaller case of the same workload (profiling): the first N area-light samples
        e = sc.emitters
        sc.emitters = S.Emitters(e.x[:args.emitters], e.y[:args.emitters], e.z[:args.emitters],
                                 e.intensity[:args.emitters])
    ds = bnb.DeviceScene(sc, dev)
    n_cells = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
    n_points = ds.n_points
    stream = torch.cuda.current_stream(dev)

    # Block size of the bound pass: the autotuner times its compiled schedules on this workload.
    from paper_2504_19163_gb300 import batch as BA
    sched = BA.autotune_bound(ds, sc.depth, use_cache=False, with_e_lo=False)
    bt = int(sched["block_threads"])
    # Buffers sized once (first call discovers the capacities), then reused every step.
    cb = bnb.bound_tuples(ds, sc.depth, with_e_lo=False, block_threads=bt)  # the index needs E_hi only
    idx = bnb.build_index(cb, grid_res=sc.grid_res)
    # gamma: expected |S| of about 4 per shading point (paper's Plane scene: |S| = 3.4)
    gamma = calibrate_gamma(bnb, ds, idx, target=4.0)
    res = bnb.sample_and_solve(ds, idx, gamma, 1)
    torch.cuda.synchronize()
    wl_cap = int(res.counters[1].item()) * 2 + 4096
    cb_ws = bnb._ws(bnb.bnb_bound_tuples_ws(bnb.C.byref(ds.s1), None, bnb.C.byref(ds.em),
                                            bnb.C.byref(bnb.bnb_bound_cfg(sc.depth, 4, 1, 0))), dev)
    pre_cap = int(idx.count[1].item()) + idx.count[1].item() // 4 + 4096
    ix_ws = bnb._ws(bnb.bnb_build_index_ws(bnb.C.byref(cb.c), sc.grid_res, pre_cap), dev)
    idx = bnb.Index(sc.grid_res, pre_cap, dev)
    sm_ws = bnb._ws(bnb.bnb_sample_and_solve_ws(bnb.C.byref(ds.s1), None, n_points, wl_cap), dev)
    E_out = torch.empty(n_points, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(seed, ev=None):
        if ev is not None:
            ev[0].record(stream)
        bnb.bound_tuples(ds, sc.depth, out=cb, ws=cb_ws, sync_check=False, block_threads=bt)
        if ev is not None:
            ev[1].record(stream)
        bnb.build_index(cb, grid_res=sc.grid_res, pre_capacity=pre_cap, capacity=pre_cap, out=idx, ws=ix_ws,
                        sync_check=False)
        if ev is not None:
            ev[2].record(stream)
        r = bnb.sample_and_solve(ds, idx, gamma, seed, worklist_capacity=wl_cap, E_out=E_out, ws=sm_ws,
                                 sync_check=False)
        if ev is not None:
            ev[3].record(stream)
        return r

    for i in range(args.warmup):
        step(1000 + i)
    torch.cuda.synchronize()
    st_ok = int(cb.status.item()) == 0 and int(idx.status.item()) == 0
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    RP.barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps
        for i in range(args.steps):
            flush.zero_()  # L2 flush (256 MiB > 129 MB L2) outside the timed events
            r = step(i, evs[i])
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    RP.barrier(dist)
    stage = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])] for e in evs])
    ms_step = float(stage.sum(axis=1).mean())
    st_ok = st_ok and int(cb.status.item()) == 0 and int(idx.status.item()) == 0 and int(r.status.item()) == 0
    counters = r.counters.cpu().numpy()
    ms_max = RP.max_over_ranks(ms_step, dist, dev)
    value = RP.whole_job_rate(n_cells, world, ms_max)

    # ---- end to end through the public API with host buffers (pinned), copies inside the region
    host = {k: v.cpu().pin_memory() for k, v in ds.t.items()}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    E_host = torch.empty(n_points, dtype=torch.float32).pin_memory()
    d2h = E_host.numel() * 4
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for i in range(e2e_steps):
        flush.zero_()
        e0.record(stream)
        for k, v in host.items():
            ds.t[k].copy_(v, non_blocking=True)
        step(500 + i)
        E_host.copy_(E_out, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms /= e2e_steps
    e2e_value = RP.whole_job_rate(n_cells, world, RP.max_over_ranks(e2e_ms, dist, dev))

    # ---- bin-packed selection (Sec. 5.3) on the same index: one draw per group instead of per tuple
    bev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(8)]
    for i in range(8):
        flush.zero_()
        bev[i][0].record(stream)
        rb = bnb.sample_and_solve(ds, idx, gamma, 900 + i, worklist_capacity=wl_cap, E_out=E_out, ws=sm_ws,
                                  sync_check=False, bins=True)
        bev[i][1].record(stream)
    torch.cuda.synchronize()
    cb_n = rb.counters.cpu().numpy()
    bins_line = {"sample_solve_ms": float(np.mean([e[0].elapsed_time(e[1]) for e in bev[3:]])),
                 "per_point": {"U": cb_n[0] / n_points, "B": cb_n[3] / n_points, "S": cb_n[1] / n_points,
                               "roots": cb_n[2] / n_points},
                 "status_ok": int(rb.status.item()) == 0}
    # ---- stochastic Newton starts with the reciprocal weighting (Sec. 6.1 "Stoc"), weights capped at 64
    for i in range(8):
        flush.zero_()
        bev[i][0].record(stream)
        rs = bnb.sample_and_solve(ds, idx, gamma, 700 + i, worklist_capacity=wl_cap, E_out=E_out, ws=sm_ws,
                                  sync_check=False, stoc_trials=64)
        bev[i][1].record(stream)
    torch.cuda.synchronize()
    cs_n = rs.counters.cpu().numpy()
    stoc_line = {"sample_solve_ms": float(np.mean([e[0].elapsed_time(e[1]) for e in bev[3:]])),
                 "stoc_trials": 64, "per_point": {"S": cs_n[1] / n_points, "roots": cs_n[2] / n_points},
                 "status_ok": int(rs.status.item()) == 0}

    # ---- measured FP32 FMA throughput (the ALU roofline's measured denominator)
    peak_info = fp32_peak_summary(dev, local)

    # ---- roofline of the dominant kernel (bound pass)
    bound_ms = float(stage[:, 0].mean())
    props = torch.cuda.get_device_properties(dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    achieved = BOUND_FLOP_PER_CELL * n_cells / (bound_ms / 1e3) / 1e12
    traffic = bound_traffic()
    # HBM accounting of the other stages (algorithmic bytes over their CUDA-event stage times)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    n_rec = cb.n_records()
    n_live = int(((cb.flags[:n_rec] & 1) != 0).sum().item())
    n_entries = int(idx.count[0].item())
    n_tuples = sc.emitters.n * sc.s1.n_tris
    index_bytes = INDEX_BYTES_LIVE * n_live + 4 * (n_rec - n_live) + INDEX_BYTES_TUPLE * n_tuples + \
        INDEX_BYTES_ENTRY * n_entries + 8 * (sc.grid_res ** 2 + 1)
    ss_bytes = SAMPLE_BYTES_LISTED * float(counters[0]) + SOLVE_BYTES_SELECTED * float(counters[1]) + \
        SAMPLE_BYTES_POINT * n_points
    stage_ms = {"bound": bound_ms, "index": float(stage[:, 1].mean()), "sample_solve": float(stage[:, 2].mean())}
    stage_roofline = {
        "index": {"bound": "hbm", "bytes": index_bytes, "achieved": index_bytes / (stage_ms["index"] / 1e3) / 1e9,
                  "peak": hbm, "unit": "GB/s", "live_cells": n_live, "entries": n_entries},
        "sample_solve": {"bound": "hbm", "bytes": ss_bytes,
                         "achieved": ss_bytes / (stage_ms["sample_solve"] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s"}}
    for v in stage_roofline.values():
        v["frac"] = v["achieved"] / v["peak"]

    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if sc.emitters.n == 16 else
                       WORKLOAD.replace("16 stratified samples", f"{sc.emitters.n} of 16 stratified samples"),
                       "parallelism": f"replicas x{world}" if world > 1 else "single",
                       "l2": "flushed between steps (256 MiB write, outside the events)",
                       "gamma": gamma, "cells_per_step": n_cells, "points_per_step": n_points,
                       "bound_schedule": sched,
                       "status_ok": st_ok},
            "shading_samples_per_s": n_points * world / (ms_max / 1e3),
            "stage_ms": stage_ms,
            "stage_roofline": stage_roofline,
            "per_point": {"U": counters[0] / n_points, "S": counters[1] / n_points, "roots": counters[2] / n_points},
            "roofline": {"bound": "alu", "kernel": "bound_base_k<float>", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                         "flop_per_cell": BOUND_FLOP_PER_CELL,
                         "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                       f"(max SM clock of MEASURED_PEAKS.json)",
                         "peak_measured": peak_info["peak"], "frac_of_measured": achieved / peak_info["peak"],
                         "peak_measured_basis": "bnb_ffma_probe: FFMA and paired FFMA2 chains over 8 x 256-thread "
                                                "blocks per SM, ~1 s each (the larger; see fp32_peak)"},
            "fp32_peak": peak_info,
            "bins": bins_line,
            "stoc": stoc_line,
            "e2e": {"value": e2e_value, "unit": "cells/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": launches_per_step(n_points, sc.grid_res) * args.steps,
            "clocks": clk.summary()}
    if not args.no_cpu_baseline and rank == 0 and world == 1 and not args.emitters:
        try:  # part of the CPU-baseline leg: the oracle runs in a spawned child
            cb = None
            torch.cuda.empty_cache()
            line["accuracy"] = accuracy_summary(bnb, ds, sc, idx, gamma, dev)
        except Exception as ex:  # reported in the line; the bound benchmark above stands
            line["accuracy"] = {"error": f"{type(ex).__name__}: {ex}"}
    if args.serving_requests > 0 and rank == 0 and world == 1 and not args.emitters:
        cb = idx = cb_ws = ix_ws = sm_ws = flush = None
        torch.cuda.empty_cache()
        line["serving"] = serving_summary(args.serving_requests, dev)
    if args.adaptive_steps > 0 and rank == 0 and world == 1 and not args.emitters:
        try:
            line["adaptive"] = adaptive_summary(dev, args.adaptive_steps)
            if args.adaptive_sweep_steps > 0:
                line["adaptive_sweep"] = adaptive_sweep(dev, args.adaptive_sweep_steps)
        except Exception as ex:  # reported in the line; the bound benchmark above stands
            line["adaptive"] = {"error": f"{type(ex).__name__}: {ex}"}
    if args.implicit_steps > 0 and rank == 0 and world == 1 and not args.emitters:
        try:
            line["implicit"] = implicit_summary(dev, args.implicit_steps)
        except Exception as ex:  # reported in the line; the bound benchmark above stands
            line["implicit"] = {"error": f"{type(ex).__name__}: {ex}"}
    if args.pairs_steps > 0 and rank == 0 and world == 1:
        try:
            line["pairs"] = pairs_summary(dev, args.pairs_steps, not args.no_cpu_baseline and not args.emitters)
        except Exception as ex:  # reported in the line; the bound benchmark above stands
            line["pairs"] = {"error": f"{type(ex).__name__}: {ex}"}
    if args.refraction_steps > 0 and rank == 0 and world == 1 and not args.emitters:
        try:
            line["refraction"] = refraction_summary(dev, args.refraction_steps, peak, peak_info["peak"])
        except Exception as ex:  # reported in the line; the bound benchmark above stands
            line["refraction"] = {"error": f"{type(ex).__name__}: {ex}"}
    if args.rough_steps > 0 and rank == 0 and world == 1 and not args.emitters:
        try:
            line["rough"] = rough_summary(dev, args.rough_steps)
        except Exception as ex:  # reported in the line; the bound benchmark above stands
            line["rough"] = {"error": f"{type(ex).__name__}: {ex}"}
    if not args.no_cpu_baseline and rank == 0 and world == 1 and not args.emitters:
        line["cpu_baseline"] = cpu_baseline(counters[0] / n_points, counters[1] / n_points)
    if rank == 0:
        print(json.dumps(line), flush=True)
    RP.finish(dist)
    return 0


def scan_launches(n: int) -> int:
    tiles = (n + 2047) // 2048
    if tiles <= 1:
        return 2
    return 1 + scan_launches(tiles) + 2


BOUND_SOURCES = ("paper_2504_19163_gb300/csrc/bnb_bound_impl.cuh", "paper_2504_19163_gb300/csrc/bnb_poly.cuh")


def bound_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in BOUND_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def bound_traffic():
    """DRAM bytes per launch of the bound kernel from the committed ncu capture, or None when the
    kernel sources changed since the counters were taken."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "bound_traffic.json")))
    except Exception:
        return None
    if d.get("sources_sha256") != bound_sources_sha():
        return None
    return d.get("bytes_per_launch")


def launches_per_step(n_points: int, G: int) -> int:
    bound = 1 + 1 + 4                                # pack, base, 4 split levels
    # merge, overflow, scan, scatter, rank/warp sort, block sort, big-cell sort, scan, compact, count
    index = 2 + scan_launches(G * G) + 4 + scan_launches(G * G) + 2
    # pack, list-length mode, count (thread and warp forms: one returns at once), scan, fill (both
    # forms), solve32 + polish, reduce
    sample = 1 + 1 + 2 + scan_launches(n_points) + 2 + 2 + 1
    return bound + index + sample


def calibrate_gamma(bnb, ds, idx, target: float) -> float:
    """gamma such that the mean expected |S| over the workload's shading points is `target`
    (Sec. 5.4: one-to-one map between gamma and E|S|), by the library's device bisection."""
    return float(bnb.gamma_for_target(idx, target, ds.t["su"], ds.t["sv"]).item())


def serving_summary(n_requests: int, dev) -> dict:
    """The request workload served by the continuous-batching loop next to the plain per-request
    paths (p50/p99 latency, shading samples/s); outside the timed region of the bound benchmark."""
    from paper_2504_19163_gb300 import serving as SV
    try:
        res = SV.run_workload(n_requests, device=dev, log=lambda *a: None)
    except Exception as ex:  # reported in the line; the bound benchmark above stands
        return {"error": f"{type(ex).__name__}: {ex}"}
    keep = ("p50_ms", "p99_ms", "samples_per_s", "requests_per_s", "mean_batch", "traces")
    out = {"workload": res["workload"], "capacity_req_per_s": res["capacity_req_per_s"],
           "served_equals_alone": res["served_equals_alone"], "autotuned_launch": res.get("autotuned_launch"),
           "scene_build_s": res["scene_build_s"]}
    for tag in ("load_plain", "load_cached", "burst"):
        b = res[tag]
        out[tag] = {"arrival_rate_req_per_s": b["arrival_rate_req_per_s"]}
        for m in ("plain", "plain_cached", "served"):
            if m in b:
                out[tag][m] = {k: b[m][k] for k in keep if k in b[m]}
    return out


def pairs_summary(dev, steps: int, oracle_too: bool) -> dict:
    """The two-vertex workload (slab48: glass slab, two 48^2 faces, 512^2 points, depth 2), run after
    the main timed region: bound pass (s2 grid, tuple construction, composite position bounds, chain
    irradiance bounds), index, rendering pass with gamma for E|S| = |U| / 2 (the chain bounds make
    P < 1), each timed with CUDA events over `steps` steps after 3 warm-up steps, with a 256 MiB L2
    flush between steps; then the bound pass without the irradiance post-pass, timed the same way."""
    import torch
    from paper_2504_19163_gb300 import bnb
    from paper_2504_19163_gb300 import scenes as S
    sc = S.config("slab48")
    ds = bnb.DeviceScene(sc, dev)
    stream = torch.cuda.current_stream(dev)
    cb = bnb.bound_tuples(ds, sc.depth, with_e_lo=False)
    idx = bnb.build_index(cb, grid_res=sc.grid_res)
    res = bnb.sample_and_solve(ds, idx, float("inf"), 1)
    torch.cuda.synchronize()
    n_points = ds.n_points
    n_base = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
    wl_cap = int(res.counters[1].item()) * 2 + 4096
    U_all = float(res.counters[0].item()) / n_points
    gamma = calibrate_gamma(bnb, ds, idx, target=0.5 * U_all)
    cfg = bnb.bnb_bound_cfg(sc.depth, 0, 1, 0)
    cb_ws = bnb._ws(bnb.bnb_bound_tuples_ws(bnb.C.byref(ds.s1), ds.s2_ref(), bnb.C.byref(ds.em),
                                            bnb.C.byref(cfg)), dev)
    pre_cap = int(idx.count[1].item()) + int(idx.count[1].item()) // 4 + 4096
    ix_ws = bnb._ws(bnb.bnb_build_index_ws(bnb.C.byref(cb.c), sc.grid_res, pre_cap), dev)
    idx = bnb.Index(sc.grid_res, pre_cap, dev)
    sm_ws = bnb._ws(bnb.bnb_sample_and_solve_ws(bnb.C.byref(ds.s1), ds.s2_ref(), n_points, wl_cap), dev)
    E_out = torch.empty(n_points, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(seed, ev):
        ev[0].record(stream)
        bnb.bound_tuples(ds, sc.depth, out=cb, ws=cb_ws, sync_check=False)
        ev[1].record(stream)
        bnb.build_index(cb, grid_res=sc.grid_res, pre_capacity=pre_cap, capacity=pre_cap, out=idx, ws=ix_ws,
                        sync_check=False)
        ev[2].record(stream)
        r = bnb.sample_and_solve(ds, idx, gamma, seed, worklist_capacity=wl_cap, E_out=E_out, ws=sm_ws,
                                 sync_check=False)
        ev[3].record(stream)
        return r

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(3 + steps)]
    for i in range(3 + steps):
        if i == 3:
            torch.cuda.nvtx.range_push("pairs")  # lets a profiler select the timed steps
        flush.zero_()
        r = step(i, evs[i])
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    st = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])] for e in evs[3:]])
    ok = int(cb.status.item()) == 0 and int(idx.status.item()) == 0 and int(r.status.item()) == 0
    flags = cb.flags[: cb.n_records()]
    n_rec = cb.n_records()
    live = int(((flags & 1) != 0).sum().item())
    c = r.counters.cpu().numpy()
    ms = st.mean(axis=0)
    n_finite = int((((flags & 1) != 0) & torch.isfinite(cb.e_hi[:n_rec])).sum().item())
    # the bound pass without the chain irradiance post-pass (position bounds only)
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(3 + steps)]
    for i in range(3 + steps):
        flush.zero_()
        pev[i][0].record(stream)
        bnb.bound_tuples(ds, sc.depth, out=cb, ws=cb_ws, sync_check=False, irradiance=False)
        pev[i][1].record(stream)
    torch.cuda.synchronize()
    pos_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in pev[3:]]))
    props = torch.cuda.get_device_properties(dev)
    try:
        sm_max = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2070.0))
    except Exception:
        sm_max = 2070.0
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    achieved = PAIR_FLOP_PER_RECORD * n_rec / (pos_ms / 1e3) / 1e12
    out = {"workload": "slab48: glass slab (ior 1.5), two 48^2 heightfield faces (4608 tris each), point light "
                       "(0,0,2), receiver z=-1, 512^2 shading points, depth 2 (73,728 base cells), FP32",
           "status_ok": ok, "steps": steps, "base_cells": n_base, "pair_records": n_rec, "live_records": live,
           "live_records_finite_e_hi": n_finite, "gamma": gamma, "gamma_target": "E|S| = |U| / 2",
           "bound_position_only_ms": pos_ms, "chain_irradiance_ms": float(ms[0]) - pos_ms,
           "records_per_base_cell": n_rec / n_base,
           "stage_ms": {"bound": float(ms[0]), "index": float(ms[1]), "sample_solve": float(ms[2])},
           "pair_records_per_s": n_rec / (ms[0] / 1e3), "base_cells_per_s": n_base / (ms[0] / 1e3),
           "shading_samples_per_s": n_points / (ms[2] / 1e3),
           "per_point": {"U": c[0] / n_points, "S": c[1] / n_points, "roots": c[2] / n_points},
           "roofline": {"bound": "alu", "kernel": "pair bound stage without the irradiance post-pass (s2 grid, "
                                                 "candidates, pair_bound_k<float>)",
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "flop_per_record": PAIR_FLOP_PER_RECORD}}
    del cb, idx, cb_ws, ix_ws, sm_ws, flush
    torch.cuda.empty_cache()
    if oracle_too:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(1) as pool:
            out["oracle"] = pool.apply(_pairs_oracle_worker, ())
    return out


ADAPT = dict(depth=0, adapt_depth=6, sigma=1e-6, alpha=2.0)


def fp32_peak_summary(dev, gpu_index: int) -> dict:
    """Measured FP32 FMA throughput (bnb_ffma_probe, scalar FFMA and paired FFMA2 over a resident
    grid, ~1 s each, CUDA events) with the SM clocks sampled while it ran."""
    from paper_2504_19163_gb300 import bnb
    with ClockSampler(gpu_index) as clk:
        r = bnb.fp32_fma_peak(dev, seconds=1.0)
    r["clocks"] = clk.summary()
    return r


def refraction_summary(dev, steps: int, peak_tflops: float, peak_measured) -> dict:
    """The refraction workload (water420: 420^2 Gerstner water, 352,800 triangles, eta' = 1/1.33, 4
    point lights, pool floor 1 below, 1920x1080 shading points, depth 3: 90,316,800 cells per step):
    bound pass with irradiance, index, gamma for E|S| = 4 (library bisection), rendering pass; each
    stage timed with CUDA events over `steps` steps after 3 warm-up steps, L2 flushed between steps."""
    import torch
    from paper_2504_19163_gb300 import bnb
    from paper_2504_19163_gb300 import scenes as S
    sc = S.config("water420")
    ds = bnb.DeviceScene(sc, dev)
    stream = torch.cuda.current_stream(dev)
    from paper_2504_19163_gb300 import batch as BA
    sched = BA.autotune_bound(ds, sc.depth, reps=2, use_cache=False, with_e_lo=False)
    bt = int(sched["block_threads"])
    cb = bnb.bound_tuples(ds, sc.depth, with_e_lo=False, block_threads=bt)
    idx = bnb.build_index(cb, grid_res=sc.grid_res)
    gamma = calibrate_gamma(bnb, ds, idx, target=4.0)
    res = bnb.sample_and_solve(ds, idx, gamma, 1)
    torch.cuda.synchronize()
    n_points = ds.n_points
    n_cells = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
    wl_cap = int(res.counters[1].item()) * 2 + 4096
    cb_ws = bnb._ws(bnb.bnb_bound_tuples_ws(bnb.C.byref(ds.s1), None, bnb.C.byref(ds.em),
                                            bnb.C.byref(bnb.bnb_bound_cfg(sc.depth, 4, 1, 0))), dev)
    pre_cap = int(idx.count[1].item()) + int(idx.count[1].item()) // 4 + 4096
    ix_ws = bnb._ws(bnb.bnb_build_index_ws(bnb.C.byref(cb.c), sc.grid_res, pre_cap), dev)
    idx = bnb.Index(sc.grid_res, pre_cap, dev)
    sm_ws = bnb._ws(bnb.bnb_sample_and_solve_ws(bnb.C.byref(ds.s1), None, n_points, wl_cap), dev)
    E_out = torch.empty(n_points, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(seed, ev):
        ev[0].record(stream)
        bnb.bound_tuples(ds, sc.depth, out=cb, ws=cb_ws, sync_check=False, block_threads=bt)
        ev[1].record(stream)
        bnb.build_index(cb, grid_res=sc.grid_res, pre_capacity=pre_cap, capacity=pre_cap, out=idx, ws=ix_ws,
                        sync_check=False)
        ev[2].record(stream)
        r = bnb.sample_and_solve(ds, idx, gamma, seed, worklist_capacity=wl_cap, E_out=E_out, ws=sm_ws,
                                 sync_check=False)
        ev[3].record(stream)
        return r

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(3 + steps)]
    for i in range(3 + steps):
        if i == 3:
            torch.cuda.nvtx.range_push("refraction")
        flush.zero_()
        r = step(i, evs[i])
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    st = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])] for e in evs[3:]])
    ms = st.mean(axis=0)
    ok = int(cb.status.item()) == 0 and int(idx.status.item()) == 0 and int(r.status.item()) == 0
    n_rec = cb.n_records()
    fl = cb.flags[:n_rec]
    n_tir = int(((fl & 128) != 0).sum().item())
    live = (fl & 1) != 0
    n_live = int(live.sum().item())
    n_live_finite = int((live & torch.isfinite(cb.e_hi[:n_rec])).sum().item())
    fma = REFRACT_FMA_POS * (n_rec - n_tir) + REFRACT_FMA_IRR * n_live
    achieved = 2.0 * fma / (ms[0] / 1e3) / 1e12
    c = r.counters.cpu().numpy()
    out = {"workload": "water420: 420^2 Gerstner water (352,800 tris, 16 waves), eta' 1/1.33, 4 point lights at "
                       "(+-0.5,+-0.5,2), pool floor z=-1, 1920x1080 shading points, depth 3 (90,316,800 cells/step), "
                       "grid 512, FP32 with outward rounding",
           "status_ok": ok, "steps": steps, "cells_per_step": n_cells, "records": n_rec, "live_records": n_live,
           "live_finite_e_hi": n_live_finite, "tir_records": n_tir, "gamma": gamma, "bound_schedule": sched,
           "stage_ms": {"bound": float(ms[0]), "index": float(ms[1]), "sample_solve": float(ms[2])},
           "ms_per_step": float(ms.sum()), "cells_per_s": n_cells / (float(ms.sum()) / 1e3),
           "bound_cells_per_s": n_cells / (ms[0] / 1e3), "shading_samples_per_s": n_points / (float(ms.sum()) / 1e3),
           "per_point": {"U": c[0] / n_points, "S": c[1] / n_points, "roots": c[2] / n_points},
           "roofline": {"bound": "alu", "kernel": "bound_base_k<float, refraction> (+ its split levels)",
                        "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                        "fma_position_per_cell": REFRACT_FMA_POS, "fma_irradiance_per_live_cell": REFRACT_FMA_IRR,
                        "flop_per_launch": 2.0 * fma}}
    if peak_measured:
        out["roofline"]["peak_measured"] = peak_measured
        out["roofline"]["frac_of_measured"] = achieved / peak_measured
    del cb, idx, cb_ws, ix_ws, sm_ws, flush
    torch.cuda.empty_cache()
    return out


def rough_summary(dev, steps: int) -> dict:
    """The bound pass alone on mirror256_rough, the literal per-vertex reading of the noise
    (independent U[-0.01, 0.01] per vertex, slopes up to ~2.5; the index of this reading would hold
    ~1e11 entries, so only the bound pass is timed), beside the smooth-noise benchmark mirror."""
    import torch
    from paper_2504_19163_gb300 import bnb
    from paper_2504_19163_gb300 import scenes as S
    sc = S.config("mirror256_rough")
    ds = bnb.DeviceScene(sc, dev)
    stream = torch.cuda.current_stream(dev)
    cb = bnb.bound_tuples(ds, sc.depth, with_e_lo=False)
    torch.cuda.synchronize()
    cb_ws = bnb._ws(bnb.bnb_bound_tuples_ws(bnb.C.byref(ds.s1), None, bnb.C.byref(ds.em),
                                            bnb.C.byref(bnb.bnb_bound_cfg(sc.depth, 4, 1, 0))), dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(3 + steps)]
    for i in range(3 + steps):
        flush.zero_()
        evs[i][0].record(stream)
        bnb.bound_tuples(ds, sc.depth, out=cb, ws=cb_ws, sync_check=False)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs[3:]]))
    n_cells = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
    n_rec = cb.n_records()
    fl = cb.flags[:n_rec]
    out = {"workload": "mirror256_rough: as mirror256 but noise U[-0.01,0.01] independent per vertex; bound pass only",
           "status_ok": int(cb.status.item()) == 0, "steps": steps, "bound_ms": ms,
           "bound_cells_per_s": n_cells / (ms / 1e3), "records": n_rec,
           "split_records": int(((fl & 2) != 0).sum().item()), "fold_records": int(((fl & 16) != 0).sum().item()),
           "live_records": int(((fl & 1) != 0).sum().item())}
    del cb, cb_ws, flush
    torch.cuda.empty_cache()
    return out


def implicit_fma_per_record() -> int:
    """FMAs of one record of the implicit-differentiation pass: a scaled-Bernstein product of forms
    with m and n coefficients is m * n FMAs, an elevation a product with the constant 1, a scaling
    one FMA per coefficient (the operation sequence of the kernel, both vectors b)."""
    T = lambda n, p, q: (n + 1) * (n + 2) // 2 * (p + 1) * (q + 1)
    mul = lambda a, b: T(*a) * T(*b)
    elev = lambda a, to: T(*a) * T(to[0] - a[0], to[1] - a[1], to[2] - a[2])
    s1, b11, s2 = (1, 0, 0), (0, 1, 1), (2, 0, 0)
    x1e = (1, 1, 1)
    base = 3 * (3 + elev(s1, x1e) + elev(b11, x1e) + 2 * T(*x1e))        # d0, d1
    base += 6 * mul(s1, s1) + 6 * mul(x1e, s1) + 3 * mul(x1e, x1e) + 3 * mul(s1, s1)  # d0n, d1n, L1, L0
    per_dir = 6 * 3 + 12 * 3 + 4 * T(*x1e) + 4 * 3 + 3 * mul(s1, x1e) + 3 * T(*s2) + elev(s2, (2, 1, 1)) + T(2, 1, 1)
    per_rec = 6 * 3 + 4 * T(*x1e) + 3 * T(*s2)
    base += 2 * per_dir + 2 * per_rec
    A, C = s2, (2, 1, 1)
    fd = (2 * T(*x1e) + elev(s1, x1e) + T(*x1e) + mul(x1e, (4, 0, 0)) + elev((5, 1, 1), (5, 2, 2)) + mul(A, s1)
          + T(3, 0, 0) + mul((2, 2, 2), (3, 0, 0)) + mul(s1, (4, 2, 2)) + mul(C, x1e) + mul(s2, (3, 2, 2)))
    fk = mul(x1e, (4, 0, 0)) + mul(C, s1) + mul(s2, (3, 1, 1))
    per_b = (mul(A, A) + T(4, 0, 0) + mul(C, C) + 2 * fd + 2 * fk + 2 * mul((5, 2, 2), (2, 1, 1))
             + 2 * mul((5, 1, 1), s2) + elev((7, 1, 1), (7, 3, 3)))
    return base + 2 * per_b


def implicit_summary(dev, steps: int) -> dict:
    """Implicit-differentiation irradiance bound (Sec. 4.4) near total internal reflection: a
    light under water below a 32^2 heightfield (2048 triangles), a wall receiver, depth 4
    (524,288 base cells); the explicit bound pass, then the intersecting implicit pass over its
    live records, timed alone with CUDA events (L2 flushed between launches)."""
    import torch
    from paper_2504_19163_gb300 import bnb
    from paper_2504_19163_gb300 import scenes as S
    sc = S.config("tir_wall", n=32, depth=4)
    ds = bnb.DeviceScene(sc, dev)
    stream = torch.cuda.current_stream(dev)
    cb = bnb.bound_tuples(ds, sc.depth, irradiance=True)
    torch.cuda.synchronize()
    n_rec = cb.n_records()
    e_hi0 = cb.e_hi[:n_rec].clone()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(3 + steps)]
    for i in range(3 + steps):
        flush.zero_()
        evs[i][0].record(stream)
        bnb.implicit_irradiance(ds, cb, n=-1, mode=1, stream=stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs[3:]]))
    fl = cb.flags[:n_rec]
    live = (fl & 1) != 0
    n_live = int(live.sum().item())
    e1 = cb.e_hi[:n_rec]
    tighter = int(((e1 < 0.5 * e_hi0) & live).sum().item())
    inf_to_finite = int((torch.isinf(e_hi0) & torch.isfinite(e1) & live).sum().item())
    fma = implicit_fma_per_record()
    tflops = 2.0 * fma * n_live / (ms * 1e-3) / 1e12
    return {"workload": "tir_wall 32^2 (2048 tris), depth 4, wall receiver; implicit pass (mode 1) over the live "
                        "records of the explicit pass", "steps": steps, "records": n_rec, "live_records": n_live,
            "ms": round(ms, 3), "live_records_per_s": round(n_live / (ms * 1e-3), 1),
            "fma_per_record": fma, "fp64_tflops": round(tflops, 4),
            "fp64_frac_of_nominal": round(tflops / 1.25, 4), "fp64_peak_note": "nominal 1.25 TFLOP/s FP64 (not measured)",
            "bounds_halved_or_better": tighter, "infinite_to_finite": inf_to_finite}


def adaptive_summary(dev, steps: int, sigma: float = ADAPT["sigma"], alpha: float = ADAPT["alpha"]) -> dict:
    """Adaptive subdivision (Sec. 6.1) on the benchmark mirror: every triangle and light sample
    starts as one cell and is subdivided down to depth 6 until its receiver box has area below
    sigma (1e-6: a quarter of a 512^2 grid cell) or E_hi < alpha E_lo (2: the paper's alpha for
    single scattering); then the index and the rendering pass at E|S| = 4.  Timed like the main
    steps."""
    import torch
    from paper_2504_19163_gb300 import bnb
    from paper_2504_19163_gb300 import scenes as S
    sc = S.config("mirror256")
    ds = bnb.DeviceScene(sc, dev)
    stream = torch.cuda.current_stream(dev)
    kw = dict(adapt_depth=ADAPT["adapt_depth"], sigma=sigma, alpha=alpha, with_e_lo=False)
    cb = bnb.bound_tuples(ds, ADAPT["depth"], **kw)
    split_cap = cb.capacity
    idx = bnb.build_index(cb, grid_res=sc.grid_res)
    gamma = calibrate_gamma(bnb, ds, idx, target=4.0)
    res = bnb.sample_and_solve(ds, idx, gamma, 1)
    torch.cuda.synchronize()
    n_points = ds.n_points
    wl_cap = int(res.counters[1].item()) * 2 + 4096
    cfg = bnb.bnb_bound_cfg(ADAPT["depth"], 4, 1, 0, ADAPT["adapt_depth"], sigma, alpha, 0, split_cap)
    cb_ws = bnb._ws(bnb.bnb_bound_tuples_ws(bnb.C.byref(ds.s1), None, bnb.C.byref(ds.em), bnb.C.byref(cfg)), dev)
    pre_cap = int(idx.count[1].item()) + int(idx.count[1].item()) // 4 + 4096
    ix_ws = bnb._ws(bnb.bnb_build_index_ws(bnb.C.byref(cb.c), sc.grid_res, pre_cap), dev)
    idx = bnb.Index(sc.grid_res, pre_cap, dev)
    sm_ws = bnb._ws(bnb.bnb_sample_and_solve_ws(bnb.C.byref(ds.s1), None, n_points, wl_cap), dev)
    E_out = torch.empty(n_points, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(seed, ev):
        ev[0].record(stream)
        bnb.bound_tuples(ds, ADAPT["depth"], out=cb, ws=cb_ws, sync_check=False, split_capacity=split_cap, **kw)
        ev[1].record(stream)
        bnb.build_index(cb, grid_res=sc.grid_res, pre_capacity=pre_cap, capacity=pre_cap, out=idx, ws=ix_ws,
                        sync_check=False)
        ev[2].record(stream)
        r = bnb.sample_and_solve(ds, idx, gamma, seed, worklist_capacity=wl_cap, E_out=E_out, ws=sm_ws,
                                 sync_check=False)
        ev[3].record(stream)
        return r

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(3 + steps)]
    for i in range(3 + steps):
        flush.zero_()
        r = step(i, evs[i])
    torch.cuda.synchronize()
    st = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])] for e in evs[3:]])
    ms = st.mean(axis=0)
    ok = int(cb.status.item()) == 0 and int(idx.status.item()) == 0 and int(r.status.item()) == 0
    n_rec = cb.n_records()
    fl = cb.flags[:n_rec]
    live = int(((fl & 1) != 0).sum().item())
    split = int(((fl & 2) != 0).sum().item())
    dep = ((fl.to(torch.int64) >> 24) & 63)[(fl & 1) != 0]
    hist = torch.bincount(dep, minlength=ADAPT["adapt_depth"] + 1).cpu().tolist()
    c = r.counters.cpu().numpy()
    n_base = sc.emitters.n * sc.s1.n_tris * 4 ** ADAPT["depth"]
    out = {"workload": "mirror256 (131,072 tris x 16 area-light samples) from depth 0, adaptive to depth "
                       f"{ADAPT['adapt_depth']}: sigma {sigma} (box area), alpha {alpha}; "
                       "1024^2 points, E|S| = 4", "status_ok": ok, "steps": steps, "base_cells": n_base,
           "records": n_rec, "live_leaves": live, "split_cells": split, "live_depth_histogram": hist,
           "gamma": gamma, "stage_ms": {"bound": float(ms[0]), "index": float(ms[1]), "sample_solve": float(ms[2])},
           "cells_per_s": n_rec / (ms[0] / 1e3), "shading_samples_per_s": n_points / (ms[2] / 1e3),
           "per_point": {"U": c[0] / n_points, "S": c[1] / n_points, "roots": c[2] / n_points}}
    del cb, idx, cb_ws, ix_ws, sm_ws, flush
    torch.cuda.empty_cache()
    return out


ADAPT_SWEEP = [(sg, al) for al in (1.25, 2.0, 10.0) for sg in (1e-5, 1e-6, 1e-7)]


def adaptive_sweep(dev, steps: int) -> list:
    """The stopping parameters of adaptive subdivision (Sec. 6.1, the sweep of Fig. fig_par) on
    the benchmark mirror: box area sigma and bound ratio alpha against the precomputation time
    (bound + index), the tuples listed per point |U| and the roots found per point at E|S| = 4."""
    rows = []
    for sg, al in ADAPT_SWEEP:
        try:
            r = adaptive_summary(dev, steps, sigma=sg, alpha=al)
        except Exception as ex:  # a configuration that does not fit is reported, the rest stand
            rows.append({"sigma": sg, "alpha": al, "error": f"{type(ex).__name__}: {ex}"})
            continue
        rows.append({"sigma": sg, "alpha": al, "status_ok": r["status_ok"], "records": r["records"],
                     "live_leaves": r["live_leaves"], "precompute_ms": r["stage_ms"]["bound"] + r["stage_ms"]["index"],
                     "stage_ms": r["stage_ms"], "U": r["per_point"]["U"], "S": r["per_point"]["S"],
                     "roots": r["per_point"]["roots"]})
    return rows


# ----------------------------------------------------------------------------- accuracy vs the oracle
# Part of the CPU-baseline leg (the oracle runs in a spawned child process; skipped with
# --no-cpu-baseline): the error of the timed path's results against the FP64 oracle on seeded
# samples of the benchmark workload.
ACC_CELLS = 100_000      # seeded base cells whose records are compared
ACC_CLUSTERS = 64        # seeded clusters of 4 x 4 adjacent grid cells: 1024 grid cells, ~4096 points
ACC_SEED = 77


def accuracy_gpu_side(bnb, ds, sc, idx, dev) -> dict:
    """GPU records of ACC_CELLS seeded base cells (plus the children of those that split), from a
    bound pass that also writes e_hi_min; the shading points of ACC_CLUSTERS x 16 seeded grid cells
    and every cell of every tuple the GPU index lists there (the oracle's index is exact on those
    grid cells: the GPU's boxes contain the oracle's, so any tuple the oracle lists there is one of
    them)."""
    import torch
    cbx = bnb.bound_tuples(ds, sc.depth, with_e_hi_min=True, with_e_lo=False)
    n_base = cbx.c.n_base
    rng = np.random.default_rng(11)
    work = np.sort(rng.choice(n_base, ACC_CELLS, replace=False))
    fields = ("u_lo", "u_hi", "v_lo", "v_hi", "e_hi", "e_hi_min", "emitter", "tri0", "cell", "flags")
    wt = torch.as_tensor(work, device=dev)
    g = {k: getattr(cbx, k)[wt].cpu().numpy() for k in fields}
    n_rec = cbx.n_records()
    if n_rec > n_base:  # children of the sampled cells that split
        ch = {k: getattr(cbx, k)[n_base:n_rec].cpu().numpy() for k in fields}
        cd = (ch["flags"].view(np.uint32).astype(np.int64) >> 24) & 63
        parent = ch["cell"].view(np.uint32).astype(np.int64) >> (2 * (cd - sc.depth))
        sk = set(zip(g["emitter"].tolist(), g["tri0"].tolist(), g["cell"].view(np.uint32).tolist()))
        keep = np.array([(int(a), int(b), int(c)) in sk for a, b, c in zip(ch["emitter"], ch["tri0"], parent)],
                        dtype=bool)
        for k in fields:
            g[k] = np.concatenate([g[k], ch[k][keep]])
    g["cell"] = g["cell"].view(np.uint32)
    g["flags"] = g["flags"].view(np.uint32)
    del cbx
    torch.cuda.empty_cache()
    G = sc.grid_res
    rng = np.random.default_rng(12)
    cx, cy = rng.integers(0, G - 4, ACC_CLUSTERS), rng.integers(0, G - 4, ACC_CLUSTERS)
    cells = np.unique(np.array([(y + dy) * G + (x + dx) for x, y in zip(cx, cy) for dy in range(4) for dx in range(4)]))
    gi = np.clip(np.floor(np.clip(sc.su, 0, 1).astype(np.float32) * np.float32(G)), 0, G - 1).astype(np.int64)
    gj = np.clip(np.floor(np.clip(sc.sv, 0, 1).astype(np.float32) * np.float32(G)), 0, G - 1).astype(np.int64)
    pts = np.nonzero(np.isin(gj * G + gi, cells))[0]
    off = idx.offsets.cpu().numpy()
    n_ent = int(idx.count[0].item())
    segs = [idx.key[off[c]:min(off[c + 1], n_ent)] for c in cells]
    keys = np.unique(torch.cat(segs).cpu().numpy().view(np.uint64)) if segs else np.zeros(0, np.uint64)
    e = (keys >> np.uint64(48)).astype(np.int64)
    t = (keys & np.uint64(0xFFFFFF)).astype(np.int64)
    per = 4 ** sc.depth
    tuple_work = (((e * sc.s1.n_tris + t) * per)[:, None] + np.arange(per)[None, :]).ravel()
    return {"records": g, "work": work, "points": pts, "tuple_work": tuple_work, "n_tuples": int(keys.shape[0])}


def _compare_records(g: dict, o) -> dict:
    """GPU records against the oracle's, matched by (emitter, triangle, cell, depth): flags (outside
    the ambiguity bands), box containment and widening, E_hi never below the oracle's, the relative
    excess of E_hi (all finite cells, and the well-conditioned ones: min |b(M)| / max |b(M)| >= 1e-3),
    and the certified enclosure [e_hi_min, e_hi] holding the oracle's float64 bound."""
    gd = (g["flags"].astype(np.int64) >> 24) & 63
    od = (o["flags"].astype(np.int64) >> 24) & 63
    gk = {(int(a), int(b), int(c), int(d)): i for i, (a, b, c, d) in
          enumerate(zip(g["emitter"], g["tri0"], g["cell"], gd))}
    rep = dict(oracle_records=int(len(o)), missing=0, flag_mismatch=0, flag_ambiguous=0, live=0,
               containment_violations=0, e_hi_below_oracle=0, enclosure_violations=0, e_finite=0)
    widen, rel, rel_wc = [], [], []
    for j in range(len(o)):
        i = gk.get((int(o["emitter"][j]), int(o["tri0"][j]), int(o["cell"][j]), int(od[j])))
        if i is None:
            rep["missing"] += 1
            continue
        gf, of = int(g["flags"][i]) & 0xBF, int(o["flags"][j]) & 0xFF
        if gf != of:
            amb = o["q_cond"][j] < 1e-10 or ((gf & 16) and not (of & 16) and o["m_cond"][j] < 1e-3
                                             and (gf & ~16) == (of & ~16))
            rep["flag_ambiguous" if amb else "flag_mismatch"] += 1
            continue
        if not (of & 1):
            continue
        rep["live"] += 1
        for a in ("u", "v"):
            gl, gh = float(g[a + "_lo"][i]), float(g[a + "_hi"][i])
            ol, oh = float(o[a + "_lo"][j]), float(o[a + "_hi"][j])
            if gl > ol + 1e-12 or gh < oh - 1e-12:
                rep["containment_violations"] += 1
            widen.append(max(ol - gl, gh - oh))
        oe, ge, gm = float(o["e_hi"][j]), float(g["e_hi"][i]), float(g["e_hi_min"][i])
        if np.isfinite(oe) and np.isfinite(ge):
            rep["e_finite"] += 1
            r = (ge - oe) / oe
            rel.append(r)
            if o["m_cond"][j] >= 1e-3:
                rel_wc.append(r)
            if ge < oe * (1 - 1e-6):
                rep["e_hi_below_oracle"] += 1
            if oe < gm * (1 - 1e-6) or oe > ge * (1 + 1e-6):
                rep["enclosure_violations"] += 1
        elif np.isfinite(ge):
            rep["e_hi_below_oracle"] += 1
    w = np.array(widen or [0.0])
    r = np.array(rel or [0.0])
    rw = np.array(rel_wc or [0.0])
    rep.update(box_widen_max=float(w.max()), box_widen_p99=float(np.percentile(w, 99)),
               e_hi_rel_excess_median=float(np.median(r)), e_hi_rel_excess_p99=float(np.percentile(r, 99)),
               e_hi_rel_excess_max=float(r.max()), e_hi_frac_within_1e4=float(np.mean(np.abs(r) <= 1e-4)),
               well_conditioned_cells=len(rel_wc),
               well_conditioned_e_hi_rel_excess_max=float(rw.max()),
               well_conditioned_e_hi_rel_excess_p99=float(np.percentile(rw, 99)))
    return rep


def _accuracy_worker(name, gside, gamma, seed):
    sys.path.insert(0, ROOT)
    import copy

    import oracle
    from paper_2504_19163_gb300 import scenes as S
    oracle.build()
    sc = S.config(name)
    n_threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    o = oracle.bound(sc, work=gside["work"], n_threads=n_threads)
    cells = _compare_records(gside["records"], o)
    o2 = oracle.bound(sc, work=gside["tuple_work"], n_threads=n_threads)
    f = oracle.records_to_f32(o2)
    off, key, et = oracle.index(f["u_lo"], f["u_hi"], f["v_lo"], f["v_hi"], f["e_hi"], f["emitter"], f["tri0"],
                                f["tri1"], f["flags"], sc.grid_res)
    pts = gside["points"]
    sub = copy.copy(sc)
    sub.su, sub.sv = sc.su[pts], sc.sv[pts]
    out = {"cells": cells, "off": off, "key": key, "et": et, "oracle_cells": int(len(o) + len(o2))}
    for tag, gm in (("sampled", gamma), ("all", float("inf"))):
        wp, wk, wP, n_u = oracle.sample(off, key, et, sc.grid_res, sub.su, sub.sv, gm, seed)
        contrib, ru, rv, st = oracle.solve(sub, wp, wk, wP, n_threads=n_threads)
        out[tag] = {"wp": wp, "wk": wk, "ru": ru, "rv": rv, "st": st,
                    "E": oracle.accumulate(pts.shape[0], wp, contrib), "n_u": n_u}
    out["seconds"] = time.perf_counter() - t0
    return out


def _x1(s1, tri, u, v):
    P = lambda i: np.stack([s1.px[i], s1.py[i], s1.pz[i]], axis=-1).astype(np.float64)
    p0 = P(s1.i0[tri])
    return p0 + u[:, None] * (P(s1.i1[tri]) - p0) + v[:, None] * (P(s1.i2[tri]) - p0)


def _point_errors(E_g, E_o) -> dict:
    E_g = np.asarray(E_g, np.float64)
    pos = E_o > 0
    rel = np.abs(E_g[pos] - E_o[pos]) / E_o[pos]
    return {"points": int(E_o.shape[0]), "lit_points": int(pos.sum()),
            "E_rel_max": float(rel.max(initial=0.0)), "E_rel_p99": float(np.percentile(rel, 99)) if rel.size else 0.0,
            "points_above_1e-4": int(np.sum(rel > 1e-4) + np.sum(E_g[~pos] != 0))}


def _root_errors(s1, gp, gk, guv, o) -> dict:
    gmap = {(int(p), int(k)): i for i, (p, k) in enumerate(zip(gp, gk))}
    oi, gi, one_side, missing = [], [], 0, 0
    for j, (p, k) in enumerate(zip(o["wp"], o["wk"])):
        i = gmap.pop((int(p), int(k)), None)
        if i is None:
            missing += 1
            continue
        gr, orr = bool(np.isfinite(guv[i, 0])), bool(o["st"][j])
        if gr and orr:
            oi.append(j)
            gi.append(i)
        elif gr != orr:
            one_side += 1
    extra_roots = int(sum(np.isfinite(guv[i, 0]) for i in gmap.values()))
    d = 0.0
    if oi:
        oi, gi = np.array(oi), np.array(gi)
        tri = (o["wk"][oi] & np.uint64(0xFFFFFF)).astype(np.int64)
        d = float(np.max(np.linalg.norm(_x1(s1, tri, guv[gi, 0], guv[gi, 1]) -
                                        _x1(s1, tri, o["ru"][oi], o["rv"][oi]), axis=1)))
    return {"roots": int(len(oi)), "root_dist_max": d, "root_on_one_side": one_side,
            "oracle_selections_missing": missing, "gpu_only_selections": len(gmap), "gpu_only_roots": extra_roots}


def accuracy_summary(bnb, ds, sc, idx, gamma, dev) -> dict:
    """Error of the timed path against the FP64 oracle (Sec. 8 parity, measured on the benchmark
    workload): (1) records of 100,000 seeded base cells; (2) ~4096 seeded points: the rendering pass
    on the oracle's index with the benchmark's gamma (selections, per-point estimates, roots); (3) the
    same points with every listed tuple selected (gamma = inf), the GPU's own index against the
    oracle's: the whole path, deterministic."""
    import multiprocessing as mp

    import torch
    gside = accuracy_gpu_side(bnb, ds, sc, idx, dev)
    with mp.get_context("spawn").Pool(1) as pool:
        o = pool.apply(_accuracy_worker, (sc.name, gside, gamma, ACC_SEED))
    pts = gside["points"]
    su = ds.t["su"][torch.as_tensor(pts, device=dev)]
    sv = ds.t["sv"][torch.as_tensor(pts, device=dev)]
    G = sc.grid_res
    io = bnb.Index(G, max(1, o["key"].shape[0]), dev)
    io.offsets.copy_(torch.as_tensor(o["off"]))
    if o["key"].shape[0]:
        io.key[: o["key"].shape[0]] = torch.as_tensor(o["key"].view(np.int64))
        io.etilde[: o["key"].shape[0]] = torch.as_tensor(o["et"])
    io.count[0] = o["key"].shape[0]
    r = bnb.sample_and_solve(ds, io, gamma, ACC_SEED, su=su, sv=sv, with_roots=True)
    gp, gk, guv = r.roots()
    sampled = {"gamma": gamma, "seed": ACC_SEED,
               "selections_equal": bool(np.array_equal(gp, o["sampled"]["wp"]) and
                                        np.array_equal(gk, o["sampled"]["wk"])),
               "selections": int(gp.shape[0])}
    sampled.update(_point_errors(r.E.cpu().numpy(), o["sampled"]["E"]))
    sampled.update(_root_errors(sc.s1, gp, gk, guv, o["sampled"]))
    r2 = bnb.sample_and_solve(ds, idx, float("inf"), ACC_SEED, su=su, sv=sv, with_roots=True)
    gp2, gk2, guv2 = r2.roots()
    whole = {"gamma": "inf", "selections_gpu": int(gp2.shape[0]), "selections_oracle": int(o["all"]["wp"].shape[0])}
    whole.update(_point_errors(r2.E.cpu().numpy(), o["all"]["E"]))
    whole.update(_root_errors(sc.s1, gp2, gk2, guv2, o["all"]))
    return {"cells": dict(o["cells"], sampled_base_cells=ACC_CELLS, seed=11),
            "points_on_oracle_index": dict(sampled, grid_cells=16 * ACC_CLUSTERS,
                                           tuples_bounded_by_oracle=gside["n_tuples"]),
            "whole_path_every_tuple": whole,
            "tolerances": {"E_rel": 1e-4, "root_scene_units": 1e-5, "box": "GPU box contains the oracle's"},
            "oracle_seconds": round(o["seconds"], 2), "oracle_cells_bounded": o["oracle_cells"]}


def _pairs_oracle_worker():
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2504_19163_gb300 import scenes as S
    oracle.build()
    sc = S.config("slab48")
    n_threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    rec = oracle.bound_pair_scene(sc, n_threads=n_threads)
    dt = time.perf_counter() - t0
    return {"kind": "oracle", "cores": n_threads, "bound_s": dt, "pair_records": int(rec.shape[0]),
            "pair_records_per_s": rec.shape[0] / dt,
            "sample": "the whole slab48 bound pass (candidates by brute force over every T2, then the records)"}


def cpu_baseline(u_per_point: float, s_per_point: float) -> dict:
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(1) as pool:
        return pool.apply(_cpu_baseline_worker, ("mirror256", u_per_point, s_per_point))


def _cpu_baseline_worker(name, u_per_point, s_per_point):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2504_19163_gb300 import scenes as S
    oracle.build()
    sc = S.config(name)
    n_threads = os.cpu_count() or 1
    per = 4 ** sc.depth
    n_sample = -(-sc.emitters.n * sc.s1.n_tris * per // 100 // per) * per  # >= 1% of the cells, whole tuples
    t_cell, t_draw, t_solve, desc = oracle_step_sample(sc, n_sample, 1024, 7, n_threads)
    step_s = oracle_step_seconds(sc, t_cell, t_draw, t_solve, u_per_point, s_per_point)
    n_cells = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
    return {"value": n_cells / step_s, "unit": "cells/s", "cores": n_threads, "kind": "oracle",
            "sample": f"{desc} on {n_threads} threads; extrapolated to {n_cells} cells and {sc.su.shape[0]} "
                      f"points x ({u_per_point:.1f} draws + {s_per_point:.2f} solves, this run's |U|, |S|)"}


def profile_case(args):
    """Small cases of single stages for ncu captures (no JSON line): `--warmup` + `--steps` launches of
    the stage named by --profile-case, inputs larger than L2 but a few GB on the device at most.
      refraction  water420 with its first light (22.6M cells): the refraction bound pass
      index       mirror256 with 4 of its 16 light samples (33.6M cells): the index pass
      sample      mirror256 with 8 light samples: the rendering pass over its index (1024^2 points)
      chain       slab48: the two-vertex bound pass with the chain irradiance post-pass
      implicit    tir_wall 32^2, depth 4: the implicit-differentiation pass"""
    import torch
    from paper_2504_19163_gb300 import bnb, build
    from paper_2504_19163_gb300 import scenes as S
    build.build()
    dev = torch.device("cuda", 0)
    case = args.profile_case

    def subset(sc, n):
        e = sc.emitters
        sc.emitters = S.Emitters(e.x[:n], e.y[:n], e.z[:n], e.intensity[:n])
        return sc

    n = args.warmup + args.steps
    if case == "refraction":
        sc = subset(S.config("water420"), 1)
        ds = bnb.DeviceScene(sc, dev)
        cb = bnb.bound_tuples(ds, sc.depth, with_e_lo=False)
        for _ in range(n):
            bnb.bound_tuples(ds, sc.depth, out=cb, sync_check=False)
    elif case in ("index", "sample"):
        sc = subset(S.config("mirror256"), 4 if case == "index" else 8)
        ds = bnb.DeviceScene(sc, dev)
        cb = bnb.bound_tuples(ds, sc.depth, with_e_lo=False)
        idx = bnb.build_index(cb, grid_res=sc.grid_res)
        if case == "index":
            for _ in range(n):
                bnb.build_index(cb, grid_res=sc.grid_res, pre_capacity=int(idx.count[1].item()) + 4096,
                                capacity=int(idx.count[1].item()) + 4096, out=idx, sync_check=False)
        else:
            del cb
            torch.cuda.empty_cache()
            gamma = calibrate_gamma(bnb, ds, idx, target=4.0)
            for i in range(n):
                bnb.sample_and_solve(ds, idx, gamma, i)
    elif case == "chain":
        sc = S.config("slab48")
        ds = bnb.DeviceScene(sc, dev)
        cb = bnb.bound_tuples(ds, sc.depth, with_e_lo=False)
        for _ in range(n):
            bnb.bound_tuples(ds, sc.depth, out=cb, sync_check=False)
    elif case == "implicit":
        sc = S.config("tir_wall", n=32, depth=4)
        ds = bnb.DeviceScene(sc, dev)
        cb = bnb.bound_tuples(ds, sc.depth, irradiance=True)
        for _ in range(n):
            bnb.implicit_irradiance(ds, cb, n=-1, mode=1)
    else:
        raise SystemExit(f"unknown profile case {case}")
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "launches": n, "stream_status": bnb.stream_status()}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--emitters", type=int, default=0, help="use only the first N area-light samples (profiling case)")
    ap.add_argument("--serving-requests", type=int, default=256,
                    help="requests of the serving workload reported under 'serving' (0: skip)")
    ap.add_argument("--adaptive-sweep-steps", type=int, default=2,
                    help="timed steps per (sigma, alpha) of the adaptive parameter sweep (0: skip)")
    ap.add_argument("--adaptive-steps", type=int, default=5,
                    help="timed steps of the adaptive-subdivision mirror256 pass reported under 'adaptive' (0: skip)")
    ap.add_argument("--implicit-steps", type=int, default=5,
                    help="timed launches of the implicit-differentiation irradiance pass (0: skip)")
    ap.add_argument("--pairs-steps", type=int, default=10,
                    help="timed steps of the two-vertex slab48 workload reported under 'pairs' (0: skip)")
    ap.add_argument("--refraction-steps", type=int, default=5,
                    help="timed steps of the water420 refraction workload reported under 'refraction' (0: skip)")
    ap.add_argument("--rough-steps", type=int, default=3,
                    help="timed bound passes of mirror256_rough reported under 'rough' (0: skip)")
    ap.add_argument("--profile-case", default="", choices=["", "refraction", "index", "sample", "chain", "implicit"],
                    help="run one stage's small profiling case (for ncu) instead of the benchmark")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_case:
        return profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

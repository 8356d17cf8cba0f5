"""bnb_stream_status (the device error word) and bnb_gamma_for_target (Sec. 5.4's gamma <-> E|S|
map) through the C ABI on the GPU."""
import os

import numpy as np
import pytest
import torch

from paper_2504_19163_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2504_19163_gb300 import build
    build.build()
    from paper_2504_19163_gb300 import bnb
    return bnb


@pytest.fixture(scope="module")
def m32(orc):
    sc = S.config("mirror32")
    rec = orc.bound(sc, n_threads=os.cpu_count())
    f = orc.records_to_f32(rec)
    off, key, et = orc.index(f["u_lo"], f["u_hi"], f["v_lo"], f["v_hi"], f["e_hi"], f["emitter"], f["tri0"],
                             f["tri1"], f["flags"], sc.grid_res)
    return sc, off, key, et


def upload_index(B, off, key, et, G):
    idx = B.Index(G, max(1, key.shape[0]), torch.device("cuda"))
    idx.offsets.copy_(torch.as_tensor(off))
    if key.shape[0]:
        idx.key[: key.shape[0]] = torch.as_tensor(key.view(np.int64))
        idx.etilde[: key.shape[0]] = torch.as_tensor(et)
    idx.count[0] = key.shape[0]
    return idx


# ----------------------------------------------------------------------------- stream status
def test_stream_status_reports_and_clears_device_errors(B, m32):
    sc, off, key, et = m32
    ds = B.DeviceScene(sc)
    B.stream_status()  # clear whatever earlier tests left
    idx = upload_index(B, off, key, et, sc.grid_res)
    r = B.sample_and_solve(ds, idx, 2.0, 3)
    assert int(r.status.item()) == 0
    assert B.stream_status() == B.BNB_OK
    # a worklist too small: the struct's status and the device word both report it
    r = B.sample_and_solve(ds, idx, 2.0, 3, worklist_capacity=10, sync_check=False)
    assert B.stream_status() == B.BNB_ERR_CAPACITY
    assert int(r.status.item()) == B.BNB_ERR_CAPACITY  # the struct's word is not touched
    assert B.stream_status() == B.BNB_OK                # read once, cleared
    # a bound pass that fits, then an index too small for its records
    cb = B.bound_tuples(ds, sc.depth)
    assert B.stream_status() == B.BNB_OK
    small = B.build_index(cb, grid_res=sc.grid_res, pre_capacity=16, capacity=16, sync_check=False)
    assert B.stream_status() == B.BNB_ERR_CAPACITY
    assert int(small.status.item()) == B.BNB_ERR_CAPACITY
    assert B.stream_status() == B.BNB_OK


def test_stream_status_sees_other_streams(B, m32):
    """The word belongs to the context: an error raised on one stream is reported to a read on
    another stream once the raising work has finished."""
    sc, off, key, et = m32
    ds = B.DeviceScene(sc)
    idx = upload_index(B, off, key, et, sc.grid_res)
    B.stream_status()
    s1 = torch.cuda.Stream()
    with torch.cuda.stream(s1):
        B.sample_and_solve(ds, idx, 2.0, 3, worklist_capacity=10, sync_check=False, stream=s1)
    s1.synchronize()
    assert B.stream_status(torch.cuda.current_stream()) == B.BNB_ERR_CAPACITY
    assert B.stream_status(s1) == B.BNB_OK


# ----------------------------------------------------------------------------- gamma for E|S|
def f32_mul_ru(a: np.float32, b: np.ndarray) -> np.ndarray:
    """float32 product rounded toward +inf (the float64 product of two float32 values is exact)."""
    p = np.float64(a) * b.astype(np.float64)
    with np.errstate(over="ignore", invalid="ignore"):
        r = p.astype(np.float32)
        low = np.isfinite(p) & (r.astype(np.float64) < p)
    r[low] = np.nextafter(r[low], np.float32(np.inf))
    return r


def expected_selections_scaled(gamma: np.float32, off, et, weights) -> int:
    """sum over grid cells g of w_g * sum over g's listed tuples of ceil(P 2^24), P = min(gamma (x)
    E~, 1): 2^24 W times the expected |S| per point under a 24-bit draw r < P."""
    P = np.minimum(f32_mul_ru(gamma, et), np.float32(1.0))
    P[np.isnan(P)] = 1.0
    c = np.ceil(P.astype(np.float64) * 16777216.0).astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(c)])
    per_cell = cs[off[1:]] - cs[off[:-1]]
    return int(np.sum(per_cell.astype(object) * weights.astype(object)))


def point_weights(sc, G):
    gi = np.clip(np.floor(np.clip(sc.su, 0, 1).astype(np.float32) * np.float32(G)), 0, G - 1).astype(np.int64)
    gj = np.clip(np.floor(np.clip(sc.sv, 0, 1).astype(np.float32) * np.float32(G)), 0, G - 1).astype(np.int64)
    return np.bincount(gj * G + gi, minlength=G * G)


def mean_listed(sc, off):
    """|U| per shading point: the largest reachable E|S| (every listed tuple selected)."""
    w = point_weights(sc, sc.grid_res)
    return float(np.sum(np.diff(off) * w) / sc.su.shape[0])


@pytest.mark.parametrize("frac", [0.1, 0.5, 0.9])
def test_gamma_is_the_smallest_float_reaching_the_target(B, m32, frac):
    sc, off, key, et = m32
    G = sc.grid_res
    target = frac * mean_listed(sc, off)
    idx = upload_index(B, off, key, et, G)
    ds = B.DeviceScene(sc)
    g = B.gamma_for_target(idx, target, ds.t["su"], ds.t["sv"])
    gamma = np.float32(g.item())
    w = point_weights(sc, G)
    thresh = target * sc.su.shape[0] * 16777216.0
    assert expected_selections_scaled(gamma, off, et, w) >= thresh
    below = np.nextafter(gamma, np.float32(0.0))
    assert expected_selections_scaled(below, off, et, w) < thresh
    # uniform weights (every grid cell once)
    target = frac * float(np.mean(np.diff(off)))
    gu = np.float32(B.gamma_for_target(idx, target).item())
    ones = np.ones(G * G, np.int64)
    assert expected_selections_scaled(gu, off, et, ones) >= target * G * G * 16777216.0
    assert expected_selections_scaled(np.nextafter(gu, np.float32(0.0)), off, et, ones) < target * G * G * 16777216.0


def test_gamma_sets_the_mean_selection_count(B, m32):
    """Rendering with the returned gamma selects about `target` tuples per point (mean over
    seeds; the exact expectation is pinned above)."""
    sc, off, key, et = m32
    idx = upload_index(B, off, key, et, sc.grid_res)
    ds = B.DeviceScene(sc)
    target = 0.5 * mean_listed(sc, off)
    gamma = float(B.gamma_for_target(idx, target, ds.t["su"], ds.t["sv"]).item())
    sel = [int(B.sample_and_solve(ds, idx, gamma, s).counters[1].item()) for s in range(16)]
    mean = np.mean(sel) / sc.su.shape[0]
    assert abs(mean - target) < 0.02 * target, (mean, target)


def test_gamma_unreachable_target_gives_float_max(B, m32):
    sc, off, key, et = m32
    idx = upload_index(B, off, key, et, sc.grid_res)
    ds = B.DeviceScene(sc)
    g = float(B.gamma_for_target(idx, 1.01 * mean_listed(sc, off), ds.t["su"], ds.t["sv"]).item())
    assert g == float(np.finfo(np.float32).max)

"""GPU parity of single refraction (Eq. eq_refr_rational, refraction, with the sqrt(beta)
remainder of Sec. 4.3): the bound pass against the oracle and against dense sweeps of the true
refracted paths, the rendering pass on the oracle's index, the whole path, and the batched pass."""
import os

import numpy as np
import pytest
import torch

import parity
from paper_2504_19163_gb300 import scenes as S
from test_oracle_bounds import cell_points
from test_oracle_refraction import flat_refract

pytestmark = pytest.mark.gpu

E_REL = 1e-4
BOX64 = 2.0 ** -22  # the float64 mode stores float32 boxes


@pytest.fixture(scope="module")
def B():
    from paper_2504_19163_gb300 import build
    build.build()
    from paper_2504_19163_gb300 import bnb
    return bnb


def gpu_bound(B, sc, fp64=False, max_extra_split=4):
    ds = B.DeviceScene(sc)
    cb = B.bound_tuples(ds, sc.depth, max_extra_split=max_extra_split, fp64=fp64)
    torch.cuda.synchronize()
    assert int(cb.status.item()) == 0
    return ds, cb, cb.to_numpy()


def sweep_violations_gpu(orc, sc, g, K=8):
    """True paths (oracle's direct Snell evaluator) landing on [0,1]^2 outside their GPU machine or its
    irradiance bound [e_lo, e_hi], or on a cell the GPU culled."""
    viol = hits = 0
    for i in range(len(g["flags"])):
        f = int(g["flags"][i])
        if f & 2:
            continue
        d = int(parity.depth_of(f))
        u, v = cell_points(orc, g["cell"][i], d, K)
        uk, vk, E, t = orc.eval_path(sc, int(g["emitter"][i]), int(g["tri0"][i]), u, v, direct=True)
        on = (uk >= 0) & (uk <= 1) & (vk >= 0) & (vk <= 1) & (t > 0)
        if not (f & 1):
            viol += int(on.sum())
            continue
        hits += int(on.sum())
        viol += int((on & ((uk < g["u_lo"][i]) | (uk > g["u_hi"][i]) | (vk < g["v_lo"][i])
                           | (vk > g["v_hi"][i]))).sum())
        ok = np.isfinite(E)
        viol += int((E[ok] > g["e_hi"][i] * (1 + 1e-6)).sum())
        if "e_lo" in g:
            viol += int((E[ok] < g["e_lo"][i] * (1 - 1e-6)).sum())
    return viol, hits


CASES = [dict(n=8, depth=2), dict(n=6, depth=2, steep=0.08, lights=[(0.3, 0.2, 1.2)]),
         dict(n=16, depth=1, extent=2.0, rec_half=2.0, lights=[(0.1, -0.05, 2.0), (-0.5, 0.5, 2.0)])]


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("fp64", [False, True])
def test_refraction_bound_parity(B, orc, kw, fp64):
    sc = S.config("water", **kw)
    ds, cb, g = gpu_bound(B, sc, fp64=fp64)
    o = orc.bound(sc, n_threads=os.cpu_count())
    rep = parity.compare_refraction(g, o, position_only=fp64)
    print(rep)
    assert rep["missing"] == 0 and rep["flag_mismatch"] == 0
    assert rep["flag_ambiguous"] <= max(2, 1e-3 * rep["n"])
    assert rep["box_diff_max"] <= (BOX64 if fp64 else parity.BOX_TOL32)
    if fp64:
        assert rep["e_finite"] == 0  # the float64 pass bounds refraction positions only
    else:
        assert rep["e_finite"] > 0.9 * rep["live"] and rep["e_below"] == 0
        assert rep["e_rel_median"] <= parity.REFR_E_MEDIAN and rep["e_rel_p99"] <= parity.REFR_E_P99
    viol, hits = sweep_violations_gpu(orc, sc, g)
    assert viol == 0 and hits > 1000


def test_total_internal_reflection_flags(B, orc):
    sc = flat_refract(n=4, eta=1.5, h=0.3, light=(0.0, 0.0), depth=2, extent=1.0, half=3.0, H=0.5)
    ds, cb, g = gpu_bound(B, sc)
    o = orc.bound(sc)
    rep = parity.compare_refraction(g, o)
    assert rep["missing"] == 0 and rep["flag_mismatch"] == 0
    assert np.any(g["flags"] & 128) and np.any(g["flags"] & 1)
    viol, hits = sweep_violations_gpu(orc, sc, g)
    assert viol == 0 and hits > 100


def upload_index(B, off, key, et, G):
    idx = B.Index(G, max(1, key.shape[0]), torch.device("cuda"))
    idx.offsets.copy_(torch.as_tensor(off))
    if key.shape[0]:
        idx.key[: key.shape[0]] = torch.as_tensor(key.view(np.int64))
        idx.etilde[: key.shape[0]] = torch.as_tensor(et)
    idx.count[0] = key.shape[0]
    return idx


@pytest.fixture(scope="module")
def w16(orc):
    sc = S.config("water", n=16, depth=1, extent=2.0, rec_half=2.0, points=48,
                  lights=[(0.1, -0.05, 2.0), (-0.5, 0.5, 2.0)])
    rec = orc.bound(sc, n_threads=os.cpu_count())
    f = orc.records_to_f32(rec)
    off, key, et = orc.index(f["u_lo"], f["u_hi"], f["v_lo"], f["v_hi"], f["e_hi"], f["emitter"], f["tri0"],
                             f["tri1"], f["flags"], sc.grid_res)
    return sc, off, key, et


def gamma_of(sc, off, et, target=4.0):
    G = sc.grid_res
    g = np.clip(np.floor(sc.sv * np.float32(G)), 0, G - 1).astype(np.int64) * G + \
        np.clip(np.floor(sc.su * np.float32(G)), 0, G - 1).astype(np.int64)
    return target / float(np.mean([et[off[i]:off[i + 1]][np.isfinite(et[off[i]:off[i + 1]])].sum() for i in g]))


@pytest.mark.parametrize("mode", ["all", "sampled"])
def test_refraction_solve_on_oracle_index(B, orc, w16, mode):
    """On the oracle's index: with gamma = inf every listed tuple is selected; with gamma for
    E|S| = 4 the selections are bit-exact; roots and estimates against the oracle."""
    sc, off, key, et = w16
    gamma = float("inf") if mode == "all" else gamma_of(sc, off, et)
    ds = B.DeviceScene(sc)
    idx = upload_index(B, off, key, et, sc.grid_res)
    r = B.sample_and_solve(ds, idx, gamma, 9, with_sel_count=True)
    torch.cuda.synchronize()
    wp, wk, wP, n_u = orc.sample(off, key, et, sc.grid_res, sc.su, sc.sv, gamma, 9)
    if mode == "all":
        assert wp.shape[0] == n_u
    assert np.array_equal(r.sel_count.cpu().numpy(), np.bincount(wp, minlength=sc.su.shape[0]))
    contrib, _, _, st = orc.solve(sc, wp, wk, wP, n_threads=os.cpu_count())
    E_o = orc.accumulate(sc.su.shape[0], wp, contrib)
    cnt = r.counters.cpu().numpy()
    assert cnt[0] == n_u and cnt[1] == wp.shape[0] and cnt[2] == int(st.sum())
    E_g = r.E.cpu().numpy().astype(np.float64)
    pos = E_o > 0
    assert int(st.sum()) > (500 if mode == "all" else 100)
    assert np.max(np.abs(E_g[pos] - E_o[pos]) / E_o[pos]) <= E_REL
    assert np.all(E_g[~pos] == 0)


def test_refraction_whole_path(B, orc, w16):
    """bound -> index -> sample -> solve on the GPU vs the oracle with every listed tuple selected
    (gamma = inf): a tuple with a root at a point is listed by both (both boxes contain the true
    paths), so the estimates agree wherever both Newton iterations reach the same roots."""
    sc, off, key, et = w16
    ds = B.DeviceScene(sc)
    cb = B.bound_tuples(ds, sc.depth)
    idx = B.build_index(cb, grid_res=sc.grid_res)
    inf = float("inf")
    r = B.sample_and_solve(ds, idx, inf, 21)
    torch.cuda.synchronize()
    wp, wk, wP, n_u = orc.sample(off, key, et, sc.grid_res, sc.su, sc.sv, inf, 21)
    contrib, _, _, st = orc.solve(sc, wp, wk, wP, n_threads=os.cpu_count())
    E_o = orc.accumulate(sc.su.shape[0], wp, contrib)
    E_g = r.E.cpu().numpy().astype(np.float64)
    close = np.abs(E_g - E_o) <= E_REL * np.maximum(np.abs(E_o), 1e-30)
    print("refraction whole path: points", E_o.size, "mismatched", int((~close).sum()))
    # no selection can flip (P = 1); a mismatch needs the float32 Newton phase and the oracle's
    # float64 iteration to reach different roots
    assert np.mean(close) >= 0.995
    assert abs(E_g.sum() - E_o.sum()) / E_o.sum() < 1e-3
    assert np.count_nonzero(E_o) > 0.3 * E_o.size


def test_refraction_batched_job_equals_single_call(B, w16):
    from paper_2504_19163_gb300 import batch as BA
    sc, off, key, et = w16
    ds = B.DeviceScene(sc)
    idx = upload_index(B, off, key, et, sc.grid_res)
    rs = BA.ResidentScene(ds, idx, 1.0)
    su, sv = ds.t["su"], ds.t["sv"]
    job = BA.Job(rs, su, sv, torch.empty(su.shape[0], device="cuda"), 4)
    runner = BA.BatchRunner(2, su.shape[0], 1 << 20)
    runner.submit([job])
    assert runner.result()[0] == 0
    single = B.sample_and_solve(ds, idx, 1.0, 4)
    torch.cuda.synchronize()
    a, b = job.E_out.cpu().numpy(), single.E.cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32)) and np.count_nonzero(a) > 100


def test_water420_full_size_sampled(B, orc):
    """420^2 water, 4 lights, depth 3 (90M cells) in one launch; 3000 seeded base cells against
    the oracle slot by slot, with the true paths of those cells swept."""
    sc = S.config("water420")
    ds = B.DeviceScene(sc)
    cb = B.bound_tuples(ds, sc.depth, with_e_lo=False)
    torch.cuda.synchronize()
    assert int(cb.status.item()) == 0
    n_base = cb.c.n_base
    assert n_base == 4 * 352800 * 64
    rng = np.random.default_rng(7)
    work = np.sort(rng.choice(n_base, 3000, replace=False))
    wt = torch.as_tensor(work, device="cuda")
    g = {k: getattr(cb, k)[wt].cpu().numpy() for k in ("u_lo", "u_hi", "v_lo", "v_hi", "e_hi", "emitter", "tri0")}
    assert np.isfinite(g["e_hi"]).any()
    g["cell"] = cb.cell[wt].cpu().numpy().view(np.uint32)
    g["flags"] = cb.flags[wt].cpu().numpy().view(np.uint32)
    o = orc.bound(sc, work=work, n_threads=os.cpu_count())
    o_base = o[parity.depth_of(o["flags"]) == sc.depth]
    assert len(o_base) == len(work)
    rep = parity.compare_refraction(g, o_base)
    print(rep)
    assert rep["missing"] == 0 and rep["flag_mismatch"] == 0 and rep["live"] > 600  # the floor sees ~1/3 of the cells
    assert rep["box_diff_max"] <= parity.BOX_TOL32
    assert rep["e_below"] == 0 and rep["e_rel_median"] <= parity.REFR_E_MEDIAN
    viol, hits = sweep_violations_gpu(orc, sc, g, K=6)
    assert viol == 0 and hits > 1000

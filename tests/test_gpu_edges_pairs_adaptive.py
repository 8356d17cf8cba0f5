"""Edge cases of the two-vertex, adaptive, bin-packed and stochastic paths on the GPU: an empty
second surface, the smallest slab, adaptive subdivision that stops at once or may go to the deepest
cell ids, groups with P = 0 and P = 1, and empty point sets."""
import dataclasses

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


def empty_surface(s):
    z = lambda dt: np.zeros(0, dt)
    return dataclasses.replace(s, px=z(np.float32), py=z(np.float32), pz=z(np.float32), nx=z(np.float32),
                               ny=z(np.float32), nz=z(np.float32), i0=z(np.int32), i1=z(np.int32), i2=z(np.int32))


def test_pairs_with_an_empty_second_surface(B):
    sc = S.config("slab", n=3, depth=1, points=8)
    sc = dataclasses.replace(sc, s2=empty_surface(sc.s2))
    ds = B.DeviceScene(sc)
    cb = B.bound_tuples(ds, sc.depth)
    assert int(cb.count.item()) == 0 and int(cb.status.item()) == 0
    idx = B.build_index(cb, sc.grid_res)
    r = B.sample_and_solve(ds, idx, float("inf"), 1)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0 and float(r.E.abs().sum().item()) == 0.0


def test_smallest_slab_matches_oracle(B, orc):
    sc = S.config("slab", n=1, depth=0, points=16, extent=0.5)
    ds = B.DeviceScene(sc)
    g = B.bound_tuples(ds, sc.depth).to_numpy()
    o = orc.bound_pair_scene(sc)
    gk = set(zip(g["emitter"].tolist(), g["tri0"].tolist(), g["cell"].tolist(), g["tri1"].tolist()))
    ok = set(zip(o["emitter"].tolist(), o["tri0"].tolist(), o["cell"].tolist(), o["tri1"].tolist()))
    assert ok <= gk and len(gk - ok) <= 1
    r = B.sample_and_solve(ds, B.build_index(B.bound_tuples(ds, sc.depth), sc.grid_res), float("inf"), 1)
    out = orc.render_pairs(sc, 1.0, 1)
    E = r.E.cpu().numpy().astype(np.float64)
    pos = out["E"] > 0
    assert pos.sum() > 0
    assert np.max(np.abs(E[pos] - out["E"][pos]) / out["E"][pos]) < 1e-4


def test_adaptive_stopping_at_once_equals_the_base_pass(B):
    sc = S.config("mirror32", depth=1)
    ds = B.DeviceScene(sc)
    a = B.bound_tuples(ds, 1, adapt_depth=5, sigma=1e9, alpha=0.0).to_numpy()  # every box is below sigma
    f = B.bound_tuples(ds, 1).to_numpy()
    assert a["flags"].shape == f["flags"].shape
    for k in ("u_lo", "u_hi", "v_lo", "v_hi", "e_hi", "flags"):
        assert np.array_equal(a[k], f[k]), k


def test_adaptive_to_the_deepest_cell_ids(B):
    """adapt_depth 11 with 4 sign-test levels below reaches the 15 levels a cell id holds; with the
    paper's thresholds the tree stays shallow and every leaf is valid."""
    sc = S.config("tiny", n=4, depth=0)
    ds = B.DeviceScene(sc)
    cb = B.bound_tuples(ds, 0, adapt_depth=11, sigma=1e-7, alpha=1.05)
    torch.cuda.synchronize()
    g = cb.to_numpy()
    assert int(cb.status.item()) == 0
    d = (g["flags"].astype(np.int64) >> 24) & 63
    leaves = (g["flags"] & 2) == 0
    assert d.max() <= 15
    mass = {}
    for t, dd in zip(g["tri0"][leaves], d[leaves]):
        mass[int(t)] = mass.get(int(t), 0.0) + 4.0 ** -int(dd)
    assert all(abs(m - 1.0) < 1e-9 for m in mass.values()) and len(mass) == sc.s1.n_tris


def test_bins_with_zero_and_certain_probabilities(B):
    sc = S.config("tiny", n=4, depth=1, points=16)
    ds = B.DeviceScene(sc)
    idx = B.build_index(B.bound_tuples(ds, sc.depth), sc.grid_res)
    r0 = B.sample_and_solve(ds, idx, 0.0, 1, bins=True)  # P = 0 for every finite bound
    r1 = B.sample_and_solve(ds, idx, float("inf"), 1, bins=True)  # P = 1: every tuple its own group
    d1 = B.sample_and_solve(ds, idx, float("inf"), 1)
    torch.cuda.synchronize()
    c0, c1 = r0.counters.cpu().numpy(), r1.counters.cpu().numpy()
    n_inf = int(torch.isinf(idx.etilde[: int(idx.count[0].item())]).sum().item())
    assert c0[1] <= n_inf  # only +inf bounds (P = 1) can be selected at gamma = 0
    assert c1[3] == c1[0] and c1[1] == c1[0]  # |B| = |S| = |U|
    assert torch.equal(r1.E, d1.E)


def test_empty_point_sets_in_the_new_modes(B):
    sc = S.config("tiny", n=4, depth=1, points=4)
    ds = B.DeviceScene(sc)
    idx = B.build_index(B.bound_tuples(ds, sc.depth), sc.grid_res)
    z = torch.zeros(0, dtype=torch.float32, device="cuda")
    for kw in (dict(bins=True), dict(stoc_trials=8)):
        r = B.sample_and_solve(ds, idx, 10.0, 1, su=z, sv=z, **kw)
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0 and r.E.numel() == 0 and int(r.counters.sum().item()) == 0

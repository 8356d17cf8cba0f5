"""Adaptive subdivision in the oracle (Sec. 6.1 "Domain subdivision": a cell is subdivided again
until its receiver box has area below sigma, its irradiance bounds are within the factor alpha, or
the depth limit is reached), pinned against the fixed-depth pass it must reduce to:

* sigma = 0 and alpha = 0 never stop a live cell, so the leaves are exactly the fixed-depth
  records at the limit depth (same values) and the cells no ray of which reaches the receiver;
* the leaves of every tuple partition its triangle (sum of 4^-depth = 1);
* every live leaf above the limit satisfies a stopping criterion, and every adaptively split
  cell, bounded alone, satisfies neither;
* with P = 1 (gamma = inf) the estimate at every point equals the fixed-depth pass's: no cell
  that carries a path is lost by stopping early.
"""
import collections

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19163_gb300 import scenes as S

SPLIT, LIVE, POS_UNBOUNDED = 2, 1, 32


def depth_of(rec):
    return (rec["flags"].astype(np.int64) >> 24) & 63


def leaves(rec):
    return rec[(rec["flags"] & SPLIT) == 0]


def f32_box_area(r):
    dn = lambda x: np.float32(x) if np.float64(np.float32(x)) <= x else np.nextafter(np.float32(x), np.float32(-np.inf))
    up = lambda x: np.float32(x) if np.float64(np.float32(x)) >= x else np.nextafter(np.float32(x), np.float32(np.inf))
    return (up(r["u_hi"]) - dn(r["u_lo"])) * (up(r["v_hi"]) - dn(r["v_lo"])), dn(r["e_lo"]), up(r["e_hi"])


@pytest.mark.parametrize("name,kw", [("tiny", dict(n=4)), ("water", dict(n=3))])
def test_never_stopping_reduces_to_the_fixed_depth_pass(name, kw):
    sc = S.config(name, depth=0, **kw)
    ad = O.bound(sc, depth=0, adapt_depth=2, sigma=0.0, alpha=0.0)
    fx = O.bound(sc, depth=2)
    fx_live = {(int(r["emitter"]), int(r["tri0"]), int(r["cell"]), int(d)): r
               for r, d in zip(fx, depth_of(fx)) if r["flags"] & LIVE}
    lv = leaves(ad)
    for r, d in zip(lv, depth_of(lv)):
        if not r["flags"] & LIVE:
            continue
        k = (int(r["emitter"]), int(r["tri0"]), int(r["cell"]), int(d))
        if r["flags"] & POS_UNBOUNDED and d < 2:
            continue  # a sign-test leaf above the limit keeps its universal box
        assert d >= 2, k
        assert k in fx_live, k
        f = fx_live.pop(k)
        for a in ("u_lo", "u_hi", "v_lo", "v_hi", "e_lo", "e_hi"):
            assert r[a] == f[a] or (np.isinf(r[a]) and np.isinf(f[a])), (k, a)
    # every fixed-depth live cell is a live adaptive leaf (or below a sign-test leaf)
    assert all(v["flags"] & POS_UNBOUNDED for v in fx_live.values()), len(fx_live)


@pytest.mark.parametrize("sigma,alpha", [(1e-4, 2.0), (1e-3, 10.0), (0.0, 1.5)])
def test_adaptive_leaves_partition_and_satisfy_the_stopping_rule(sigma, alpha):
    sc = S.config("tiny", n=4, depth=0)
    lim = 5
    ad = O.bound(sc, depth=0, adapt_depth=lim, sigma=sigma, alpha=alpha)
    lv = leaves(ad)
    mass = collections.defaultdict(float)
    for r, d in zip(lv, depth_of(lv)):
        mass[(int(r["emitter"]), int(r["tri0"]))] += 4.0 ** -int(d)
    assert len(mass) == sc.s1.n_tris
    assert all(abs(m - 1.0) < 1e-12 for m in mass.values())
    n_checked = 0
    for r, d in zip(lv, depth_of(lv)):
        if not r["flags"] & LIVE or r["flags"] & POS_UNBOUNDED or d >= lim:
            continue
        area, el, eh = f32_box_area(r)
        assert area < np.float32(sigma) or eh < np.float32(alpha) * el
        n_checked += 1
    assert n_checked > 10
    # every adaptively split cell, bounded alone at its depth, met neither stopping criterion
    sp = ad[(ad["flags"] & SPLIT) != 0]
    sd = depth_of(sp)
    rng = np.random.default_rng(0)
    for i in rng.choice(sp.shape[0], min(40, sp.shape[0]), replace=False):
        d = int(sd[i])
        w = (int(sp["emitter"][i]) * sc.s1.n_tris + int(sp["tri0"][i])) * 4 ** d + int(sp["cell"][i])
        alone = O.bound(sc, depth=d, max_extra_split=0, work=np.array([w]))
        a = alone[0]
        if not a["flags"] & LIVE:
            continue  # a sign-test split
        area, el, eh = f32_box_area(a)
        assert area >= np.float32(sigma) and not (eh < np.float32(alpha) * el)
    # adaptivity saves cells against the full subdivision at the limit
    assert lv.shape[0] < sc.s1.n_tris * 4 ** lim


def test_adaptive_render_keeps_every_path():
    sc = S.config("tiny", n=4, depth=0, points=24)
    fixed = O.render(sc, float("inf"), 1, depth=3)
    rec = O.bound(sc, depth=0, adapt_depth=3, sigma=1e-3, alpha=2.0)
    f = O.records_to_f32(rec)
    off, key, et = O.index(f["u_lo"], f["u_hi"], f["v_lo"], f["v_hi"], f["e_hi"], f["emitter"], f["tri0"],
                           f["tri1"], f["flags"], sc.grid_res)
    wp, wk, wP, _ = O.sample(off, key, et, sc.grid_res, sc.su, sc.sv, float("inf"), 1)
    contrib, _, _, st = O.solve(sc, wp, wk, wP)
    E = O.accumulate(sc.su.shape[0], wp, contrib)
    assert np.count_nonzero(fixed["E"]) > 100
    np.testing.assert_allclose(E, fixed["E"], rtol=1e-12, atol=0.0)

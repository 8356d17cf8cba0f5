"""Implicit-differentiation irradiance bound of two-vertex chains whose first vertex reflects (Sec. 4.4,
"Implicit differentiation": the specular constraint at the last specular vertex in u1 and u_k, with
u2 substituted by its exact rational function of u1) in the oracle:

* on the path manifold the homogenized constraints F~, G~ vanish (relative to their size off it) and
  the irradiance from the implicit Jacobian equals the direct chain evaluator's (dual-number
  derivatives through both vertices), for both vectors b, at a mirror (periscope) and a refracting
  (mirror_glass) second vertex;
* every swept chain of a record that reaches the receiver through T2 lies in [E_lo, E_hi];
* with subdivision the bound becomes finite on most records and tight where finite.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19163_gb300 import scenes as S


def depth_of(rec):
    return ((rec["flags"] >> 24) & 63).astype(np.int32)


def chain_records(sc, bounded_only=False):
    e, t1, cell, t2 = O.pair_candidates(sc, n_threads=8)
    rec = O.bound_pairs(sc, e, t1, cell, t2, n_threads=8)
    keep = (rec["flags"] & O.LIVE) != 0
    if bounded_only:
        keep &= (rec["flags"] & O.POS_UNBOUNDED) == 0
    return rec[keep]


def cell_uv(r, a, b):
    C = O.cell_corners(int(r["cell"]), int(depth_of(r)))
    return (C[0, 0] + a * (C[1, 0] - C[0, 0]) + b * (C[2, 0] - C[0, 0]),
            C[0, 1] + a * (C[1, 1] - C[0, 1]) + b * (C[2, 1] - C[0, 1]))


def swept_chains(sc, r, k):
    """Chains of the record's cell that pass through T2, forward, onto the receiver: E."""
    a, b = np.meshgrid(np.linspace(0, 1, k), np.linspace(0, 1, k))
    m = a + b <= 1
    u, v = cell_uv(r, a[m], b[m])
    P = O.eval_pair(sc, int(r["emitter"]), int(r["tri0"]), int(r["tri1"]), u, v)
    ok = (np.isfinite(P["E"]) & (P["t1"] > 0) & (P["t2"] > 0) & (P["u2"] >= 0) & (P["v2"] >= 0)
          & (P["u2"] + P["v2"] <= 1) & (P["uk"] >= 0) & (P["uk"] <= 1) & (P["vk"] >= 0) & (P["vk"] <= 1))
    return P["E"][ok]


def bounds(sc, live):
    return O.implicit_bound_pairs(sc, live["emitter"], live["tri0"], live["cell"], depth_of(live), live["tri1"],
                                  live["u_lo"], live["u_hi"], live["v_lo"], live["v_hi"], n_threads=8)


@pytest.mark.parametrize("name", ["periscope", "mirror_glass"])
def test_chain_forms_on_the_manifold(name):
    sc = S.config(name, n=4, depth=1, amp=0.04)
    live = chain_records(sc)
    rng = np.random.default_rng(0)
    checked = 0
    for r in live[:40]:
        box = (r["u_lo"], r["u_hi"], r["v_lo"], r["v_hi"])
        if box[1] <= box[0] or box[3] <= box[2]:
            continue
        a = rng.uniform(0, 1, 30)
        b = rng.uniform(0, 1, 30) * (1 - a)
        u, v = cell_uv(r, a, b)
        P = O.eval_pair(sc, int(r["emitter"]), int(r["tri0"]), int(r["tri1"]), u, v)
        ok = (np.isfinite(P["E"]) & (P["t1"] > 0) & (P["t2"] > 0) & (P["uk"] >= box[0]) & (P["uk"] <= box[1])
              & (P["vk"] >= box[2]) & (P["vk"] <= box[3]))
        if not ok.any():
            continue
        s = (P["uk"][ok] - box[0]) / (box[1] - box[0])
        t = (P["vk"][ok] - box[2]) / (box[3] - box[2])
        for wb in (0, 1):
            args = (sc, int(r["emitter"]), int(r["tri0"]), int(r["cell"]), int(depth_of(r)), int(r["tri1"]), box, wb)
            f = O.implicit_eval_pair(*args, a[ok], b[ok], s, t)
            off = O.implicit_eval_pair(*args, a, b, rng.uniform(0, 1, 30), rng.uniform(0, 1, 30))
            assert np.all(np.abs(f["F"]) <= 1e-9 * np.max(np.abs(off["F"])))
            assert np.all(np.abs(f["G"]) <= 1e-9 * np.max(np.abs(off["G"])))
            np.testing.assert_allclose(f["E"], P["E"][ok], rtol=1e-8)
            checked += int(ok.sum())
    assert checked > 1000


@pytest.mark.parametrize("name", ["periscope", "mirror_glass"])
def test_chain_bound_contains_every_chain(name):
    sc = S.config(name, n=2, depth=3, amp=0.04)
    live = chain_records(sc)
    lo, hi = bounds(sc, live)
    assert np.all(lo <= hi)
    checked = 0
    for i, r in enumerate(live):
        E = swept_chains(sc, r, 12)
        if E.size == 0:
            continue
        assert np.all(E <= hi[i] * (1 + 1e-9)), (i, E.max(), hi[i])
        assert np.all(E >= lo[i] * (1 - 1e-9)), (i, E.min(), lo[i])
        checked += E.size
    assert checked > 2000
    assert np.isfinite(hi).sum() > 30


def test_chain_bound_converges_under_subdivision():
    """Finite on more records at every level (det A's sign certified on smaller cells and boxes),
    and within 1.3x of the largest swept irradiance at the median where finite."""
    frac, med = [], None
    for depth in (2, 3, 4):
        sc = S.config("periscope", n=2, depth=depth, amp=0.04)
        live = chain_records(sc, bounded_only=True)
        _, hi = bounds(sc, live)
        frac.append(np.isfinite(hi).mean())
        if depth == 4:
            pick = np.random.default_rng(0).choice(len(live), 120, replace=False)
            ratio = []
            for i in pick:
                E = swept_chains(sc, live[i], 14)
                if E.size and np.isfinite(hi[i]):
                    ratio.append(hi[i] / E.max())
            med = float(np.median(ratio))
    assert frac[0] < frac[1] < frac[2] and frac[2] > 0.6, frac
    assert 1.0 <= med < 1.3, med

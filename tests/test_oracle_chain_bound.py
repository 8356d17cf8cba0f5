"""Pins of the oracle's irradiance bound of two-vertex chains (refract-refract slabs, and chains
with a reflecting vertex): the chain map of the direct evaluator in interval arithmetic with
forward-mode derivatives over the cell (Eq. eq_dwda through both vertices).

* Containment: every chain found by a dense sweep of a live record's cell that passes through T2
  and reaches the receiver has its irradiance (the direct evaluator's GGT form, dual-number
  Jacobian) inside [E_lo, E_hi] -- zero violations, on curved slabs, on the 48^2 workload slab and
  on mirror chains.
* Closed form: on the flat slab every chain's irradiance is E = I0 h r / ((r^2 + h^2)^(3/2) rho
  rho'(r)); the bounds hold it, and E_hi / max E over the cell falls toward 1 under subdivision
  (1.97, 1.55, 1.16 at depths 3, 4, 5: the interval enclosure of the derivatives shrinks with the
  cell).
* The bound is finite on the workload slab (every live record of a 48^2 slab sample), so
  Algorithm 1 samples chains with P < 1.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19163_gb300 import scenes as S
from test_oracle_pairs import e_closed, flat_slab, receiver_xy, rho_of_r, sweep_cell, through_t2, tri_points


def chains_of(sc, r, k):
    u, v = sweep_cell(sc.depth, r["cell"], k)
    P = O.eval_pair(sc, int(r["emitter"]), int(r["tri0"]), int(r["tri1"]), u, v)
    h = through_t2(P) & (P["t2"] > 0) & np.isfinite(P["E"])
    return u[h], v[h], P["E"][h]


def containment(sc, k=18, max_records=None, seed=0):
    rec = O.bound_pair_scene(sc, irradiance=True, n_threads=8)
    live = rec[(rec["flags"] & O.LIVE) != 0]
    if max_records is not None and live.shape[0] > max_records:
        live = live[np.random.default_rng(seed).choice(live.shape[0], max_records, replace=False)]
    viol = checked = 0
    ratios = []
    for r in live:
        if not np.isfinite(r["e_hi"]):
            continue
        _, _, E = chains_of(sc, r, k)
        if E.size == 0:
            continue
        checked += E.size
        viol += int(np.sum((E > r["e_hi"] * (1 + 1e-12)) | (E < r["e_lo"] * (1 - 1e-12))))
        ratios.append(r["e_hi"] / E.max())
    finite = float(np.mean(np.isfinite(live["e_hi"]))) if live.shape[0] else 0.0
    return viol, checked, finite, np.array(ratios)


@pytest.mark.parametrize("name,kw", [("slab", dict(n=6, depth=2, amp=0.02)),
                                     ("slab", dict(n=6, depth=2, amp=0.05, lights=[(0.3, -0.2, 1.5)])),
                                     ("slab", dict(n=4, depth=3, amp=0.08)),
                                     ("periscope", dict(n=4, depth=2, amp=0.04)),
                                     ("mirror_glass", dict(n=4, depth=2, amp=0.04))])
def test_swept_chains_lie_in_their_irradiance_bounds(name, kw):
    sc = S.config(name, **kw)
    viol, checked, finite, ratios = containment(sc)
    print(name, kw, "finite", finite, "checked", checked, "median E_hi/max", np.median(ratios))
    assert checked > 3000
    assert viol == 0
    assert finite > 0.5 and np.all(ratios >= 1.0 - 1e-12)


def test_workload_slab_bounds_are_finite_and_tight():
    """A seeded sample of the 48^2 slab's live records (depth 2): every bound finite, every swept
    chain inside it, E_hi within 2x of the swept maximum on 90% of them."""
    sc = S.config("slab48")
    viol, checked, finite, ratios = containment(sc, k=12, max_records=300, seed=3)
    print("slab48 finite", finite, "median", np.median(ratios), "p90", np.percentile(ratios, 90))
    assert viol == 0 and checked > 3000
    assert finite == 1.0
    assert np.percentile(ratios, 90) < 2.0


def test_flat_slab_closed_form_and_tightening():
    med = []
    for depth in (3, 4, 5):  # the flat slab's 8 triangles are large: cells of 1/8 to 1/32 of a side
        sc = flat_slab(depth=depth, points=8)
        rec = O.bound_pair_scene(sc, irradiance=True, n_threads=8)
        live = rec[((rec["flags"] & O.LIVE) != 0) & np.isfinite(rec["e_hi"])]
        assert live.shape[0] > 10
        rs = []
        for r in live[:: max(1, live.shape[0] // 60)]:
            u, v, E = chains_of(sc, r, 14)
            if E.size < 5:
                continue
            x1 = tri_points(sc.s1, int(r["tri0"]), u, v)[:, :2]
            rr = np.linalg.norm(x1, axis=1)
            keep = rr > 1e-9  # on the axis the closed form is 0/0
            E, rr = E[keep], rr[keep]
            if E.size < 5:
                continue
            Ec = np.array([e_closed(a) for a in rr])
            np.testing.assert_allclose(E, Ec, rtol=1e-9)  # the evaluator on the flat slab
            assert np.all(Ec <= r["e_hi"] * (1 + 1e-12)) and np.all(Ec >= r["e_lo"] * (1 - 1e-12))
            rs.append(r["e_hi"] / Ec.max())
        med.append(float(np.median(rs)))
    print("median E_hi / max E by depth", med)
    assert med[2] < med[1] < med[0]
    assert med[2] < 1.25


@pytest.mark.parametrize("name,kw", [("slab", dict(n=6, depth=2, amp=0.02)),
                                     ("slab", dict(n=4, depth=6, amp=0.02, extent=1.0, lights=[(0.05, 0.03, 0.3)],
                                                   rec_half=3.0)),
                                     ("mirror_glass", dict(n=4, depth=3, amp=0.04))])
def test_box_factors_enclose_sampled_factors(name, kw):
    """Per box (a cell's barycentric bounding box): the intervals of s = |x1 - x0|^2 and of det du_k/du1
    hold every sampled chain's values (the direct evaluator's dual-number Jacobian), and the box's
    E_hi / E_lo bound the irradiance formed from the separately extremal sampled factors,
    I0 |C1| / (|N_k| s^(3/2) |det|) at (min s, min |det|) and (max s, max |det|): each factor is
    enclosed on its own."""
    sc = S.config(name, **kw)
    rec = O.bound_pair_scene(sc, irradiance=True, n_threads=8)
    live = rec[((rec["flags"] & O.LIVE) != 0) & np.isfinite(rec["e_hi"]) & (rec["e_hi"] > 0)]
    live = live[np.random.default_rng(1).choice(live.shape[0], min(150, live.shape[0]), replace=False)]
    Rc = sc.receiver
    nk = np.linalg.norm(np.cross(np.asarray(Rc.e1, np.float64), np.asarray(Rc.e2, np.float64)))
    checked = 0
    for r in live:
        C = O.cell_corners(int(r["cell"]), sc.depth)
        box = dict(u0=C[:, 0].min(), u1=C[:, 0].max(), v0=C[:, 1].min(), v1=C[:, 1].max())
        b = O.chain_box(sc, int(r["emitter"]), int(r["tri0"]), int(r["tri1"]), **box)
        if b["rc"] != 0:
            continue  # this record needed sub-boxes: covered by the containment tests
        u, v, E = chains_of(sc, r, 12)
        if E.size < 3:
            continue
        P = O.eval_pair(sc, int(r["emitter"]), int(r["tri0"]), int(r["tri1"]), u, v)
        x0 = np.array([sc.emitters.x[int(r["emitter"])], sc.emitters.y[int(r["emitter"])],
                       sc.emitters.z[int(r["emitter"])]], np.float64)
        x1 = tri_points(sc.s1, int(r["tri0"]), u, v)
        s = np.sum((x1 - x0) ** 2, axis=1)
        det = O.eval_pair(sc, int(r["emitter"]), int(r["tri0"]), int(r["tri1"]), u, v)["detJ"]
        assert np.all(s >= b["s"][0] * (1 - 1e-12)) and np.all(s <= b["s"][1] * (1 + 1e-12))
        assert np.all(det >= b["det"][0] - 1e-12 * np.abs(det)) and np.all(det <= b["det"][1] + 1e-12 * np.abs(det))
        i = [int(sc.s1.i0[int(r["tri0"])]), int(sc.s1.i1[int(r["tri0"])]), int(sc.s1.i2[int(r["tri0"])])]
        Pt = np.stack([sc.s1.px, sc.s1.py, sc.s1.pz], 1).astype(np.float64)[i]
        K = float(sc.emitters.intensity[int(r["emitter"])]) * abs(np.dot(Pt[0] - x0, np.cross(Pt[1] - Pt[0], Pt[2] - Pt[0]))) / nk
        ad = np.abs(det)
        assert b["e_hi"] >= K / (s.min() ** 1.5 * ad.min()) * (1 - 1e-12)
        assert b["e_lo"] <= K / (s.max() ** 1.5 * ad.max()) * (1 + 1e-12)
        checked += 1
    print(name, kw, "boxes checked", checked)
    assert checked >= 25

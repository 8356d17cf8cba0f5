"""The implicit-differentiation irradiance bound of a single refraction (Sec. 4.4, "Implicit
differentiation", with the specular polynomials F, G of its footnote) in the oracle:

* on the manifold of true paths (u1 in the cell, u_k its receiver hit) F and G vanish, and the
  irradiance from the implicit Jacobian |det B| / |det A| equals the direct path's (dual-number
  forward derivatives, an independent route), for both vectors b;
* every true path's irradiance in a cell lies in [E_lo, E_hi];
* near total internal reflection the explicit bound is loose or infinite while the implicit one is
  finite and tighter (the claim of Fig. fig_refraction), and the implicit bound tightens with depth;
* each of the footnote's two vectors b certifies cells where the other's det A changes sign, and the
  combined bound is the tighter of the two.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19163_gb300 import scenes as S


def cell_points(rec, depth, k):
    C = O.cell_corners(int(rec["cell"]), depth)
    a, b = np.meshgrid(np.linspace(0, 1, k), np.linspace(0, 1, k))
    m = a + b <= 1
    a, b = a[m], b[m]
    u = C[0, 0] + a * (C[1, 0] - C[0, 0]) + b * (C[2, 0] - C[0, 0])
    v = C[0, 1] + a * (C[1, 1] - C[0, 1]) + b * (C[2, 1] - C[0, 1])
    return a, b, u, v


def depth_of(rec):
    return ((rec["flags"] >> 24) & 63).astype(np.int32)


def live_records(sc):
    rec = O.bound(sc, n_threads=8)
    return rec[(rec["flags"] & O.LIVE) != 0]


def true_paths(sc, r, k):
    """Direct paths of the cell that land on the receiver, in front: cell barycentrics, u_k, E."""
    a, b, u, v = cell_points(r, int(depth_of(r)), k)
    uk, vk, E, t = O.eval_path(sc, int(r["emitter"]), int(r["tri0"]), u, v, direct=True)
    ok = np.isfinite(E) & (t > 0) & (uk >= 0) & (uk <= 1) & (vk >= 0) & (vk <= 1)
    return a[ok], b[ok], uk[ok], vk[ok], E[ok]


def scene_consts(sc, r):
    T = sc.s1
    t = int(r["tri0"])
    P = np.stack([T.px, T.py, T.pz], 1).astype(np.float64)
    i0, i1, i2 = T.i0[t], T.i1[t], T.i2[t]
    N1 = np.cross(P[i1] - P[i0], P[i2] - P[i0])
    e = int(r["emitter"])
    x0 = np.array([sc.emitters.x[e], sc.emitters.y[e], sc.emitters.z[e]], np.float64)
    rc = sc.receiver
    Nk = np.linalg.norm(np.cross(np.asarray(rc.e1, np.float64), np.asarray(rc.e2, np.float64)))
    return float(sc.emitters.intensity[e]) * abs(np.dot(P[i0] - x0, N1)) / Nk


@pytest.mark.parametrize("name,kw", [("water", dict(n=4, depth=1)), ("tir_wall", dict(depth=2))])
def test_implicit_forms_on_the_manifold(name, kw):
    sc = S.config(name, **kw)
    live = live_records(sc)
    checked = 0
    for r in live:
        a, b, uk, vk, E = true_paths(sc, r, 8)
        box = (r["u_lo"], r["u_hi"], r["v_lo"], r["v_hi"])
        inb = (uk >= box[0]) & (uk <= box[1]) & (vk >= box[2]) & (vk <= box[3])
        if not inb.any() or box[1] <= box[0] or box[3] <= box[2]:
            continue
        s = (uk[inb] - box[0]) / (box[1] - box[0])
        t = (vk[inb] - box[2]) / (box[3] - box[2])
        k = scene_consts(sc, r)
        for wb in (0, 1):
            f = O.implicit_eval(sc, int(r["emitter"]), int(r["tri0"]), int(r["cell"]), int(depth_of(r)), box, wb,
                                a[inb], b[inb], s, t)
            # F and G vanish (relative to the size of their terms, |d|^4 and |d|^2 scale)
            assert np.all(np.abs(f["G"]) <= 1e-12 * (1 + f["L0"])), np.max(np.abs(f["G"]))
            assert np.all(np.abs(f["F"]) <= 1e-12 * (1 + f["L0"]) ** 3), np.max(np.abs(f["F"]))
            Ei = k * np.abs(f["detB"]) / (f["L0"] ** 1.5 * np.abs(f["detA"]))
            np.testing.assert_allclose(Ei, E[inb], rtol=1e-7)
            checked += int(inb.sum())
    assert checked > 400


@pytest.mark.parametrize("name,kw", [("water", dict(n=4, depth=2)), ("tir_wall", dict(depth=3))])
def test_implicit_bound_contains_every_path(name, kw):
    sc = S.config(name, **kw)
    live = live_records(sc)
    lo, hi = O.implicit_bound(sc, live["emitter"], live["tri0"], live["cell"], depth_of(live), live["u_lo"],
                              live["u_hi"], live["v_lo"], live["v_hi"], n_threads=8)
    assert np.all(lo <= hi)
    checked = 0
    for i, r in enumerate(live):
        _, _, _, _, E = true_paths(sc, r, 12)
        if E.size == 0:
            continue
        assert np.all(E <= hi[i] * (1 + 1e-9)), (i, E.max(), hi[i])
        assert np.all(E >= lo[i] * (1 - 1e-9)), (i, E.min(), lo[i])
        checked += E.size
    assert checked > 2000
    assert np.mean(np.isfinite(hi)) > 0.5


def tightness(sc):
    """Per live cell with paths on the receiver: (explicit E_hi, implicit E_hi) / true max."""
    live = live_records(sc)
    _, hi = O.implicit_bound(sc, live["emitter"], live["tri0"], live["cell"], depth_of(live), live["u_lo"],
                             live["u_hi"], live["v_lo"], live["v_hi"], n_threads=8)
    ex, im = [], []
    for i, r in enumerate(live):
        _, _, _, _, E = true_paths(sc, r, 12)
        if E.size == 0:
            continue
        ex.append(r["e_hi"] / E.max())
        im.append(hi[i] / E.max())
    return np.array(ex), np.array(im)


def test_implicit_bound_is_tight_near_total_internal_reflection():
    """Fig. fig_refraction: near TIR the explicit bound (sqrt(beta) by a remainder variable) is
    loose or infinite; the implicit one is finite and tighter on every such cell."""
    ex, im = tightness(S.config("tir_wall", depth=4))
    loose = ~(ex <= 10.0)  # includes +inf
    assert loose.sum() >= 20
    assert np.all(np.isfinite(im[loose]))
    assert np.all(im[loose] < ex[loose])
    assert np.median(im[loose]) < 3.0


def test_implicit_bound_tightens_with_depth():
    med = [np.median(tightness(S.config("tir_wall", depth=d))[1]) for d in (2, 3, 4)]
    assert med[0] > med[1] > med[2] >= 1.0, med
    assert med[2] < 1.5, med


def test_two_vectors_b_cover_each_others_degenerate_cells():
    """The footnote's reason for intersecting the bounds of b1 = (1,0,0) and b2 = (0,1,0): where
    (d0 x n1).b vanishes inside a cell, det A of that b changes sign and its bound is +inf; the
    other b certifies most such cells.  The combined bound is the smaller E_hi and larger E_lo."""
    sc = S.config("water", n=4, depth=2)
    live = live_records(sc)
    args = (sc, live["emitter"], live["tri0"], live["cell"], depth_of(live), live["u_lo"], live["u_hi"],
            live["v_lo"], live["v_hi"])
    (lo1, hi1), (lo2, hi2), (lo, hi) = (O.implicit_bound(*args, n_threads=8, b_mask=m) for m in (1, 2, 3))
    f1, f2 = np.isfinite(hi1), np.isfinite(hi2)
    assert np.sum(f1 & ~f2) >= 20 and np.sum(f2 & ~f1) >= 20
    np.testing.assert_array_equal(hi, np.minimum(hi1, hi2))
    np.testing.assert_array_equal(lo, np.maximum(lo1, lo2))
    assert np.sum(np.isfinite(hi)) > max(f1.sum(), f2.sum())

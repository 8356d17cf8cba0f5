"""Pins of the oracle's two-vertex (refraction -> refraction) path against what the geometry fixes.

* A flat slab with flat normals has a closed form: a ray from the light (0,0,h) that meets the top
  at radius r is shifted by D tan(theta_t) inside the slab (sin theta_t = eta1' r / sqrt(r^2+h^2))
  and leaves at sin(theta_3) = eta2' sin(theta_t), so it lands at radius
  rho(r) = r + D tan(theta_t) + L tan(theta_3) (L: bottom face to receiver), at the same azimuth, with
  irradiance E = I0 h r / ((r^2 + h^2)^(3/2) rho rho'(r)) (flux through an annulus).
* On curved slabs: every path found by a dense sweep of a cell lies in the cell's box (zero
  violations), every (cell, T2) through which a swept ray passes is a candidate (tuple
  construction prunes nothing that carries a path), boxes tighten toward the image under
  subdivision, and the estimator equals exhaustive enumeration of every (T1, T2) pair.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19163_gb300 import scenes as S

H = 2.0
# the scene stores its inputs in float32: the bottom face sits at float32(-0.2) and eta' = 1/1.5 is
# not exact, so the thickness and the exit angle (sin theta_3 = eta2' sin theta_t) use the stored values
D = -float(np.float32(-0.2))
L_REC = float(np.float32(-0.2)) + 1.0
ETA1, ETA2 = float(np.float32(1.0 / 1.5)), float(np.float32(1.5))


def flat_slab(**kw):
    return S.config("slab", n=kw.pop("n", 2), extent=1.0, flat=True, lights=[(0.0, 0.0, H)], rec_half=1.5,
                    thickness=0.2, **kw)


def _sines(r):
    s1 = ETA1 * r / math.sqrt(r * r + H * H)
    return s1, ETA2 * s1, ETA1 * H * H / (r * r + H * H) ** 1.5


def rho_of_r(r):
    s1, s3, _ = _sines(r)
    return r + D * s1 / math.sqrt(1.0 - s1 * s1) + L_REC * s3 / math.sqrt(1.0 - s3 * s3)


def drho_dr(r):
    s1, s3, ds1 = _sines(r)
    return 1.0 + D * ds1 / (1.0 - s1 * s1) ** 1.5 + L_REC * ETA2 * ds1 / (1.0 - s3 * s3) ** 1.5


def e_closed(r):
    return H * r / ((r * r + H * H) ** 1.5 * rho_of_r(r) * drho_dr(r))


def tri_points(s, t, u, v):
    i = [int(s.i0[t]), int(s.i1[t]), int(s.i2[t])]
    P = np.stack([s.px, s.py, s.pz], 1).astype(np.float64)[i]
    return P[0] + np.outer(u, P[1] - P[0]) + np.outer(v, P[2] - P[0])


def receiver_xy(sc, uk, vk):
    r = sc.receiver
    X = np.asarray(r.p0, np.float64)[None, :] + np.outer(uk, r.e1) + np.outer(vk, r.e2)
    return X[:, :2]


def test_flat_slab_chain_matches_closed_form():
    sc = flat_slab()
    rng = np.random.default_rng(0)
    for t in range(sc.s1.n_tris):
        u = rng.uniform(0, 1, 50)
        v = rng.uniform(0, 1, 50) * (1 - u)
        P = O.eval_pair(sc, 0, t, 0, u, v)  # the flat bottom: every T2 spans the same plane
        x1 = tri_points(sc.s1, t, u, v)[:, :2]
        X = receiver_xy(sc, P["uk"], P["vk"])
        r = np.linalg.norm(x1, axis=1)
        rho = np.linalg.norm(X, axis=1)
        np.testing.assert_allclose(rho, [rho_of_r(a) for a in r], rtol=1e-12, atol=1e-12)
        # same azimuth: X parallel to x1
        np.testing.assert_allclose(X[:, 0] * x1[:, 1] - X[:, 1] * x1[:, 0], 0.0, atol=1e-12)
        np.testing.assert_allclose(P["E"], [e_closed(a) for a in r], rtol=1e-10)
        assert np.all(P["t1"] > 0) and np.all(P["t2"] > 0)


def test_flat_slab_render_matches_closed_form():
    """Candidates -> pair bounds -> index -> Algorithm 1 (P = 1: chains carry no irradiance bound)
    -> Newton -> estimate: each point of the flat slab is reached by exactly one path."""
    sc = flat_slab(points=24, depth=1)
    out = O.render_pairs(sc, gamma=1.0, seed=3)
    X = receiver_xy(sc, sc.su.astype(np.float64), sc.sv.astype(np.float64))
    rho = np.linalg.norm(X, axis=1)
    r_max = 1.0  # the slab covers [-1,1]^2
    ok = 0
    for p in range(sc.su.shape[0]):
        lo, hi = 0.0, 3.0
        for _ in range(200):  # bisection of the monotone rho(r) = rho_p
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if rho_of_r(mid) < rho[p] else (lo, mid)
        r = 0.5 * (lo + hi)
        x1 = r * X[p] / rho[p]
        s1 = ETA1 * r / math.sqrt(r * r + H * H)
        x2 = x1 * (1.0 + D * s1 / math.sqrt(1.0 - s1 * s1) / r)  # exit point on the bottom face
        edge = max(np.max(np.abs(x1)), np.max(np.abs(x2)))
        if edge > r_max + 1e-6:
            assert out["E"][p] == 0.0  # the chain leaves through the slab's side: no TT path
            continue
        if edge > r_max - 1e-3:
            continue  # near the slab's rim
        assert out["E"][p] == pytest.approx(e_closed(r), rel=1e-9)
        ok += 1
    assert ok > 300
    assert np.all(out["wl_p"] == 1.0)


def sweep_cell(depth, cell, k=30):
    C = O.cell_corners(int(cell), depth)
    a, b = np.meshgrid(np.linspace(0, 1, k), np.linspace(0, 1, k))
    m = a + b <= 1
    a, b = a[m], b[m]
    return (C[0, 0] + a * (C[1, 0] - C[0, 0]) + b * (C[2, 0] - C[0, 0]),
            C[0, 1] + a * (C[1, 1] - C[0, 1]) + b * (C[2, 1] - C[0, 1]))


def through_t2(P):
    return (np.isfinite(P["uk"]) & (P["u2"] >= 0) & (P["v2"] >= 0) & (P["u2"] + P["v2"] <= 1) & (P["t1"] > 0))


# (n, depth, amplitude): the last case has large, strongly curved cells, where the remainder of the
# sqrt chord (the xi faces) and the degree reduction are large enough for a sweep to resolve them
@pytest.mark.parametrize("n,depth,amp,k", [(4, 1, 0.02, 30), (4, 1, 0.06, 30), (2, 0, 0.15, 90)])
def test_pair_boxes_contain_dense_sweep_and_prune_nothing(n, depth, amp, k):
    check_containment(S.config("slab", n=n, depth=depth, amp=amp), depth, k)


# reflection at the first vertex (then a mirror or a refracting interface), curved faces
@pytest.mark.parametrize("name,amp", [("periscope", 0.04), ("mirror_glass", 0.04), ("periscope", 0.12)])
def test_reflecting_chains_contain_dense_sweep_and_prune_nothing(name, amp):
    check_containment(S.config(name, n=4, depth=1, amp=amp), 1, 30)


def test_flat_periscope_closed_form():
    """Two flat parallel mirrors (z = 0 facing up, z = 1 facing down) and a light at (0,0,2): the
    chain unfolds into the straight ray from the double image (0,0,4), so the hit on the receiver
    z = 0.5 is x3 = 1.75 x1 and E = I0 3.5 / |x3 - (0,0,4)|^3."""
    sc = S.config("periscope", n=2, flat=True, extent=1.0, lights=[(0.0, 0.0, 2.0)], rec_half=1.5)
    rng = np.random.default_rng(2)
    for t in range(sc.s1.n_tris):
        u = rng.uniform(0, 1, 40)
        v = rng.uniform(0, 1, 40) * (1 - u)
        P = O.eval_pair(sc, 0, t, 0, u, v)
        x1 = tri_points(sc.s1, t, u, v)[:, :2]
        X = receiver_xy(sc, P["uk"], P["vk"])
        np.testing.assert_allclose(X, 1.75 * x1, atol=1e-12)
        np.testing.assert_allclose(P["E"], 3.5 / (np.sum(X ** 2, axis=1) + 3.5 ** 2) ** 1.5, rtol=1e-12)


def check_containment(sc, depth, k):
    e, t1, cell, t2 = O.pair_candidates(sc)
    cand = set(zip(e.tolist(), t1.tolist(), cell.tolist(), t2.tolist()))
    rec = O.bound_pairs(sc, e, t1, cell, t2)
    recs = {(int(r["emitter"]), int(r["tri0"]), int(r["cell"]), int(r["tri1"])): r for r in rec}
    viol = checked = 0
    for t in range(sc.s1.n_tris):
        for c in range(4 ** depth):
            u, v = sweep_cell(depth, c, k)
            for b in range(sc.s2.n_tris):
                P = O.eval_pair(sc, 0, t, b, u, v)
                hit = through_t2(P)
                if not hit.any():
                    continue
                # tuple construction never drops a (cell, T2) that a ray of the cell passes through
                assert (0, t, c, b) in cand
                r = recs[(0, t, c, b)]
                ok = hit & (P["t2"] > 0) & (P["uk"] >= 0) & (P["uk"] <= 1) & (P["vk"] >= 0) & (P["vk"] <= 1)
                if not ok.any():
                    continue
                assert r["flags"] & O.LIVE
                checked += int(ok.sum())
                uk, vk = P["uk"][ok], P["vk"][ok]
                viol += int(np.sum((uk < r["u_lo"]) | (uk > r["u_hi"]) | (vk < r["v_lo"]) | (vk > r["v_hi"])))
    assert checked > 2000
    assert viol == 0


def test_pair_boxes_tighten_under_subdivision():
    ratios = []
    for depth in (0, 1, 2, 3):
        sc = S.config("slab", n=4, depth=depth, amp=0.04)
        e, t1, cell, t2 = O.pair_candidates(sc)
        rec = O.bound_pairs(sc, e, t1, cell, t2)
        live = rec[(rec["flags"] & O.LIVE) != 0]
        rs = []
        for r in live[:: max(1, live.shape[0] // 40)]:
            u, v = sweep_cell(depth, r["cell"], 40)
            P = O.eval_pair(sc, int(r["emitter"]), int(r["tri0"]), int(r["tri1"]), u, v)
            f = np.isfinite(P["uk"])
            if f.sum() < 10 or (r["flags"] & O.POS_UNBOUNDED):
                continue
            rs.append((r["u_hi"] - r["u_lo"] + r["v_hi"] - r["v_lo"]) /
                      (np.ptp(np.clip(P["uk"][f], 0, 1)) + np.ptp(np.clip(P["vk"][f], 0, 1))))
        ratios.append(float(np.median(rs)))
    assert all(x >= 1.0 - 1e-9 for x in ratios)
    assert ratios[3] < ratios[0] and ratios[3] < 1.01


@pytest.mark.parametrize("name", ["slab", "periscope", "mirror_glass"])
def test_estimator_equals_exhaustive_enumeration(name):
    """With P = 1 the estimate at a point is the sum of E over the roots of the tuples listed there;
    running the same Newton solve over every (T1, T2) pair must give the same sum: no tuple that
    carries a root was pruned by tuple construction, the bounds or the index."""
    sc = S.config(name, n=3, depth=1, amp=0.04, points=20)
    out = O.render_pairs(sc, gamma=1.0, seed=1)
    n_pts = sc.su.shape[0]
    pts = np.repeat(np.arange(n_pts), sc.s1.n_tris * sc.s2.n_tris)
    t1 = np.tile(np.repeat(np.arange(sc.s1.n_tris), sc.s2.n_tris), n_pts)
    t2 = np.tile(np.arange(sc.s2.n_tris), n_pts * sc.s1.n_tris)
    keys = O.tuple_key(0, t1.astype(np.uint64), t2.astype(np.int64))
    contrib, _, _, st = O.solve_pair(sc, pts, keys, np.ones(pts.shape[0], np.float32))
    E_all = O.accumulate(n_pts, pts, contrib)
    assert st.sum() > 50
    assert np.count_nonzero(out["E"]) > 50
    np.testing.assert_allclose(out["E"], E_all, rtol=1e-12, atol=0.0)


@pytest.mark.parametrize("name", ["slab", "periscope"])
def test_pair_gap_agrees_with_candidates_and_is_a_distance(name):
    """The gap by which T2's xy box misses a cell's footprint (the measure the GPU parity tests use
    for GPU-only candidates): <= 0 exactly for the enumerated candidates; shifting s2 by delta
    along x moves T2's box and not the footprint (same z-range), so every finite gap changes by at
    most |delta|, and by exactly |delta| where the x separation decides it."""
    import dataclasses
    sc = S.config(name, n=4, depth=1, amp=0.04)
    cand = set(zip(*[a.tolist() for a in O.pair_candidates(sc)]))
    n_c = 4 ** sc.depth
    items = [(0, t, c, b) for t in range(sc.s1.n_tris) for c in range(n_c) for b in range(sc.s2.n_tris)]
    e, t1, cell, t2 = (np.array(x) for x in zip(*items))
    gap = O.pair_gap(sc, e, t1, cell, t2)
    is_cand = np.array([it in cand for it in items])
    assert is_cand.sum() > 50 and (~is_cand).sum() > 50
    np.testing.assert_array_equal(gap <= 0, is_cand)
    delta = 0.013
    s2 = dataclasses.replace(sc.s2, px=(sc.s2.px + np.float32(delta)).astype(np.float32))
    gap2 = O.pair_gap(dataclasses.replace(sc, s2=s2), e, t1, cell, t2)
    fin = np.isfinite(gap) & np.isfinite(gap2)
    assert fin.sum() > 100
    d = np.abs(gap2[fin] - gap[fin])
    assert np.all(d <= delta + 1e-6)
    assert np.sum(np.abs(d - delta) < 1e-6) > 20


def test_flat_mirror_glass_closed_form():
    """A flat mirror at z = 0 (light (0,0,2)) and a flat glass interface at z = 1 (eta' = 1/1.5 from
    the air below), receiver z = 1.5: rotationally symmetric about the light's axis.  A ray leaving
    at theta0 from the vertical meets the mirror at r = 2 tan(theta0), the interface at 1.5 r and
    the receiver at rho = 3 tan(theta0) + 0.5 tan(theta_t), sin(theta_t) = sin(theta0) / 1.5, and
    the irradiance is I0 dOmega0 / dA = I0 sin(theta0) / (rho drho/dtheta0)."""
    sc = S.config("mirror_glass", n=2, flat=True, extent=1.0, lights=[(0.0, 0.0, 2.0)], rec_half=1.5)
    eta = float(np.float32(1.0 / 1.5))  # the surface stores eta' in float32
    rng = np.random.default_rng(5)
    checked = 0
    for t in range(sc.s1.n_tris):
        u = rng.uniform(0, 1, 40)
        v = rng.uniform(0, 1, 40) * (1 - u)
        x1 = tri_points(sc.s1, t, u, v)[:, :2]
        r = np.linalg.norm(x1, axis=1)
        ok = (np.max(np.abs(1.5 * x1), axis=1) < 1.0 - 1e-6) & (r > 1e-3)  # the interface hit is on T2's face
        for b in range(sc.s2.n_tris):
            P = O.eval_pair(sc, 0, t, b, u, v)
            hit = ok & through_t2(P) & (P["t2"] > 0)
            if not hit.any():
                continue
            th0 = np.arctan(r[hit] / 2.0)
            tht = np.arcsin(eta * np.sin(th0))
            rho = 3.0 * np.tan(th0) + 0.5 * np.tan(tht)
            drho = 3.0 / np.cos(th0) ** 2 + 0.5 / np.cos(tht) ** 2 * eta * np.cos(th0) / np.cos(tht)
            X = receiver_xy(sc, P["uk"][hit], P["vk"][hit])
            np.testing.assert_allclose(np.linalg.norm(X, axis=1), rho, rtol=1e-9)
            np.testing.assert_allclose(X / np.linalg.norm(X, axis=1)[:, None], x1[hit] / r[hit][:, None], atol=1e-9)
            np.testing.assert_allclose(P["E"][hit], np.sin(th0) / (rho * drho), rtol=1e-9)
            checked += int(hit.sum())
    assert checked > 30


# ----------------------------------------------------------------------------- remainder-form sweeps
# The bound of a pair record holds over the whole product domain of the cell and the remainder
# variables (Sec. 4.3 "Remainder variables"; Sec. 6.1 "Degree reduction"), not only on true chains:
# with W1 = a1 beta1 + b1 + delta1(xi1) at the first vertex, u2 replaced by its degree-1 interpolant
# plus any (rho_u, rho_v) in the reduction's remainder ranges, and W2 = a2 beta2 + b2 + delta2(xi2)
# at the second, every point of that domain must land in the record's box.  These sweeps evaluate
# the remainder forms pointwise (the textbook ray-plane intersection, no Bernstein arithmetic) at
# both ends of every remainder interval, so a bound that drops one xi face or one end of a
# reduction remainder misses points of the domain by the width of that remainder, which on coarse,
# steep cells under grazing light is far above the bound's slack.


def _tri(s, t):
    i = [int(s.i0[t]), int(s.i1[t]), int(s.i2[t])]
    P = np.stack([s.px, s.py, s.pz], 1).astype(np.float64)[i]
    N = np.stack([s.nx, s.ny, s.nz], 1).astype(np.float64)[i]
    return P, N


def _scatter(d, n, kind, eta, chord, xi):
    """Direction leaving a vertex with incoming d and (un-normalized) normal n: reflection
    (n.n) d - 2 (d.n) n; refraction eta' ((n.n) d - (d.n) n) - W n with W the remainder form
    a beta + b + delta_lo + xi (delta_hi - delta_lo) of sqrt(beta), beta = (1 - eta'^2)(n.n)(d.d)
    + eta'^2 (d.n)^2 (Eq. eq_refr_rational and the chord remainder of Sec. 4.3)."""
    nn = np.sum(n * n, -1)[..., None]
    dn = np.sum(d * n, -1)[..., None]
    if kind == 0:
        return nn * d - 2.0 * dn * n
    ss = np.sum(d * d, -1)[..., None]
    beta = (1.0 - eta * eta) * nn * ss + eta * eta * dn * dn
    a, b, dlo, dhi = chord
    W = a * beta + b + dlo + xi * (dhi - dlo)
    return eta * (nn * d - dn * n) - W * n


def _plane_coords(x, d, p0, e1, e2):
    """(u, v) with x + s d = p0 + u e1 + v e2 (Cramer's rule)."""
    M = np.stack([np.broadcast_to(e1, d.shape), np.broadcast_to(e2, d.shape), -d], -1)
    sol = np.linalg.solve(M, (x - p0)[..., None])[..., 0]
    return sol[..., 0], sol[..., 1]


def remainder_sweep(sc, depth, k=12):
    """Count the points of every live, bounded record's remainder domain (cell x xi1 x rho x xi2,
    remainder variables at both ends and the middle) that fall outside its intermediate bounds or
    its box.  Returns (violations by stage, points checked)."""
    e, t1, cell, t2 = O.pair_candidates(sc)
    rec, dg = O.bound_pairs_diag(sc, e, t1, cell, t2)
    s1, s2, R = sc.s1, sc.s2, sc.receiver
    p0r, e1r, e2r = (np.asarray(a, np.float64) for a in (R.p0, R.e1, R.e2))
    eta1, eta2 = float(np.float32(s1.eta)), float(np.float32(s2.eta))  # stored as float32 in the scene views
    viol = {"ratios": 0, "u2box": 0, "corner_interp": 0, "rho": 0, "box": 0}
    checked = 0
    tol = 1e-9
    for i in range(rec.shape[0]):
        r, g = rec[i], dg[i]
        if not (r["flags"] & O.LIVE) or (r["flags"] & O.POS_UNBOUNDED) or g["stage"] != 3:
            continue
        C = O.cell_corners(int(r["cell"]), depth)
        a, b = np.meshgrid(np.linspace(0, 1, k), np.linspace(0, 1, k))
        m = a + b <= 1 + 1e-12
        lam1, lam2 = a[m], b[m]
        u1 = C[0, 0] + lam1 * (C[1, 0] - C[0, 0]) + lam2 * (C[2, 0] - C[0, 0])
        v1 = C[0, 1] + lam1 * (C[1, 1] - C[0, 1]) + lam2 * (C[2, 1] - C[0, 1])
        P1, N1 = _tri(s1, int(r["tri0"]))
        P2, N2 = _tri(s2, int(r["tri1"]))
        x0 = np.array([sc.emitters.x[int(r["emitter"])], sc.emitters.y[int(r["emitter"])],
                       sc.emitters.z[int(r["emitter"])]], np.float64)
        x1 = P1[0] + u1[:, None] * (P1[1] - P1[0]) + v1[:, None] * (P1[2] - P1[0])
        n1 = N1[0] + u1[:, None] * (N1[1] - N1[0]) + v1[:, None] * (N1[2] - N1[0])
        d0 = x1 - x0
        lu = g["lu"][0] * (1 - lam1 - lam2) + g["lu"][1] * lam1 + g["lu"][2] * lam2
        lv = g["lv"][0] * (1 - lam1 - lam2) + g["lv"][1] * lam1 + g["lv"][2] * lam2
        e21, e22 = P2[1] - P2[0], P2[2] - P2[0]
        for xi1 in (0.0, 0.5, 1.0):
            d1t = _scatter(d0, n1, s1.kind, eta1, g["chord1"], xi1)
            rx, ry = d1t[:, 0] / d1t[:, 2], d1t[:, 1] / d1t[:, 2]
            viol["ratios"] += int(np.sum((rx < g["rx"][0] - tol) | (rx > g["rx"][1] + tol) |
                                         (ry < g["ry"][0] - tol) | (ry > g["ry"][1] + tol)))
            u2, v2 = _plane_coords(x1, d1t, P2[0], e21, e22)
            viol["u2box"] += int(np.sum((u2 < g["u2box"][0] - tol) | (u2 > g["u2box"][1] + tol) |
                                        (v2 < g["u2box"][2] - tol) | (v2 > g["u2box"][3] + tol)))
            viol["rho"] += int(np.sum((u2 - lu < g["rho"][0] - tol) | (u2 - lu > g["rho"][1] + tol) |
                                      (v2 - lv < g["rho"][2] - tol) | (v2 - lv > g["rho"][3] + tol)))
            if xi1 == 0.5:  # the interpolant takes u2's values at the corners at xi1 = 1/2
                corner = (np.abs(lam1) + np.abs(lam2) < 1e-12) | (np.abs(lam1 - 1) < 1e-12) | \
                    (np.abs(lam2 - 1) < 1e-12)
                viol["corner_interp"] += int(np.sum(corner & ((np.abs(u2 - lu) > 1e-9) | (np.abs(v2 - lv) > 1e-9))))
            checked += u1.shape[0]
        for ru in np.linspace(g["rho"][0], g["rho"][1], 3):
            for rv in np.linspace(g["rho"][2], g["rho"][3], 3):
                u2, v2 = lu + ru, lv + rv
                x2 = P2[0] + u2[:, None] * e21 + v2[:, None] * e22
                n2 = N2[0] + u2[:, None] * (N2[1] - N2[0]) + v2[:, None] * (N2[2] - N2[0])
                for xi2 in (0.0, 0.5, 1.0):
                    d2t = _scatter(x2 - x1, n2, s2.kind, eta2, g["chord2"], xi2)
                    uk, vk = _plane_coords(x2, d2t, p0r, e1r, e2r)
                    inu = (uk >= 0) & (uk <= 1)
                    inv = (vk >= 0) & (vk <= 1)
                    viol["box"] += int(np.sum(inu & ((uk < r["u_lo"] - tol) | (uk > r["u_hi"] + tol))))
                    viol["box"] += int(np.sum(inv & ((vk < r["v_lo"] - tol) | (vk > r["v_hi"] + tol))))
                    checked += int(np.sum(inu | inv))
    return viol, checked


# coarse, steep slabs lit from the side (large sqrt chords at both vertices, exits near the
# critical angle at the bottom face, large reduction remainders), the workloads' gentle slab, and a
# mirror followed by a refracting interface.  A planted copy of the oracle in which one xi face is
# dropped (in the direction ratios, the u2 bounds, the reduction remainder, either vertex's W, or the
# receiver ratio bound) fails this test on each of the three slab cases.
@pytest.mark.parametrize("name,kw", [("slab", dict(n=3, depth=1, amp=0.1, lights=[(0.9, -0.5, 1.0)], rec_half=3.0)),
                                     ("slab", dict(n=3, depth=1, amp=0.15, lights=[(0.5, 0.3, 1.2)], rec_half=3.0)),
                                     ("slab", dict(n=4, depth=1, amp=0.04)),
                                     ("mirror_glass", dict(n=4, depth=1, amp=0.04))])
def test_pair_bound_holds_over_the_remainder_domain(name, kw):
    depth = kw["depth"]
    sc = S.config(name, **kw)
    viol, checked = remainder_sweep(sc, depth)
    print(name, kw, viol, checked)
    assert checked > 5000
    assert all(v == 0 for v in viol.values()), viol

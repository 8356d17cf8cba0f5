"""Pins of the oracle's single-refraction path (Eq. eq_refr_rational, refraction; Sec. 4.3
"Remainder variables") against the chord's closed form, the textbook vector form of Snell's law,
angle checks at the hits, a flat-interface closed form, dense sweeps of the direct geometry and
exhaustive root enumeration on a tiny mesh."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2504_19163_gb300 import scenes as S

from test_oracle_bounds import cell_points, depth_of, sweep_violations


def flat_refract(n=4, eta=1.0 / 1.33, h=1.5, H=1.0, light=(0.0, 0.0), depth=1, half=1.5, extent=1.0):
    """Flat interface z = 0 (normal +z) over [-extent, extent]^2, light at (lx, ly, h), receiver
    plane z = -H over [-half, half]^2."""
    s1 = S.heightfield(n, 0, n_waves=1, amp_total=0.0, normals="flat_up")
    s1 = S.dataclasses.replace(s1, px=(s1.px * extent).astype(np.float32), py=(s1.py * extent).astype(np.float32),
                               kind=S.SURFACE_REFRACT, eta=float(eta))
    em = S.point_emitters([(light[0], light[1], h)], 1.0)
    rec = S.receiver_square(-H, half)
    su, sv = S.shading_points(8, 8, 3)
    return S.Scene("flat_refract", s1, None, rec, em, depth, su, sv)


def test_sqrt_chord_closed_forms(orc):
    a, b, dlo, dhi = orc.chord_sqrt(1.0, 4.0)
    assert (a, b, dlo) == pytest.approx((1 / 3, 2 / 3, 0.0), abs=1e-15)
    assert dhi == pytest.approx(1 / 12, abs=1e-15)  # at beta* = 9/4: 3/2 - 3/4 - 2/3
    for hi in (0.25, 2.0, 9.0):
        a, b, dlo, dhi = orc.chord_sqrt(0.0, hi)
        assert dhi == pytest.approx(math.sqrt(hi) / 4, rel=1e-14)
    assert orc.chord_sqrt(2.0, 2.0) == pytest.approx((0.0, math.sqrt(2.0), 0.0, 0.0))


@pytest.mark.parametrize("lo,hi", [(0.0, 1.0), (0.3, 0.31), (1e-4, 5.0), (2.0, 3.0)])
def test_sqrt_chord_envelope(orc, lo, hi):
    a, b, dlo, dhi = orc.chord_sqrt(lo, hi)
    x = np.linspace(lo, hi, 100001)
    d = np.sqrt(x) - (a * x + b)
    assert d.min() >= dlo - 1e-15 and d.max() <= dhi + 1e-15
    assert d.max() >= dhi - 1e-9 * max(1.0, dhi)  # the upper end is attained


def direct_vs_rational(orc, sc, n_tris=12, n_pts=40, seed=0):
    rng = np.random.default_rng(seed)
    for t in rng.choice(sc.s1.n_tris, min(n_tris, sc.s1.n_tris), replace=False):
        m = rng.dirichlet([1, 1, 1], size=n_pts)
        a = orc.eval_path(sc, 0, int(t), m[:, 1], m[:, 2])
        b = orc.eval_path(sc, 0, int(t), m[:, 1], m[:, 2], direct=True)
        yield a, b


def test_rational_refraction_equals_vector_snell(orc):
    """The un-normalized rational direction of Eq. eq_refr_rational and its forward derivatives
    agree with the textbook unit-vector refraction and dual-number Jacobians."""
    sc = S.config("water", n=10, steep=0.05)
    for a, b in direct_vs_rational(orc, sc):
        np.testing.assert_allclose(a[0], b[0], atol=1e-12)
        np.testing.assert_allclose(a[1], b[1], atol=1e-12)
        np.testing.assert_allclose(a[2], b[2], rtol=1e-9)
        assert np.array_equal(np.sign(a[3]), np.sign(b[3]))  # t scales with the direction's length


def test_total_internal_reflection_agrees(orc):
    """eta' = 1.5 (dense to thin) with a light close to a flat interface: both evaluators report
    no path exactly where 1 - eta'^2 sin^2(theta_i) < 0."""
    sc = flat_refract(n=2, eta=1.5, h=0.3, light=(0.0, 0.0), extent=1.0)
    P = np.stack([sc.s1.px, sc.s1.py, sc.s1.pz], 1).astype(np.float64)
    n_tir = 0
    for t in range(sc.s1.n_tris):
        rng = np.random.default_rng(t)
        m = rng.dirichlet([1, 1, 1], size=400)
        a = orc.eval_path(sc, 0, t, m[:, 1], m[:, 2])
        b = orc.eval_path(sc, 0, t, m[:, 1], m[:, 2], direct=True)
        i0, i1, i2 = sc.s1.i0[t], sc.s1.i1[t], sc.s1.i2[t]
        x1 = P[i0] + np.outer(m[:, 1], P[i1] - P[i0]) + np.outer(m[:, 2], P[i2] - P[i0])
        r = np.hypot(x1[:, 0], x1[:, 1])
        sin_i = r / np.hypot(r, 0.3)
        tir = 1.5 ** 2 * sin_i ** 2 > 1.0
        assert np.array_equal(np.isnan(a[0]), tir) and np.array_equal(np.isnan(b[0]), tir)
        n_tir += int(tir.sum())
    assert n_tir > 100


def test_snell_law_at_the_hits(orc):
    """At every evaluated path: the transmitted ray lies in the plane of incidence, on the far side,
    and eta' sin(theta_i) = sin(theta_t) (angles from numpy, independent of both evaluators)."""
    sc = S.config("water", n=10, steep=0.05)
    P = np.stack([sc.s1.px, sc.s1.py, sc.s1.pz], 1).astype(np.float64)
    N = np.stack([sc.s1.nx, sc.s1.ny, sc.s1.nz], 1).astype(np.float64)
    x0 = np.array([sc.emitters.x[0], sc.emitters.y[0], sc.emitters.z[0]], np.float64)
    r = sc.receiver
    rng = np.random.default_rng(5)
    eta = sc.s1.eta
    for t in rng.choice(sc.s1.n_tris, 10, replace=False):
        m = rng.dirichlet([1, 1, 1], size=30)
        uk, vk, E, tt = orc.eval_path(sc, 0, int(t), m[:, 1], m[:, 2])
        i0, i1, i2 = sc.s1.i0[t], sc.s1.i1[t], sc.s1.i2[t]
        x1 = P[i0] + np.outer(m[:, 1], P[i1] - P[i0]) + np.outer(m[:, 2], P[i2] - P[i0])
        n = N[i0] + np.outer(m[:, 1], N[i1] - N[i0]) + np.outer(m[:, 2], N[i2] - N[i0])
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        X = r.p0.astype(np.float64) + np.outer(uk, r.e1) + np.outer(vk, r.e2)
        di = x1 - x0
        dt = X - x1
        di /= np.linalg.norm(di, axis=1, keepdims=True)
        dt /= np.linalg.norm(dt, axis=1, keepdims=True)
        ci = np.cross(di, n)
        ct = np.cross(dt, n)
        np.testing.assert_allclose(eta * np.linalg.norm(ci, axis=1), np.linalg.norm(ct, axis=1), atol=1e-10)
        np.testing.assert_allclose(np.einsum("ij,ij->i", np.cross(ci, ct), n), 0.0, atol=1e-10)
        assert np.all(np.einsum("ij,ij->i", ci, ct) > 0)  # same side of the normal: no sign flip
        assert np.all(np.einsum("ij,ij->i", dt, n) < 0) and np.all(tt > 0)


@pytest.mark.parametrize("h,H", [(1.5, 1.0), (2.0, 0.5)])
def test_flat_interface_closed_form_and_newton(orc, h, H):
    """Flat interface, light (0,0,h), floor z = -H: a point at radius r lands at
    R(r) = r + H tan(theta_t), sin(theta_t) = eta' r / sqrt(r^2 + h^2); Newton (Sec. 6.1) on a
    target recovers the r that solves R(r) = target (bracketed root of the closed form)."""
    eta = 1.0 / 1.33
    sc = flat_refract(n=4, eta=eta, h=h, H=H, light=(0.0, 0.0), depth=1, half=1.5)
    P = np.stack([sc.s1.px, sc.s1.py, sc.s1.pz], 1).astype(np.float64)

    def Rof(r):
        st = eta * r / math.hypot(r, h)
        return r + H * st / math.sqrt(1 - st * st)

    for t in range(sc.s1.n_tris):
        rng = np.random.default_rng(t)
        m = rng.dirichlet([1, 1, 1], size=25)
        uk, vk, E, tt = orc.eval_path(sc, 0, t, m[:, 1], m[:, 2])
        i0, i1, i2 = sc.s1.i0[t], sc.s1.i1[t], sc.s1.i2[t]
        x1 = P[i0] + np.outer(m[:, 1], P[i1] - P[i0]) + np.outer(m[:, 2], P[i2] - P[i0])
        r = np.hypot(x1[:, 0], x1[:, 1])
        Xk = -1.5 + 3.0 * uk
        Yk = -1.5 + 3.0 * vk
        Rk = np.hypot(Xk, Yk)
        np.testing.assert_allclose(Rk, [Rof(q) for q in r], atol=1e-12)
        # same azimuth (the plane of incidence contains the vertical through the light)
        np.testing.assert_allclose(Xk * x1[:, 1] - Yk * x1[:, 0], 0.0, atol=1e-12)
    # Newton: targets at azimuth phi (off the mesh's grid lines); the root lies at the same
    # azimuth at the radius that solves R(r) = |target|
    phi = 0.3
    radii = [0.2, 0.7, 1.1]
    su = np.array([(R * math.cos(phi) + 1.5) / 3.0 for R in radii], np.float32)
    sv = np.array([(R * math.sin(phi) + 1.5) / 3.0 for R in radii], np.float32)
    sc.su, sc.sv = su, sv
    keys = [int(orc.tuple_key(0, t)) for p in range(3) for t in range(sc.s1.n_tris)]
    pts = [p for p in range(3) for t in range(sc.s1.n_tris)]
    contrib, ru, rv, st = orc.solve(sc, np.array(pts), np.array(keys, np.uint64), np.ones(len(keys), np.float32))
    pts = np.array(pts)
    for p in range(3):
        X, Y = -1.5 + 3.0 * float(su[p]), -1.5 + 3.0 * float(sv[p])
        r_star = brentq(lambda q: Rof(q) - math.hypot(X, Y), 0.0, math.hypot(X, Y))
        sel = (pts == p) & (st == 1)
        assert sel.sum() == 1
        i = int(np.nonzero(sel)[0][0])
        t = keys[i] & 0xFFFFFF
        i0, i1, i2 = sc.s1.i0[t], sc.s1.i1[t], sc.s1.i2[t]
        x1 = P[i0] + ru[i] * (P[i1] - P[i0]) + rv[i] * (P[i2] - P[i0])
        assert abs(math.hypot(x1[0], x1[1]) - r_star) < 1e-6  # float32 targets: 1e-5 scene-unit tolerance
        assert abs(math.atan2(x1[1], x1[0]) - math.atan2(Y, X)) < 1e-9


@pytest.mark.parametrize("kw", [dict(n=6, depth=2), dict(n=4, depth=1, steep=0.08, lights=[(0.3, 0.2, 1.2)])])
def test_refraction_bound_contains_dense_sweep(orc, kw):
    """Every refracted path that lands on the receiver region lies inside its cell's box; culled
    and TIR cells carry no such path."""
    sc = S.config("water", **kw)
    rec = orc.bound(sc)
    assert np.any(rec["flags"] & orc.LIVE)
    viol, hits = sweep_violations(orc, sc, rec, K=10)
    assert viol == 0 and hits > 200


def test_refraction_tir_cells_have_no_paths(orc):
    sc = flat_refract(n=4, eta=1.5, h=0.3, light=(0.0, 0.0), depth=2, extent=1.0, half=3.0, H=0.5)
    rec = orc.bound(sc)
    assert np.any(rec["flags"] & orc.TIR) and np.any(rec["flags"] & orc.LIVE)
    viol, hits = sweep_violations(orc, sc, rec, K=8)
    assert viol == 0 and hits > 100


def test_refraction_boxes_converge_under_subdivision(orc):
    """The box of a cell approaches the true image of the cell as the cell shrinks (Sec. 4.1's
    convergence; the chord's remainder shrinks quadratically with beta's range)."""
    sc = S.config("water", n=4, steep=0.05)
    ratios = []
    for d in (0, 2, 4):
        rec = orc.bound(sc, depth=d)
        live = rec[(rec["flags"] & orc.LIVE) != 0]
        r = []
        for row in live[:: max(1, len(live) // 20)]:
            u, v = cell_points(orc, row["cell"], depth_of(np.array([row]))[0], 12)
            uk, vk, _, _ = orc.eval_path(sc, int(row["emitter"]), int(row["tri0"]), u, v, direct=True)
            if np.all((uk > 0) & (uk < 1) & (vk > 0) & (vk < 1)):
                r.append((row["u_hi"] - row["u_lo"]) / (uk.max() - uk.min()))
        ratios.append(np.median(r))
    assert ratios[0] > ratios[1] > ratios[2] >= 1.0 - 1e-9
    assert ratios[2] - 1.0 < 0.1 * (ratios[0] - 1.0)


def test_refraction_estimate_matches_root_enumeration(orc):
    """With every listed tuple selected (gamma = +inf, so P = 1), the whole path's estimate at each
    point is the sum of E over the roots, enumerated here independently (dense grid + Newton on
    the direct evaluator) on a tiny mesh; every root's tuple carries E~ >= E."""
    sc = S.config("water", n=3, depth=1, points=6, steep=0.05)
    out = orc.render(sc, gamma=float("inf"), seed=3)
    E_est = out["E"]
    assert np.all(out["wl_p"] == 1.0)
    roots = out["status"] == 1
    assert np.all(out["contrib"][roots] <= out["etilde"].max())  # E(root) / 1 below the largest E~
    P = np.stack([sc.s1.px, sc.s1.py, sc.s1.pz], 1).astype(np.float64)
    K = 60
    mu = np.array([(i / K, j / K) for i in range(K + 1) for j in range(K + 1 - i)])
    E_ref = np.zeros(sc.su.shape[0])
    for t in range(sc.s1.n_tris):
        uk, vk, E, tt = orc.eval_path(sc, 0, t, mu[:, 0], mu[:, 1], direct=True)
        for p in range(sc.su.shape[0]):
            tu, tv = float(sc.su[p]), float(sc.sv[p])
            d = np.hypot(uk - tu, vk - tv)
            if not np.any(d < 0.05):
                continue
            roots = []
            for s in np.argsort(d)[:6]:
                u, v = mu[s]
                for _ in range(30):
                    h = 1e-7
                    a = orc.eval_path(sc, 0, t, np.array([u, u + h, u]), np.array([v, v, v + h]), direct=True)
                    f = np.array([a[0][0] - tu, a[1][0] - tv])
                    J = np.array([[(a[0][1] - a[0][0]) / h, (a[0][2] - a[0][0]) / h],
                                  [(a[1][1] - a[1][0]) / h, (a[1][2] - a[1][0]) / h]])
                    step = np.linalg.solve(J, f)
                    u, v = u - step[0], v - step[1]
                    if np.max(np.abs(step)) < 1e-13:
                        break
                a = orc.eval_path(sc, 0, t, np.array([u]), np.array([v]), direct=True)
                if (u >= -1e-12 and v >= -1e-12 and u + v <= 1 + 1e-12 and a[3][0] > 0
                        and math.hypot(a[0][0] - tu, a[1][0] - tv) < 1e-9
                        and not any(abs(u - q[0]) + abs(v - q[1]) < 1e-7 for q in roots)):
                    roots.append((u, v, a[2][0]))
            E_ref[p] += sum(r[2] for r in roots)
    assert np.count_nonzero(E_ref) >= 5
    np.testing.assert_allclose(E_est, E_ref, rtol=1e-6, atol=1e-12)


def test_refraction_irradiance_encloses_and_converges(orc):
    """Refraction irradiance bound (sqrt(beta) kept as a symbol, 2W-scaled derivatives, M' = 4 beta M,
    remainder variables for sqrt(beta) and s^(-3/2)): every swept path's E lies in [E_lo, E_hi],
    and E_hi approaches the cell's maximum as the cells shrink."""
    sc = S.config("water", n=4, steep=0.05, lights=[(0.3, 0.2, 1.2)])
    excess = []
    for d in (0, 2, 3):
        rec = orc.bound(sc, depth=d)
        live = rec[((rec["flags"] & orc.LIVE) != 0) & np.isfinite(rec["e_hi"])]
        assert len(live) > 0.9 * np.count_nonzero(rec["flags"] & orc.LIVE)
        ex = []
        for r in live[:: max(1, len(live) // 40)]:
            u, v = cell_points(orc, r["cell"], d, 12)
            uk, vk, E, t = orc.eval_path(sc, int(r["emitter"]), int(r["tri0"]), u, v, direct=True)
            assert np.all(E <= r["e_hi"] * (1 + 1e-9)) and np.all(E >= r["e_lo"] * (1 - 1e-9))
            ex.append(r["e_hi"] / E.max() - 1.0)
        excess.append(np.median(ex))
    assert excess[0] > excess[1] > excess[2] >= 0.0
    assert excess[2] < 0.05 * excess[0]

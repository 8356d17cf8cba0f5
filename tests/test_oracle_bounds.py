"""Pins of the oracle's bound pass (Secs. 4.3-4.5) against closed forms,
dense sweeps of the direct geometry, and the subdivision property of Sec. 4.1.

Slack: the oracle runs in float64; where a bound is attained (at cell corners)
its own rounding puts the swept value above the bound by up to ~2e-12
relative (cancellation in the Jacobian numerator M), so containment checks
allow 1e-9 relative on irradiance and 1e-12 absolute on receiver coordinates.
"""
import numpy as np
import pytest

from paper_2504_19163_gb300 import scenes as S

E_SLACK = 1e-9
U_SLACK = 1e-12


def cell_points(orc, cell, depth, K):
    c = orc.cell_corners(int(cell), int(depth))
    mu = np.array([(i / K, j / K) for i in range(K + 1) for j in range(K + 1 - i)])
    m0 = 1 - mu[:, 0] - mu[:, 1]
    u = m0 * c[0, 0] + mu[:, 0] * c[1, 0] + mu[:, 1] * c[2, 0]
    v = m0 * c[0, 1] + mu[:, 0] * c[1, 1] + mu[:, 1] * c[2, 1]
    return u, v


def depth_of(rec):
    return (rec["flags"].astype(np.int64) >> 24) & 63


def sweep_violations(orc, scene, rec, K=10):
    """Count swept paths that land on the receiver region but fall outside a record's bound."""
    viol = 0
    hits = 0
    for r in rec:
        if r["flags"] & orc.SPLIT:
            continue
        u, v = cell_points(orc, r["cell"], depth_of(np.array([r]))[0], K)
        uk, vk, E, t = orc.eval_path(scene, int(r["emitter"]), int(r["tri0"]), u, v, direct=True)
        on = (uk >= 0) & (uk <= 1) & (vk >= 0) & (vk <= 1) & (t > 0)
        if not (r["flags"] & orc.LIVE):
            viol += int(on.sum())
            continue
        hits += int(on.sum())
        bad = on & ((uk < r["u_lo"] - U_SLACK) | (uk > r["u_hi"] + U_SLACK) | (vk < r["v_lo"] - U_SLACK)
                    | (vk > r["v_hi"] + U_SLACK) | (E > r["e_hi"] * (1 + E_SLACK)))
        viol += int(bad.sum())
    return viol, hits


def test_rational_form_equals_vector_reflection(orc):
    """Eqs. eq_rct / eq_refr_rational (un-normalized) agree with normalized vector reflection."""
    sc = S.config("mirror32")
    rng = np.random.default_rng(0)
    for t in rng.choice(sc.s1.n_tris, 20, replace=False):
        m = rng.dirichlet([1, 1, 1], size=50)
        a = orc.eval_path(sc, 0, int(t), m[:, 1], m[:, 2])
        b = orc.eval_path(sc, 0, int(t), m[:, 1], m[:, 2], direct=True)
        np.testing.assert_allclose(a[0], b[0], atol=1e-12)
        np.testing.assert_allclose(a[1], b[1], atol=1e-12)
        np.testing.assert_allclose(a[2], b[2], rtol=1e-9)


@pytest.mark.parametrize("h,c", [(2.0, 1.0), (1.5, 0.5)])
def test_flat_mirror_closed_form(orc, h, c):
    """Point light (0,0,h), mirror z=0, receiver z=c: hit = ((h+c)/h)(x,y) and
    E = I0 (h+c) / (X^2+Y^2+(h+c)^2)^(3/2) (image source).  The map is affine, so
    the Bernstein box equals the box of the three corner images exactly."""
    sc = S.config("flat", n=4, h=h, c=c, depth=2)
    rec = orc.bound(sc)
    assert np.all(rec["flags"] & orc.LIVE)
    for r in rec:
        u, v = cell_points(orc, r["cell"], 2, 1)  # corners only
        tri = int(r["tri0"])
        i0, i1, i2 = sc.s1.i0[tri], sc.s1.i1[tri], sc.s1.i2[tri]
        P = np.stack([sc.s1.px, sc.s1.py, sc.s1.pz], 1).astype(np.float64)
        x1 = P[i0] + np.outer(u, P[i1] - P[i0]) + np.outer(v, P[i2] - P[i0])
        X = (h + c) / h * x1[:, :2]
        uk = (X[:, 0] + 1.5) / 3.0
        vk = (X[:, 1] + 1.5) / 3.0
        assert r["u_lo"] == pytest.approx(np.clip(uk.min(), 0, 1), abs=1e-12)
        assert r["u_hi"] == pytest.approx(np.clip(uk.max(), 0, 1), abs=1e-12)
        assert r["v_lo"] == pytest.approx(np.clip(vk.min(), 0, 1), abs=1e-12)
        assert r["v_hi"] == pytest.approx(np.clip(vk.max(), 0, 1), abs=1e-12)
        # closed-form irradiance over a dense sweep of the cell
        u, v = cell_points(orc, r["cell"], 2, 12)
        x1 = P[i0] + np.outer(u, P[i1] - P[i0]) + np.outer(v, P[i2] - P[i0])
        X = (h + c) / h * x1[:, :2]
        Ecf = (h + c) / ((X ** 2).sum(1) + (h + c) ** 2) ** 1.5
        uk2, vk2, E2, _ = orc.eval_path(sc, 0, tri, u, v, direct=True)
        np.testing.assert_allclose(E2, Ecf, rtol=1e-10)
        np.testing.assert_allclose(uk2, (X[:, 0] + 1.5) / 3, atol=1e-12)
        assert Ecf.max() <= r["e_hi"] * (1 + E_SLACK)
        assert Ecf.min() >= r["e_lo"] * (1 - E_SLACK)


def _worst_ratio(orc, sc, d):
    rec = orc.bound(sc, depth=d)
    worst = 0.0
    for r in rec[:: max(1, len(rec) // 256)]:
        if not (r["flags"] & orc.LIVE) or not np.isfinite(r["e_hi"]):
            continue
        u, v = cell_points(orc, r["cell"], d, 8)
        _, _, E, _ = orc.eval_path(sc, int(r["emitter"]), int(r["tri0"]), u, v, direct=True)
        worst = max(worst, r["e_hi"] / E.max())
    return worst


def test_flat_mirror_irradiance_bound_exact_at_corners(orc):
    """Light above a mesh vertex of a flat mirror: on every cell the irradiance maximum sits at a
    corner, where the Bernstein bound is attained, so E_hi / max E = 1 at every depth."""
    for d in range(4):
        sc = S.config("flat", n=2, depth=d)
        assert _worst_ratio(orc, sc, d) == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("name", ["flat_offset", "tiny"])
def test_irradiance_bound_converges_quadratically(orc, name):
    """Sec. 4.1: Bernstein bounds converge quadratically in the cell size, so the excess
    E_hi / max E - 1 shrinks by about 4x per 4-way split (required: at least 2x)."""
    ex = []
    for d in range(5):
        if name == "flat_offset":
            sc = S.config("flat", n=2, depth=d)
            sc.emitters = S.point_emitters([(0.13, -0.07, 2.0)], 1.0)
        else:
            sc = S.config("tiny", n=4, depth=d)
        w = _worst_ratio(orc, sc, d)
        assert w >= 1 - 1e-9
        ex.append(w - 1)
    assert ex[0] > 1e-3
    assert all(ex[i + 1] < 0.5 * ex[i] for i in range(4))


def test_dense_sweep_containment_heightfield(orc):
    """No swept path on the receiver falls outside its cell's position and irradiance bound."""
    sc = S.config("mirror32")
    rec = orc.bound(sc)
    rng = np.random.default_rng(11)
    pick = rec[rng.choice(len(rec), 1500, replace=False)]
    viol, hits = sweep_violations(orc, sc, pick)
    assert hits > 50000
    assert viol == 0


@pytest.mark.parametrize("name", ["mirror256", "mirror256_rough"])
def test_dense_sweep_containment_noisy_area_light(orc, name):
    """Same on the 256^2 noisy mirrors (smooth and per-vertex noise) with face-averaged normals
    and 16 area-light samples."""
    sc = S.config(name)
    rng = np.random.default_rng(12)
    n_base = sc.emitters.n * sc.s1.n_tris * 4 ** sc.depth
    work = np.sort(rng.choice(n_base, 1500, replace=False))
    rec = orc.bound(sc, work=work)
    viol, hits = sweep_violations(orc, sc, rec, K=8)
    assert hits > 20000
    assert viol == 0


def test_position_bounds_nest_under_subdivision(orc):
    """For reflection positions the child's coefficient ratios are convex combinations of the
    parent's (de Casteljau weights are the same for P and Q), so child boxes lie in parent boxes."""
    sc = S.config("mirror32")
    p = orc.bound(sc, depth=1, irradiance=False)
    c = orc.bound(sc, depth=2, irradiance=False)
    pkey = {(int(r["emitter"]), int(r["tri0"]), int(r["cell"])): r for r in p if depth_of(np.array([r]))[0] == 1}
    checked = 0
    for r in c:
        if depth_of(np.array([r]))[0] != 2 or r["flags"] & orc.SPLIT:
            continue
        par = pkey.get((int(r["emitter"]), int(r["tri0"]), int(r["cell"]) >> 2))
        if par is None or par["flags"] & orc.SPLIT:
            continue
        if not (par["flags"] & orc.LIVE):
            assert not (r["flags"] & orc.LIVE)
            continue
        if r["flags"] & orc.LIVE:
            assert r["u_lo"] >= par["u_lo"] - 1e-12 and r["u_hi"] <= par["u_hi"] + 1e-12
            assert r["v_lo"] >= par["v_lo"] - 1e-12 and r["v_hi"] <= par["v_hi"] + 1e-12
            checked += 1
    assert checked > 5000


def test_irradiance_bounds_tighten_with_depth(orc):
    """With the remainder variable exact nesting is not guaranteed; the mean log(E_hi/E_lo) and the
    mean box area must still fall monotonically over depth 0..4 (Sec. 6.5, Fig. fig_par trend)."""
    sc = S.config("tiny", n=4)
    logr, area = [], []
    for d in range(5):
        rec = orc.bound(sc, depth=d)
        live = rec[((rec["flags"] & orc.LIVE) != 0) & np.isfinite(rec["e_hi"])]
        logr.append(np.mean(np.log(live["e_hi"] / live["e_lo"])))
        area.append(np.mean((live["u_hi"] - live["u_lo"]) * (live["v_hi"] - live["v_lo"])))
    assert all(logr[i + 1] < logr[i] for i in range(4))
    assert all(area[i + 1] < area[i] for i in range(4))


def test_receiver_behind_mirror_is_culled(orc):
    """Receiver below the mirror while reflected rays go up: every cell is forward-culled."""
    sc = S.config("mirror32", receiver_z=-1.0)
    rec = orc.bound(sc)
    assert not np.any(rec["flags"] & orc.LIVE)
    assert np.all((rec["flags"] & (orc.CULL_BEHIND | orc.SPLIT)) != 0)

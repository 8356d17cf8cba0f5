"""Pins of the oracle's index, Algorithm 1 and Newton solve (Secs. 5, 6.1) on tiny
meshes, against exhaustive enumeration of every tuple, closed forms, and the
statistical identities of Sec. 5.3 (expectation, variance bound Eq. eq_varbound_u)."""
import numpy as np
import pytest

from paper_2504_19163_gb300 import scenes as S

G = 512


def oracle_index(orc, sc):
    rec = orc.bound(sc)
    f = orc.records_to_f32(rec)
    off, key, et = orc.index(f["u_lo"], f["u_hi"], f["v_lo"], f["v_hi"], f["e_hi"], f["emitter"], f["tri0"],
                             f["tri1"], f["flags"], G)
    return rec, f, off, key, et


def point_cell(su, sv):
    gi = np.clip(np.floor(su.astype(np.float32) * np.float32(G)).astype(np.int64), 0, G - 1)
    gj = np.clip(np.floor(sv.astype(np.float32) * np.float32(G)).astype(np.int64), 0, G - 1)
    return gj * G + gi


def enumerate_all(orc, sc):
    """E(T) at every shading point for every tuple (P = 1 so contrib = E)."""
    n_p = sc.su.shape[0]
    keys = np.array([orc.tuple_key(e, t) for e in range(sc.emitters.n) for t in range(sc.s1.n_tris)], np.uint64)
    wp = np.repeat(np.arange(n_p), keys.shape[0])
    wk = np.tile(keys, n_p)
    contrib, ru, rv, st = orc.solve(sc, wp, wk, np.ones(wp.shape[0], np.float32))
    return wp, wk, contrib.reshape(n_p, -1), st.reshape(n_p, -1), keys


def test_index_matches_geometric_overlap(orc):
    """Every LIVE record's tuple is listed in exactly the grid cells its box touches (closed box
    against the half-open cell [i/G, (i+1)/G), last row/column closed), with the max bound."""
    sc = S.config("tiny", n=4, depth=2)
    rec, f, off, key, et = oracle_index(orc, sc)
    assert np.all(np.diff(off) >= 0)
    live = np.nonzero(f["flags"] & orc.LIVE)[0]
    expect = {}
    for r in live:
        k = int(orc.tuple_key(int(f["emitter"][r]), int(f["tri0"][r])))
        cols = [i for i in range(G) if f["u_lo"][r] < (i + 1) / G and f["u_hi"][r] >= i / G]
        rows = [j for j in range(G) if f["v_lo"][r] < (j + 1) / G and f["v_hi"][r] >= j / G]
        for j in rows:
            for i in cols:
                g = j * G + i
                expect[(g, k)] = max(expect.get((g, k), -1.0), float(f["e_hi"][r]))
    got = {}
    for g in np.nonzero(np.diff(off))[0]:
        ks = key[off[g]:off[g + 1]]
        assert np.all(np.diff(ks.astype(np.float64)) > 0)  # sorted, unique
        for k, e in zip(ks, et[off[g]:off[g + 1]]):
            got[(int(g), int(k))] = float(e)
    assert got.keys() == expect.keys()
    for k in got:
        assert got[k] == expect[k]


def test_flat_mirror_newton_root_closed_form(orc):
    """Flat mirror: the root for receiver point X is x1 = h/(h+c) X; E is the image-source law."""
    h, c = 2.0, 1.0
    sc = S.config("flat", n=4, h=h, c=c, points=8)
    wp, wk, E, st, keys = enumerate_all(orc, sc)
    P = np.stack([sc.s1.px, sc.s1.py, sc.s1.pz], 1).astype(np.float64)
    for p in range(sc.su.shape[0]):
        X = np.array([3.0 * float(sc.su[p]) - 1.5, 3.0 * float(sc.sv[p]) - 1.5])
        x1 = h / (h + c) * X
        hits = np.nonzero(st[p])[0]
        assert hits.size == 1
        t = hits[0]
        i0, i1, i2 = sc.s1.i0[t], sc.s1.i1[t], sc.s1.i2[t]
        _, ru, rv, _ = orc.solve(sc, np.array([p]), np.array([keys[t]]), np.ones(1, np.float32))
        xr = P[i0] + ru[0] * (P[i1] - P[i0]) + rv[0] * (P[i2] - P[i0])
        np.testing.assert_allclose(xr[:2], x1, atol=1e-12)
        Ecf = (h + c) / (X @ X + (h + c) ** 2) ** 1.5
        assert E[p, t] == pytest.approx(Ecf, rel=1e-10)


@pytest.fixture(scope="module")
def tiny_setup(orc):
    sc = S.config("tiny", n=4, depth=2, points=12, lights=[(0.1, -0.05, 2.0), (-0.3, 0.2, 1.8)])
    rec, f, off, key, et = oracle_index(orc, sc)
    wp, wk, E, st, keys = enumerate_all(orc, sc)
    return sc, off, key, et, E, st, keys


def test_every_root_is_listed_and_bounded(orc, tiny_setup):
    """Validity (Sec. 6.3): every tuple with a root at a shading point is in U(p), and its
    per-tuple bound covers the root's irradiance (E~/E >= 1)."""
    sc, off, key, et, E, st, keys = tiny_setup
    g = point_cell(sc.su, sc.sv)
    n_roots = 0
    for p in range(sc.su.shape[0]):
        lst = dict(zip(key[off[g[p]]:off[g[p] + 1]].tolist(), et[off[g[p]]:off[g[p] + 1]].tolist()))
        for t in np.nonzero(st[p])[0]:
            n_roots += 1
            k = int(keys[t])
            assert k in lst
            assert lst[k] >= E[p, t] * (1 - 1e-9)
    assert n_roots > 50


def test_estimator_is_unbiased_against_enumeration(orc, tiny_setup):
    """Sec. 5.3: E[<E>] = sum over U of E(T) = sum over all tuples (no root outside U); the mean of
    K independent estimates lies within the Chebyshev radius built from the bound mu2_bar of
    Eq. eq_varbound_u (failure probability 1e-3 per point)."""
    sc, off, key, et, E, st, keys = tiny_setup
    gamma = 4.0 / max(1e-30, float(np.median(et)))
    enum = E.sum(axis=1)
    K = 400
    acc = np.zeros(sc.su.shape[0])
    size_acc = np.zeros(sc.su.shape[0])
    for seed in range(K):
        wp, wk, wP, n_u = orc.sample(off, key, et, G, sc.su, sc.sv, gamma, seed)
        contrib, _, _, _ = orc.solve(sc, wp, wk, wP)
        acc += orc.accumulate(sc.su.shape[0], wp, contrib)
        size_acc += np.bincount(wp, minlength=sc.su.shape[0])
    mean = acc / K
    g = point_cell(sc.su, sc.sv)
    for p in range(sc.su.shape[0]):
        ets = et[off[g[p]]:off[g[p] + 1]].astype(np.float64)
        P = np.minimum(np.float64(np.float32(gamma)) * ets, 1.0)
        mu2 = float(np.sum(ets ** 2 / P)) if ets.size else 0.0
        radius = np.sqrt(mu2 / (K * 1e-3))
        assert abs(mean[p] - enum[p]) <= radius + 1e-12
        # expected number of selected tuples: sum of P (Sec. 5.4); variance <= sum P
        sp = float(P.sum())
        assert abs(size_acc[p] / K - sp) <= np.sqrt(max(sp, 1e-12) / (K * 1e-3)) + 1e-12
    # the Chebyshev radius is meaningful: estimates do vary and the mean is close overall
    assert np.sum(enum) > 0
    assert abs(mean.sum() - enum.sum()) / enum.sum() < 0.05


def test_variance_below_bound(orc, tiny_setup):
    """Eq. eq_varbound_u, read as a bound on the variance: with independent selections,
    Var<E> = sum E^2/P - sum E^2 <= sum over U of E~^2 / P (E <= E~).  Checked exactly and
    against the empirical variance of 300 seeded estimates."""
    sc, off, key, et, E, st, keys = tiny_setup
    gamma = 2.0 / max(1e-30, float(np.median(et)))
    g = point_cell(sc.su, sc.sv)
    kidx = {int(k): i for i, k in enumerate(keys)}
    K = 300
    est = np.zeros((K, sc.su.shape[0]))
    for seed in range(K):
        wp, wk, wP, _ = orc.sample(off, key, et, G, sc.su, sc.sv, gamma, 1000 + seed)
        contrib, _, _, _ = orc.solve(sc, wp, wk, wP)
        est[seed] = orc.accumulate(sc.su.shape[0], wp, contrib)
    for p in range(sc.su.shape[0]):
        ks = key[off[g[p]]:off[g[p] + 1]]
        ets = et[off[g[p]]:off[g[p] + 1]].astype(np.float64)
        P = np.minimum(np.float64(np.float32(gamma)) * ets, 1.0)
        Et = np.array([E[p, kidx[int(k)]] for k in ks])
        var = float(np.sum(Et ** 2 / P) - np.sum(Et ** 2)) if ks.size else 0.0
        bound = float(np.sum(ets ** 2 / P)) if ks.size else 0.0
        assert var <= bound * (1 + 1e-9) + 1e-30
        assert np.var(est[:, p]) <= 2.0 * bound + 1e-30


def test_selection_probability_positive_when_bound_positive(orc):
    """P = min(gamma E~, 1) rounded up in float32 stays > 0 for tiny positive E~ (unbiasedness)."""
    off = np.array([0] * (G * G) + [3], np.int64)
    off[1:] = 3
    key = np.array([1, 2, 3], np.uint64)
    et = np.array([1e-38, 1e-30, np.inf], np.float32)
    su = np.array([0.0], np.float32)
    sv = np.array([0.0], np.float32)
    wp, wk, wP, n_u = orc.sample(off, key, et, G, su, sv, 1e-6, 0)
    assert n_u == 3
    assert 3 in wk.tolist()  # E~ = inf -> P = 1, always selected
    assert np.all(wP > 0)


@pytest.mark.parametrize("name,kw", [("tiny", dict(n=6, depth=1, points=24)),
                                     ("water", dict(n=6, depth=1, steep=0.08, points=24))])
def test_one_polish_step_is_enough(orc, name, kw):
    """Sec. 6.1 Newton: after the damped float32-level phase leaves a root within ~1e-6, one
    quadratically convergent float64 step reaches the float64 limit.  Every (point, tuple) pair
    solved with 1 and with 2 float64 polish steps: the same roots accepted, contributions within
    1e-12 relative, roots within 1e-12 in barycentric coordinates (the oracle's polish count)."""
    sc = S.config(name, **kw)
    n_p = sc.su.shape[0]
    keys = np.array([orc.tuple_key(e, t) for e in range(sc.emitters.n) for t in range(sc.s1.n_tris)], np.uint64)
    wp = np.repeat(np.arange(n_p), keys.shape[0])
    wk = np.tile(keys, n_p)
    ones = np.ones(wp.shape[0], np.float32)
    c1, u1, v1, s1 = orc.solve(sc, wp, wk, ones, polish_iters=1)
    c2, u2, v2, s2 = orc.solve(sc, wp, wk, ones, polish_iters=2)
    acc1, acc2 = c1 > 0, c2 > 0
    assert acc1.sum() > 20
    assert np.array_equal(acc1, acc2)
    assert np.max(np.abs(c1[acc1] - c2[acc1]) / c2[acc1]) <= 1e-12
    assert np.max(np.abs(u1[acc1] - u2[acc1])) <= 1e-12 and np.max(np.abs(v1[acc1] - v2[acc1])) <= 1e-12

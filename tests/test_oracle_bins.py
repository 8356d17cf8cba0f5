"""Bin-packed selection (Sec. 5.3: the listed tuples are packed into groups whose probabilities sum
to at most 1, and one tuple is importance-sampled per group) in the oracle:

* every tuple is selected with probability P (the frequencies over many independently drawn points
  sharing one list agree with P within 5 binomial standard deviations), never two of one group;
* the number of groups satisfies the greedy packing's guarantee |B| <= 2 ceil(sum P) + 1 and
  |B| >= ceil(sum P);
* the estimator stays unbiased (mean of seeded estimates within the Chebyshev radius of the
  enumerated sum) and its variance stays below the bound of Eq. eq_varbound_u.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from test_oracle_estimator import G, point_cell, tiny_setup  # noqa: F401  (fixture)


@pytest.fixture(scope="module")
def orc():
    O.build()
    return O


def one_list(et):
    """An index whose every grid cell is empty except cell 0, holding keys 1..n with bounds et."""
    n = len(et)
    off = np.zeros(G * G + 1, np.int64)
    off[1:] = n
    return off, np.arange(1, n + 1, dtype=np.uint64), np.asarray(et, np.float32)


def test_each_tuple_selected_with_its_probability(orc):
    rng = np.random.default_rng(3)
    et = rng.uniform(0.02, 0.45, 24).astype(np.float32)
    off, key, et = one_list(et)
    n_pts = 40000
    su = np.zeros(n_pts, np.float32)
    sv = np.zeros(n_pts, np.float32)
    wp, wk, wP, n_u, n_b = orc.sample(off, key, et, G, su, sv, 1.0, 11, bins=True, with_bins=True)
    assert n_u == 24 * n_pts
    P = np.minimum(et.astype(np.float64), 1.0)
    freq = np.bincount(wk.astype(np.int64), minlength=25)[1:] / n_pts
    sd = np.sqrt(P * (1 - P) / n_pts)
    assert np.all(np.abs(freq - P) <= 5 * sd + 1e-6), np.max(np.abs(freq - P) / sd)
    # groups: every point packs the same list, so |B| per point is fixed; the greedy guarantee
    b = n_b // n_pts
    assert n_b == b * n_pts
    s = float(P.sum())
    assert math.ceil(s - 1e-6) <= b <= 2 * math.ceil(s) + 1
    # at most one selection per group and point: count per point never exceeds the group count,
    # and the expected count is sum P
    cnt = np.bincount(wp, minlength=n_pts)
    assert cnt.max() <= b
    assert abs(cnt.mean() - s) <= 5 * math.sqrt(s / n_pts)


def test_groups_select_mutually_exclusively(orc):
    """Three tuples of P = 0.3 share one group (sum 0.9): a point selects at most one of them, each
    with probability 0.3, none with 0.1."""
    off, key, et = one_list([0.3, 0.3, 0.3])
    n_pts = 30000
    z = np.zeros(n_pts, np.float32)
    wp, wk, wP, n_u, n_b = orc.sample(off, key, et, G, z, z, 1.0, 5, bins=True, with_bins=True)
    assert n_b == n_pts
    cnt = np.bincount(wp, minlength=n_pts)
    assert cnt.max() == 1
    assert abs(np.mean(cnt == 0) - 0.1) < 5 * math.sqrt(0.09 / n_pts) + 1e-6
    # without bins the three draws are independent: two or three selections happen
    wp2, _, _, _ = orc.sample(off, key, et, G, z, z, 1.0, 5)
    assert np.bincount(wp2, minlength=n_pts).max() >= 2


def test_binned_estimator_is_unbiased_with_bounded_variance(orc, tiny_setup):
    sc, off, key, et, E, st, keys = tiny_setup
    gamma = 4.0 / max(1e-30, float(np.median(et)))
    enum = E.sum(axis=1)
    K = 400
    est = np.zeros((K, sc.su.shape[0]))
    for seed in range(K):
        wp, wk, wP, _ = orc.sample(off, key, et, G, sc.su, sc.sv, gamma, seed, bins=True)
        contrib, _, _, _ = orc.solve(sc, wp, wk, wP)
        est[seed] = orc.accumulate(sc.su.shape[0], wp, contrib)
    mean = est.mean(axis=0)
    g = point_cell(sc.su, sc.sv)
    for p in range(sc.su.shape[0]):
        ets = et[off[g[p]]:off[g[p] + 1]].astype(np.float64)
        P = np.minimum(np.float64(np.float32(gamma)) * ets, 1.0)
        mu2 = float(np.sum(ets ** 2 / P)) if ets.size else 0.0
        assert abs(mean[p] - enum[p]) <= np.sqrt(mu2 / (K * 1e-3)) + 1e-12
        # groups remove the positive cross terms of independent selection: Var <= sum E~^2/P
        assert np.var(est[:, p]) <= 2.0 * mu2 + 1e-30
    assert abs(mean.sum() - enum.sum()) / enum.sum() < 0.05

"""Stochastic Newton starts with the reciprocal weighting (Sec. 6.1 "Stoc", after Zeltner et al.
2020) in the oracle:

* on a flat mirror every start reaches the tuple's single root, so every weight N is 1 and the
  contribution equals the deterministic start's;
* on a curved heightfield the mean of the weighted contributions over independent seeds equals the
  sum of E over every root of the tuple (found by Newton from a dense grid of starts) within five
  standard errors, including tuples whose root the centroid start (Det) misses or where it finds
  one of several roots.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19163_gb300 import scenes as S


def all_pairs(sc):
    keys = np.array([O.tuple_key(e, t) for e in range(sc.emitters.n) for t in range(sc.s1.n_tris)], np.uint64)
    n_p = sc.su.shape[0]
    return np.repeat(np.arange(n_p), keys.shape[0]), np.tile(keys, n_p)


def test_flat_mirror_weights_are_one():
    sc = S.config("flat", n=2, points=12)
    wp, wk = all_pairs(sc)
    ones = np.ones(wp.shape[0], np.float32)
    det, _, _, st_d = O.solve(sc, wp, wk, ones)
    sto, _, _, st_s, tr = O.solve(sc, wp, wk, ones, stoc_trials=64, seed=5, with_trials=True)
    assert st_d.sum() > 50
    assert np.array_equal(st_d, st_s)
    assert np.all(tr[st_s == 1] == 1)
    np.testing.assert_allclose(sto, det, rtol=1e-10, atol=0)


def test_stochastic_weighting_is_unbiased_against_root_enumeration():
    """Newton is cut to one damped step (+ the polish step), so only starts near a root converge
    within tolerance: the probability p of reaching a root is well below 1, the centroid start
    misses many roots, and the weight N (geometric, mean 1/p) is exercised.  The weighted mean still
    equals the sum over every root (exact E from fully converged multi-start Newton), within five
    standard errors plus the 1e-4 accuracy of a one-step root's E."""
    sc = S.config("tiny", n=3, points=10, lights=[(0.3, -0.2, 1.2)])
    wp, wk = all_pairs(sc)
    exact = np.zeros(wp.shape[0])
    n_roots = np.zeros(wp.shape[0], np.int64)
    for i in range(wp.shape[0]):
        t = int(wk[i] & np.uint64(0xFFFFFF))
        exact[i], n_roots[i] = O.roots(sc, 0, t, float(sc.su[wp[i]]), float(sc.sv[wp[i]]), n=20)
    has = n_roots > 0
    assert has.sum() > 20
    sel = np.nonzero(has)[0]
    ones = np.ones(sel.shape[0], np.float32)
    det, _, _, st_d = O.solve(sc, wp[sel], wk[sel], ones, newton_iters=1)
    assert st_d.sum() < 0.8 * sel.shape[0]  # the centroid start misses roots
    K = 300
    est = np.zeros((K, sel.shape[0]))
    n_w = []
    for k in range(K):
        c, _, _, st, tr = O.solve(sc, wp[sel], wk[sel], ones, newton_iters=1, stoc_trials=4096, seed=1000 + k,
                                  with_trials=True)
        est[k] = c
        n_w.append(tr[st == 1])
    n_w = np.concatenate(n_w)
    assert n_w.mean() > 1.5 and n_w.max() < 4096  # weights vary, the cap is never reached
    mean = est.mean(axis=0)
    se = est.std(axis=0) / np.sqrt(K)
    err = np.abs(mean - exact[sel])
    assert np.all(err <= 5 * se + 1e-4 * exact[sel]), np.max(err / (5 * se + 1e-4 * exact[sel]))
    # the deterministic start's estimate is biased low here
    assert det.sum() < 0.8 * exact[sel].sum()

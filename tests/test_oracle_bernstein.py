"""Pins of the oracle's Bernstein algebra (Sec. 4.1) against the paper's worked
example and against evaluations that do not go through the coefficient formulas
under test (de Casteljau, finite differences, products of factor values)."""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def de_casteljau(n, coeffs, mu):
    """Evaluate a classical Bernstein form on the 2-simplex by repeated convex combination."""
    from oracle import bb_index
    idx = {g: c for g, c in zip(bb_index(n), coeffs)}
    for d in range(n, 0, -1):
        nxt = {}
        for g0 in range(d):
            for g1 in range(d - g0):
                g2 = d - 1 - g0 - g1
                nxt[(g0, g1, g2)] = (mu[0] * idx[(g0 + 1, g1, g2)] + mu[1] * idx[(g0, g1 + 1, g2)]
                                     + mu[2] * idx[(g0, g1, g2 + 1)])
        idx = nxt
    return idx[(0, 0, 0)]


def rand_mu(rng, k):
    m = rng.dirichlet([1.0, 1.0, 1.0], size=k)
    return m


def test_worked_example(orc):
    """Sec. 4.1 footnote: x(4-x) on [0,1] -> coefficients 0, 2, 3, bound [0, 3]."""
    g = json.load(open(os.path.join(GOLD, "worked_example_bbound.json")))
    prod = orc.bb_mul(1, 1, g["factor_g"]["coefficients"], 1, g["factor_h"]["coefficients"])
    np.testing.assert_array_equal(prod, g["product_coefficients"])
    assert [prod.min(), prod.max()] == g["bernstein_bound"]
    # the bound really contains the function, and the function reaches 3 at x = 1
    xs = np.linspace(0, 1, 101)
    f = xs * (4 - xs)
    assert f.min() >= prod.min() and f.max() <= prod.max()
    assert orc.bb_eval(1, 2, prod, 1.0) == pytest.approx(3.0)


def test_product_matches_pointwise_product(orc):
    rng = np.random.default_rng(1)
    for m, n in [(1, 1), (2, 3), (3, 4), (4, 5), (9, 2)]:
        p = rng.normal(size=orc.lib().orc_bb_size(2, m))
        q = rng.normal(size=orc.lib().orc_bb_size(2, n))
        r = orc.bb_mul(2, m, p, n, q)
        for mu in rand_mu(rng, 20):
            lhs = de_casteljau(m + n, r, mu)
            rhs = de_casteljau(m, p, mu) * de_casteljau(n, q, mu)
            assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


def test_direct_evaluation_matches_de_casteljau(orc):
    rng = np.random.default_rng(2)
    for n in [1, 2, 5, 11]:
        p = rng.normal(size=orc.lib().orc_bb_size(2, n))
        for mu in rand_mu(rng, 10):
            assert orc.bb_eval(2, n, p, mu[1], mu[2]) == pytest.approx(de_casteljau(n, p, mu), rel=1e-12, abs=1e-12)


def test_corner_coefficients_are_values_and_unity(orc):
    rng = np.random.default_rng(3)
    n = 6
    p = rng.normal(size=orc.lib().orc_bb_size(2, n))
    idx = orc.bb_index(n)
    for corner, mu in [((n, 0, 0), (0.0, 0.0)), ((0, n, 0), (1.0, 0.0)), ((0, 0, n), (0.0, 1.0))]:
        assert orc.bb_eval(2, n, p, *mu) == pytest.approx(p[idx.index(corner)], rel=1e-13)
    one = np.ones(orc.lib().orc_bb_size(2, n))
    for mu in rand_mu(rng, 5):
        assert orc.bb_eval(2, n, one, mu[1], mu[2]) == pytest.approx(1.0, rel=1e-13)


def test_elevation_preserves_values(orc):
    rng = np.random.default_rng(4)
    for n in [1, 3, 8]:
        p = rng.normal(size=orc.lib().orc_bb_size(2, n))
        e = orc.bb_elevate(2, n, p)
        for mu in rand_mu(rng, 10):
            assert de_casteljau(n + 1, e, mu) == pytest.approx(de_casteljau(n, p, mu), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("j", [1, 2])
def test_derivative_matches_finite_difference(orc, j):
    rng = np.random.default_rng(5 + j)
    n = 5
    p = rng.normal(size=orc.lib().orc_bb_size(2, n))
    d = orc.bb_deriv(n, p, j)
    h = 1e-6
    for mu in rand_mu(rng, 10) * 0.8 + 0.2 / 3:
        step = np.zeros(3)
        step[j] = h
        step[0] = -h  # move along mu_j while staying on the simplex
        fd = (de_casteljau(n, p, mu + step) - de_casteljau(n, p, mu - step)) / (2 * h)
        assert de_casteljau(n - 1, d, mu) == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_ratio_bound_contains_rational_function(orc):
    """Eq. eq_bbound: with b(q) of one sign, min/max of b(p)/b(q) bound p/q."""
    rng = np.random.default_rng(9)
    n = 4
    for _ in range(20):
        p = rng.normal(size=orc.lib().orc_bb_size(2, n))
        q = rng.uniform(0.2, 2.0, size=orc.lib().orc_bb_size(2, n))
        r = p / q
        for mu in rand_mu(rng, 50):
            f = de_casteljau(n, p, mu) / de_casteljau(n, q, mu)
            assert r.min() - 1e-12 <= f <= r.max() + 1e-12


def test_chord_remainder_brackets_error(orc):
    """Remainder variable for s^(-3/2): f - r lies in [dlo, dhi] on the whole interval."""
    f = lambda s: s ** -1.5
    for lo, hi in [(4.0, 4.4), (0.5, 3.0), (1.0, 1.0 + 1e-6), (2.0, 2.0)]:
        a, b, dlo, dhi = orc.chord_inv32(lo, hi)
        s = np.linspace(lo, hi, 20001)
        err = f(s) - (a * s + b)
        assert err.min() >= dlo - 1e-12 * f(lo)
        assert err.max() <= dhi + 1e-12 * f(lo)
        if lo == hi:
            assert a == 0.0 and dlo == 0.0 and dhi == 0.0
        else:
            # the chord is exact at both ends and the minimum is reached inside
            assert abs(err[0]) < 1e-12 and abs(err[-1]) < 1e-12
            assert err.min() == pytest.approx(dlo, rel=1e-6, abs=1e-15)


def test_cell_corners_partition(orc):
    """4-way midpoint split: children tile the parent, areas quarter, ids are base-4 paths."""
    for depth in [1, 2, 3]:
        tot = 0.0
        for cid in range(4 ** depth):
            c = orc.cell_corners(cid, depth)
            a, b = c[1] - c[0], c[2] - c[0]
            area = abs(a[0] * b[1] - a[1] * b[0]) / 2
            assert area == pytest.approx(0.5 / 4 ** depth, rel=1e-15)
            tot += area
        assert tot == pytest.approx(0.5)
    # child k of cell c at depth d is cell 4c+k at depth d+1 and lies inside it
    c = orc.cell_corners(3, 1)
    for k in range(4):
        ch = orc.cell_corners(4 * 3 + k, 2)
        for pt in ch:
            lam = np.linalg.solve(np.array([c[1] - c[0], c[2] - c[0]]).T, pt - c[0])
            assert lam.min() >= -1e-15 and lam.sum() <= 1 + 1e-15

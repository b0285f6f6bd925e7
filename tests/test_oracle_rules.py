"""Pins of the oracle's quadrature rules against exact integrals (rule exactness).

Gauss-Legendre, the Radon rule and the Duffy rule are checked on monomials they
must integrate exactly; the Sauter-Schwab subdomain rules are checked on all
monomials x1^a x2^b y1^c y2^d with a+b+c+d <= 6 over D x D, whose exact value
is the product of the two triangle moments 1/((b+1)(a+b+2)) * 1/((d+1)(c+d+2)).
A missing or overlapping subdomain, or a wrong Jacobian, fails these.
"""
import itertools
import math

import numpy as np
import pytest


def tri_moment(a, b):
    """int over D = {0 <= t <= s <= 1} of s^a t^b."""
    return 1.0 / ((b + 1) * (a + b + 2))


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 8, 12, 20])
def test_gauss_legendre_exactness(oracle_mod, q):
    x, w = oracle_mod.gauss_legendre01(q)
    assert np.all(np.diff(x) > 0) and np.all((x > 0) & (x < 1))
    for k in range(2 * q):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 2e-15
    # degree 2q carries the textbook Gauss error (q!)^4 / ((2q+1) ((2q)!)^2) on [0,1]
    if q <= 8:
        err = 1.0 / (2 * q + 1) - np.sum(w * x ** (2 * q))
        exact = math.factorial(q) ** 4 / ((2 * q + 1) * math.factorial(2 * q) ** 2)
        assert abs(err - exact) < 1e-14 + 1e-9 * exact


@pytest.mark.parametrize("q", [3, 7, 15])
def test_gauss_legendre_matches_library(oracle_mod, q):
    x, w = oracle_mod.gauss_legendre01(q)
    z, wz = np.polynomial.legendre.leggauss(q)
    assert np.allclose(x, np.sort((z + 1) / 2), atol=1e-15, rtol=0)
    assert np.allclose(w, wz[np.argsort(z)] / 2, atol=1e-15, rtol=0)


def test_radon7_degree5(oracle_mod):
    s, t, w = oracle_mod.radon7()
    assert np.all(t >= 0) and np.all(t <= s) and np.all(s <= 1)
    for a in range(6):
        for b in range(6 - a):
            assert abs(np.sum(w * s ** a * t ** b) - tri_moment(a, b)) < 1e-15
    errs = [abs(np.sum(w * s ** a * t ** (6 - a)) - tri_moment(a, 6 - a)) for a in range(7)]
    assert max(errs) > 1e-8  # degree 6 is not exact


@pytest.mark.parametrize("q", [2, 3, 4])
def test_duffy_rule_exactness(oracle_mod, q):
    x1, x2, y1, y2, w = oracle_mod.rule_points("regular", q, "duffy")
    assert len(w) == q ** 4
    for a, b, c, d in itertools.product(range(4), repeat=4):
        # Duffy: s^a t^b -> xi1^(a+b+1) xi2^b, exact while a+b+1 <= 2q-1
        if a + b + 1 > 2 * q - 1 or c + d + 1 > 2 * q - 1:
            continue
        got = np.sum(w * x1 ** a * x2 ** b * y1 ** c * y2 ** d)
        assert abs(got - tri_moment(a, b) * tri_moment(c, d)) < 1e-15


def test_tri7_tensor_rule(oracle_mod):
    x1, x2, y1, y2, w = oracle_mod.rule_points("regular", 1, "tri7")
    assert len(w) == 49
    for a, b, c, d in itertools.product(range(4), repeat=4):
        if a + b > 5 or c + d > 5:
            continue
        got = np.sum(w * x1 ** a * x2 ** b * y1 ** c * y2 ** d)
        assert abs(got - tri_moment(a, b) * tri_moment(c, d)) < 1e-15


@pytest.mark.parametrize("case,nsub", [("vertex", 2), ("edge", 4), ("identical", 6)])
def test_sauter_schwab_moment_exactness(oracle_mod, case, nsub):
    q = 8
    x1, x2, y1, y2, w = oracle_mod.rule_points(case, q)
    assert len(w) == nsub * q ** 4
    eps = 1e-14
    for (s, t) in ((x1, x2), (y1, y2)):
        assert np.all(t >= -eps) and np.all(t <= s + eps) and np.all(s <= 1 + eps)
    assert np.all(w > 0)
    assert abs(np.sum(w) - 0.25) < 1e-15
    worst = 0.0
    for a, b, c, d in itertools.product(range(7), repeat=4):
        if a + b + c + d > 6:
            continue
        exact = tri_moment(a, b) * tri_moment(c, d)
        got = np.sum(w * x1 ** a * x2 ** b * y1 ** c * y2 ** d)
        worst = max(worst, abs(got - exact) / exact)
    assert worst < 1e-13


@pytest.mark.parametrize("case", ["vertex", "edge", "identical"])
def test_sauter_schwab_singular_set_is_collapsed(oracle_mod, case):
    """The weight of every point is bounded by a constant times |x - y|^2 in
    reference coordinates near the singular set (Jacobian cancels 1/r):
    check that w / |x - y| stays bounded as the points approach it."""
    x1, x2, y1, y2, w = oracle_mod.rule_points(case, 10)
    # physical |x-y| on the reference geometry of the case is comparable to the
    # distance to the singular set; use the reference distance for the check
    if case == "identical":
        dist = np.hypot(x1 - y1, x2 - y2)
    elif case == "edge":
        dist = np.sqrt((x1 - y1) ** 2 + x2 ** 2 + y2 ** 2)
    else:
        dist = np.sqrt(x1 ** 2 + x2 ** 2 + y1 ** 2 + y2 ** 2)
    ratio = w / dist
    assert np.isfinite(ratio).all() and ratio.max() < 1.0


def test_classification(oracle_mod):
    c = oracle_mod.classify
    assert c([0, 1, 2], [0, 1, 2]) == "identical"
    assert c([0, 1, 2], [2, 0, 1]) == "identical"
    assert c([0, 1, 2], [1, 0, 3]) == "edge"
    assert c([0, 1, 2], [5, 2, 1]) == "edge"
    assert c([0, 1, 2], [2, 7, 8]) == "vertex"
    assert c([0, 1, 2], [3, 4, 5]) == "regular"

"""The library's own rule generator (exported by bem_rule_points; no GPU
needed): moment exactness of every case on D x D, the analytic difference
columns, and agreement with the oracle's independently written rules (the
same derivation written twice must give the same points)."""
import itertools

import numpy as np
import pytest

import paper_1510_07244_gb300 as pkg
from paper_1510_07244_gb300 import build as libbuild


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    pkg.load()


def tri_moment(a, b):
    return 1.0 / ((b + 1) * (a + b + 2))


@pytest.mark.parametrize("case,nsub", [("vertex", 2), ("edge", 4), ("identical", 6)])
def test_library_rule_moments(case, nsub):
    r = pkg.bem_rule_points(case, 8)
    assert len(r["w"]) == nsub * 8 ** 4
    worst = 0.0
    for a, b, c, d in itertools.product(range(7), repeat=4):
        if a + b + c + d > 6:
            continue
        exact = tri_moment(a, b) * tri_moment(c, d)
        got = np.sum(r["w"] * r["x1"] ** a * r["x2"] ** b * r["y1"] ** c * r["y2"] ** d)
        worst = max(worst, abs(got - exact) / exact)
    assert worst < 1e-13


@pytest.mark.parametrize("case", ["vertex", "edge", "identical", "regular"])
def test_library_rule_differences(case):
    r = pkg.bem_rule_points(case, 5)
    assert np.allclose(r["d1"], r["x1"] - r["y1"], rtol=0, atol=4e-16)
    assert np.allclose(r["d2"], r["x2"] - r["y2"], rtol=0, atol=4e-16)


@pytest.mark.parametrize("case,q,rule", [("vertex", 5, "duffy"), ("edge", 4, "duffy"),
                                         ("identical", 5, "duffy"), ("regular", 3, "duffy"),
                                         ("regular", 1, "tri7")])
def test_library_rules_match_oracle(oracle_mod, case, q, rule):
    lib = pkg.bem_rule_points(case, q, rule)
    A = np.stack([lib[k] for k in ("x1", "x2", "y1", "y2", "w")], axis=1)
    B = np.stack(oracle_mod.rule_points(case, q, rule), axis=1)
    # the same point set (the two generators may list points in another order)
    A = A[np.lexsort(np.round(A[:, :4], 12).T[::-1])]
    B = B[np.lexsort(np.round(B[:, :4], 12).T[::-1])]
    assert A.shape == B.shape
    assert np.allclose(A, B, rtol=1e-13, atol=1e-16)


def test_library_rule_rejects_bad_orders():
    with pytest.raises(pkg.BemError):
        pkg.bem_rule_points("edge", 0)


@pytest.mark.parametrize("q", [1, 5, 10])
def test_library_high_order_regular_rule(q):
    """Duffy orders beyond the block engine's product-rule limit (used by pivot
    entries and by the order model's reference values)."""
    r = pkg.bem_rule_points("regular", q)
    assert len(r["w"]) == q ** 4
    for a, b, c, d in itertools.product(range(4), repeat=4):
        if a + b + 1 > 2 * q - 1 or c + d + 1 > 2 * q - 1:
            continue
        got = np.sum(r["w"] * r["x1"] ** a * r["x2"] ** b * r["y1"] ** c * r["y2"] ** d)
        assert abs(got - tri_moment(a, b) * tri_moment(c, d)) < 1e-14

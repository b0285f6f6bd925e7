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


# ---- touching rules with xi integrated out ---------------------------------
def _canonical_pair(case, rng):
    """Flat triangles in the canonical vertex orders of a touching case: the
    shared vertices come first (common vertex: v0; common edge: v0 -> v1)."""
    p0 = rng.standard_normal(3)
    a = [p0, p0 + rng.standard_normal(3), p0 + rng.standard_normal(3)]
    if case == "identical":
        b = list(a)
    elif case == "edge":
        b = [a[0], a[1], p0 + rng.standard_normal(3)]
    else:
        b = [p0, p0 + rng.standard_normal(3), p0 + rng.standard_normal(3)]
    return a, b


def _moments(r, case, a, b, kernel):
    """Sum over the rule of w k(x - y) (1, x1, x2)_i (1, y1, y2)_j (3 x 3)."""
    e1a, e2a = a[1] - a[0], a[2] - a[1]
    e1b, e2b = b[1] - b[0], b[2] - b[1]
    if case == "identical":
        d = np.outer(r["d1"], e1a) + np.outer(r["d2"], e2a)
    elif case == "edge":
        d = np.outer(r["d1"], e1a) + np.outer(r["x2"], e2a) - np.outer(r["y2"], e2b)
    else:
        d = (np.outer(r["x1"], e1a) + np.outer(r["x2"], e2a) - np.outer(r["y1"], e1b)
             - np.outer(r["y2"], e2b))
    rr = np.linalg.norm(d, axis=1)
    nb = np.cross(e1b, e2b)
    nb /= np.linalg.norm(nb)
    f = 1.0 / rr if kernel == "slp" else (d @ nb) / rr ** 3
    mx = np.stack([np.ones_like(rr), r["x1"], r["x2"]])
    my = np.stack([np.ones_like(rr), r["y1"], r["y2"]])
    return np.einsum("p,ip,jp->ij", r["w"] * f, mx, my)


@pytest.mark.parametrize("case,nsub", [("vertex", 2), ("edge", 4), ("identical", 6)])
@pytest.mark.parametrize("q", [3, 5])
def test_xi_integrated_rule_equals_full_rule(case, nsub, q):
    """For the Laplace kernels the q^4 rule's sum equals 1/(n+1) times the sum
    over the q^3 points at xi = 1, moment by moment (n = 2 single layer, 1
    double layer, plus one per coordinate factor): the Sauter-Schwab maps
    scale every coordinate by xi and the Gauss rule in xi is exact for these
    degrees.  Brute force on random flat pairs of every touching case."""
    full = pkg.bem_rule_points(case, q)
    xi = pkg.bem_rule_points_xi(case, q)
    assert len(xi["w"]) == nsub * q ** 3
    rng = np.random.default_rng(7 + q)
    for _ in range(3):
        a, b = _canonical_pair(case, rng)
        for kernel, base in (("slp", 2), ("dlp", 1)):
            if kernel == "dlp" and case == "identical":
                continue      # the double layer of a flat identical pair vanishes
            m4 = _moments(full, case, a, b, kernel)
            m3 = _moments(xi, case, a, b, kernel)
            fac = np.array([[1.0 / (base + (i > 0) + (j > 0) + 1) for j in range(3)]
                            for i in range(3)])
            assert np.abs(m4 - fac * m3).max() <= 1e-12 * np.abs(m4).max(), (kernel, m4, fac * m3)


def test_xi_integration_needs_an_exact_xi_rule():
    """With q = 2 the Gauss rule in xi integrates degree 3 but not 4: the
    piecewise-linear single layer's (x, y) moments (degree 4) differ, so the
    library keeps the q^4 rule there (its own selection asks 2q - 1 >= n)."""
    rng = np.random.default_rng(3)
    a, b = _canonical_pair("vertex", rng)
    m4 = _moments(pkg.bem_rule_points("vertex", 2), "vertex", a, b, "slp")
    m3 = _moments(pkg.bem_rule_points_xi("vertex", 2), "vertex", a, b, "slp")
    assert abs(m4[0, 0] - m3[0, 0] / 3) <= 1e-13 * abs(m4[0, 0])     # degree 2: exact
    assert abs(m4[1, 1] - m3[1, 1] / 5) > 1e-6 * abs(m4[1, 1])       # degree 4: not


@pytest.mark.parametrize("case", ["vertex", "edge", "identical"])
@pytest.mark.parametrize("q", [4, 5])
def test_helmholtz_xi_sum_in_node_pairs(case, q):
    """The float Helmholtz touching kernel keeps the q^4 rule's sum but takes
    it as, per point of the xi-integrated rule, the Gauss sum over xi of
    w_k xi_k^(2+m) exp(i kappa xi_k |u|) / |u|, written with the node pairs
    xi = 1/2 -+ t (symmetric nodes and weights): exp(i th/2) (c_mid + sum_j
    (w_j (a^p + b^p) cos(th t_j) + i w_j (a^p - b^p) sin(th t_j))).  Brute
    force against the q^4 rule, every moment, kappa = 9."""
    kappa = 9.0
    rng = np.random.default_rng(11 + q)
    a, b = _canonical_pair(case, rng)
    full = pkg.bem_rule_points(case, q)
    xi = pkg.bem_rule_points_xi(case, q)

    def dvec(r):
        e1a, e2a, e1b, e2b = a[1] - a[0], a[2] - a[1], b[1] - b[0], b[2] - b[1]
        if case == "identical":
            return np.outer(r["d1"], e1a) + np.outer(r["d2"], e2a)
        if case == "edge":
            return np.outer(r["d1"], e1a) + np.outer(r["x2"], e2a) - np.outer(r["y2"], e2b)
        return (np.outer(r["x1"], e1a) + np.outer(r["x2"], e2a) - np.outer(r["y1"], e1b)
                - np.outer(r["y2"], e2b))

    def mom(r):
        mx = np.stack([np.ones(len(r["w"])), r["x1"], r["x2"]])
        my = np.stack([np.ones(len(r["w"])), r["y1"], r["y2"]])
        return mx, my

    rr = np.linalg.norm(dvec(full), axis=1)
    mx, my = mom(full)
    m4 = np.einsum("p,ip,jp->ij", full["w"] * np.exp(1j * kappa * rr) / rr, mx, my)
    g, gw = np.polynomial.legendre.leggauss(q)
    g, gw = (g + 1) / 2, gw / 2
    u = np.linalg.norm(dvec(xi), axis=1)
    th = kappa * u
    S = []
    for p in range(2, 5):
        s = np.full(len(u), gw[q // 2] * 0.5 ** p if q % 2 else 0.0, complex)
        for k in range(q // 2):
            hi, lo, w = g[q - 1 - k], g[k], 0.5 * (gw[k] + gw[q - 1 - k])
            t = hi - 0.5
            s += w * (hi ** p + lo ** p) * np.cos(th * t) + 1j * w * (hi ** p - lo ** p) * np.sin(th * t)
        S.append(np.exp(0.5j * th) * s)
    mx3, my3 = mom(xi)
    m3 = np.array([[np.sum(xi["w"] / u * S[(i > 0) + (j > 0)] * mx3[i] * my3[j]) for j in range(3)]
                   for i in range(3)])
    assert np.abs(m4 - m3).max() <= 1e-13 * np.abs(m4).max()

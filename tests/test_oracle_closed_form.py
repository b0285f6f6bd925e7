"""Pins of the oracle's pair integrals against closed-form flat-triangle
potentials (tests/analytic.py) integrated by a graded high-order outer rule.

Covers every Sauter-Schwab case (identical, common edge at several dihedral
angles including the coplanar one, common vertex) and the regular case, for
the Laplace single and double layer, with constant and all nine pairs of
piecewise-linear local basis functions, and with the triangles' vertex lists
rotated and reflected (so the canonical reordering inside the oracle is
exercised).  The oracle runs at a high order so that its quadrature error is
below the tolerance.
"""
import numpy as np
import pytest

import analytic
import synth

HIGH = dict(q_regular=12, q_identical=14, q_edge=14, q_vertex=20)

CONFIGS = [("identical", 0.0), ("edge", 90.0), ("edge", 150.0), ("edge", 180.0),
           ("vertex", 0.0), ("far", 0.0)]
ORDERS = [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1)]


def _mesh(case, angle, oa, ob):
    m = synth.two_triangles(case, angle)
    tris = m.tris.copy()
    tris[0] = tris[0][list(oa)]
    tris[1] = tris[1][list(ob)]
    return m.verts, tris


def _check(ref, got, rtol, scale):
    assert abs(got - ref) <= rtol * max(abs(ref), scale), (ref, got)


@pytest.mark.parametrize("case,angle", CONFIGS)
@pytest.mark.parametrize("kernel", ["laplace_slp", "laplace_dlp"])
def test_p0_closed_form(oracle_mod, case, angle, kernel):
    for oa, ob in [(ORDERS[0], ORDERS[0]), (ORDERS[1], ORDERS[2]), (ORDERS[3], ORDERS[1])]:
        if case == "identical" and oa != ob:
            continue
        verts, tris = _mesh(case, angle, oa, ob)
        ref = analytic.pair_reference(verts[tris[0]], verts[tris[1]], kernel, n=96, p=6)
        got = oracle_mod.pair(verts, tris, 0, 1, kernel=kernel, **HIGH)
        assert abs(got.imag) == 0.0
        _check(ref, got.real, 1e-11, 1e-3)


@pytest.mark.parametrize("case,angle", CONFIGS)
@pytest.mark.parametrize("kernel", ["laplace_slp", "laplace_dlp"])
def test_p1_closed_form(oracle_mod, case, angle, kernel):
    oa, ob = (ORDERS[1], ORDERS[1]) if case == "identical" else (ORDERS[2], ORDERS[3])
    verts, tris = _mesh(case, angle, oa, ob)
    ta, tb = verts[tris[0]], verts[tris[1]]
    for la in range(3):
        for lb in range(3):
            ref = analytic.pair_reference(ta, tb, kernel, la, lb, n=96, p=6)
            got = oracle_mod.pair(verts, tris, 0, 1, la, lb, kernel=kernel, **HIGH)
            _check(ref, got.real, 1e-10, 1e-4)


def test_p1_sums_to_p0(oracle_mod):
    """sum_k lambda_k = 1 on each triangle: the 3x3 local matrix sums to the P0 value."""
    for case, angle in CONFIGS:
        m = synth.two_triangles(case, angle)
        p0 = oracle_mod.pair(m.verts, m.tris, 0, 1, kernel="laplace_slp")
        tot = sum(oracle_mod.pair(m.verts, m.tris, 0, 1, la, lb, kernel="laplace_slp")
                  for la in range(3) for lb in range(3))
        assert abs(tot - p0) < 1e-14 * abs(p0)


def test_octahedron_dense_brute_force(oracle_mod):
    """All 64 pairs of the octahedron (every case incl. regular) against the closed forms."""
    m = synth.octahedron()
    n = m.nt
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    for kernel in ("laplace_slp", "laplace_dlp"):
        got = oracle_mod.entries(m.verts, m.tris, rows, cols, kernel=kernel, **HIGH).real
        ref = np.array([analytic.pair_reference(m.verts[m.tris[i]], m.verts[m.tris[j]], kernel,
                                                n=80, p=6) for i, j in zip(rows, cols)])
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-10 * scale

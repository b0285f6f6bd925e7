"""Pins of the real part of the oracle's Helmholtz kernel (Eq. 2 with kappa > 0).

Re exp(i kappa r)/(4 pi r) = 1/(4 pi r) + (cos(kappa r) - 1)/(4 pi r).  The
Laplace part is pinned elsewhere against closed forms, so these tests pin the
excess, Re V_kappa - V_0, against an independent reference: the series
sum_{k>=1} (-1)^k kappa^(2k)/(2k)! int int r^(2k-1)/(4 pi) whose inner
integrals are closed-form flat-triangle potentials of odd powers of the
distance (tests/analytic.py, divergence theorem), integrated over the test
triangle by the graded outer rule.  The pairs are scaled so that kappa times
the pair's diameter stays near 2, where the series converges to rounding in a
few dozen terms.

A mis-scaled or mis-signed cosine argument in the oracle would give the value
of another wave number; every test also checks that a 1% change of kappa moves
the reference far outside the tolerance, so such a mistake cannot pass.
"""
import numpy as np
import pytest

import analytic
import synth

HIGH = dict(q_regular=14, q_identical=14, q_edge=14, q_vertex=18)
CONFIGS = [("identical", 0.0), ("edge", 60.0), ("vertex", 0.0), ("far", 0.0)]


def _scaled(case, angle, kappa):
    m = synth.two_triangles(case, angle)
    v = m.verts - m.verts.mean(axis=0)
    diam = max(np.linalg.norm(a - b) for a in v for b in v)
    return v * (2.0 / (kappa * diam)), m.tris


@pytest.mark.parametrize("kappa", [5.0, 8.0, 16.0])
@pytest.mark.parametrize("case,angle", CONFIGS)
def test_real_part_p0(oracle_mod, case, angle, kappa):
    verts, tris = _scaled(case, angle, kappa)
    ta, tb = verts[tris[0]], verts[tris[1]]
    helm = oracle_mod.pair(verts, tris, 0, 1, kernel="helmholtz_slp", kappa=kappa, **HIGH)
    lap = oracle_mod.pair(verts, tris, 0, 1, kernel="laplace_slp", **HIGH)
    ref = analytic.helmholtz_real_excess_pair(ta, tb, kappa, n=96, p=6)
    tol = 1e-13 * abs(lap.real)
    assert abs((helm.real - lap.real) - ref) <= tol, (helm.real - lap.real, ref)
    # the pin separates kappa from a 1% different wave number
    other = analytic.helmholtz_real_excess_pair(ta, tb, 1.01 * kappa, n=96, p=6)
    assert abs(other - ref) > 1e3 * tol


@pytest.mark.parametrize("case,angle", [("identical", 0.0), ("edge", 60.0), ("vertex", 0.0)])
def test_real_part_p1(oracle_mod, case, angle):
    kappa = 8.0
    verts, tris = _scaled(case, angle, kappa)
    ta, tb = verts[tris[0]], verts[tris[1]]
    for la, lb in [(0, 0), (1, 2), (2, 1)]:
        helm = oracle_mod.pair(verts, tris, 0, 1, la, lb, kernel="helmholtz_slp", kappa=kappa,
                               **HIGH)
        lap = oracle_mod.pair(verts, tris, 0, 1, la, lb, kernel="laplace_slp", **HIGH)
        ref = analytic.helmholtz_real_excess_pair(ta, tb, kappa, la, lb, n=96, p=6)
        assert abs((helm.real - lap.real) - ref) <= 1e-12 * abs(lap.real), (la, lb)


def test_real_part_unscaled_dense(oracle_mod):
    """A dense jittered icosahedron (every case, kappa r up to about 6) at kappa = 3."""
    kappa = 3.0
    mesh = synth.jitter(synth.icosahedron(), 0.05, 11)
    n = mesh.nt
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    helm = oracle_mod.entries(mesh.verts, mesh.tris, rows, cols, kernel="helmholtz_slp",
                              kappa=kappa, **HIGH).real
    lap = oracle_mod.entries(mesh.verts, mesh.tris, rows, cols, kernel="laplace_slp",
                             **HIGH).real
    pick = [(0, 0)] + [(i, j) for i, j in zip(rows, cols) if i < j][::9]
    for i, j in pick:
        ta, tb = mesh.verts[mesh.tris[i]], mesh.verts[mesh.tris[j]]
        ref = analytic.helmholtz_real_excess_pair(ta, tb, kappa, n=80, p=6, kmax=40)
        k = i * n + j
        assert abs((helm[k] - lap[k]) - ref) <= 1e-12 * np.abs(lap).max(), (i, j)


@pytest.mark.parametrize("basis", ["p0", "p1"])
@pytest.mark.parametrize("kappa", [5.0, 16.0])
def test_green_plus_real_part(oracle_mod, basis, kappa):
    """The 'plus' Green entry int phi_i g(x, z) dx at points z off the surface:
    its real part minus the Laplace entry against the odd-power series."""
    mesh = synth.jitter(synth.icosahedron(), 0.05, 5)
    v = mesh.verts * (1.0 / kappa)
    rng = synth.SplitMix64(17)
    n_idx = mesh.nt if basis == "p0" else mesh.nv
    idx = rng.integers(12, n_idx).astype(np.int64)
    d = rng.uniform(12 * 3, -1.0, 1.0).reshape(12, 3)
    z = d / np.linalg.norm(d, axis=1)[:, None] * (2.2 / kappa)     # outside the mesh
    nz = np.tile([0.0, 0.0, 1.0], (12, 1))
    ph, _ = oracle_mod.green_entries(v, mesh.tris, basis, idx, z, nz, kappa=kappa,
                                     rule="duffy", q=24)
    p0, _ = oracle_mod.green_entries(v, mesh.tris, basis, idx, z, nz, kappa=0.0,
                                     rule="duffy", q=24)
    for k in range(12):
        if basis == "p0":
            sup = [(int(idx[k]), -1)]
        else:
            sup = [(t, int(np.where(mesh.tris[t] == idx[k])[0][0]))
                   for t in np.where((mesh.tris == idx[k]).any(axis=1))[0]]
        ref = sum(analytic.helmholtz_real_excess(z[k:k + 1], v[mesh.tris[t]], kappa, lb)[0]
                  for t, lb in sup)
        assert abs((ph[k].real - p0[k].real) - ref) <= 1e-12 * abs(p0[k].real), k

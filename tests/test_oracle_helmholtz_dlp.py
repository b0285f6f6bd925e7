"""Pins of the oracle's Helmholtz double layer (the Brakhage-Werner operator's
K of Section 4): dg/dn_y = (x-y).n_y (1 - i kappa r) exp(i kappa r)/(4 pi r^3).

- Imaginary part: (x-y).n_y (sin z - z cos z)/(4 pi r^3), z = kappa r, and
  sin z - z cos z = z^3 (1/3 - z^2/30 + ...), so the imaginary integrand is
  the height (affine in x, constant in y) times an entire function of r^2:
  any pair, identical included, equals a plain tensor Gauss rule.
- Real part minus the Laplace double layer: the height times a series of
  closed-form odd-power potentials (tests/analytic.py).
- kappa -> 0 reproduces the Laplace double layer; a flat identical pair and a
  coplanar edge pair give exactly zero (the height vanishes).
Every check also separates kappa from a 1% different wave number.
"""
import numpy as np
import pytest

import analytic
import synth

HIGH = dict(q_regular=14, q_identical=14, q_edge=14, q_vertex=18)
CONFIGS = [("identical", 0.0), ("edge", 60.0), ("edge", 150.0), ("vertex", 0.0), ("far", 0.0)]


def _scaled(case, angle, kappa):
    m = synth.two_triangles(case, angle)
    v = m.verts - m.verts.mean(axis=0)
    diam = max(np.linalg.norm(a - b) for a in v for b in v)
    return v * (2.0 / (kappa * diam)), m.tris


def _plain(ta, tb, kappa, qa=13, qb=12):
    """Plain Duffy tensor Gauss of the imaginary part (different orders on the
    two triangles, so no point pair coincides)."""
    def pts(tri, q):
        z, w = np.polynomial.legendre.leggauss(q)
        z, w = (z + 1) / 2, w / 2
        S, T = np.meshgrid(z, z, indexing="ij")
        W = np.outer(w, w) * S
        s, t = S.ravel(), (S * T).ravel()
        X = tri[0] + s[:, None] * (tri[1] - tri[0]) + t[:, None] * (tri[2] - tri[1])
        g = np.linalg.norm(np.cross(tri[1] - tri[0], tri[2] - tri[1]))
        return X, W.ravel() * g
    X, WX = pts(ta, qa)
    Y, WY = pts(tb, qb)
    nb = np.cross(tb[1] - tb[0], tb[2] - tb[1])
    nb /= np.linalg.norm(nb)
    D = X[:, None, :] - Y[None, :, :]
    r = np.linalg.norm(D, axis=2)
    z = kappa * r
    # (sin z - z cos z)/z^3 by its series where z is small
    with np.errstate(all="ignore"):
        f = np.where(z > 1e-2, (np.sin(z) - z * np.cos(z)) / z ** 3,
                     1.0 / 3.0 - z * z / 30.0 + z ** 4 / 840.0)
    return float(np.sum(WX[:, None] * WY[None, :] * (D @ nb) * kappa ** 3 * f / (4 * np.pi)))


@pytest.mark.parametrize("kappa", [3.0, 8.0, 16.0])
@pytest.mark.parametrize("case,angle", CONFIGS)
def test_imaginary_part_plain_gauss(oracle_mod, case, angle, kappa):
    verts, tris = _scaled(case, angle, kappa)
    ta, tb = verts[tris[0]], verts[tris[1]]
    got = oracle_mod.pair(verts, tris, 0, 1, kernel="helmholtz_dlp", kappa=kappa, **HIGH)
    ref = _plain(ta, tb, kappa)
    scale = abs(oracle_mod.pair(verts, tris, 0, 1, kernel="helmholtz_slp", kappa=kappa,
                                **HIGH).imag)
    assert abs(got.imag - ref) <= 1e-13 * scale, (got.imag, ref)
    if case != "identical":
        assert abs(_plain(ta, tb, 1.01 * kappa) - ref) > 1e3 * 1e-13 * scale


@pytest.mark.parametrize("kappa", [5.0, 16.0])
@pytest.mark.parametrize("case,angle", CONFIGS)
def test_real_part_closed_form(oracle_mod, case, angle, kappa):
    verts, tris = _scaled(case, angle, kappa)
    ta, tb = verts[tris[0]], verts[tris[1]]
    helm = oracle_mod.pair(verts, tris, 0, 1, kernel="helmholtz_dlp", kappa=kappa, **HIGH)
    lap = oracle_mod.pair(verts, tris, 0, 1, kernel="laplace_dlp", **HIGH)
    ref = analytic.helmholtz_dlp_real_excess_pair(ta, tb, kappa, n=96, p=6)
    scale = max(abs(helm), abs(lap))
    assert abs((helm.real - lap.real) - ref) <= 1e-12 * scale, (helm.real - lap.real, ref)
    if case not in ("identical", "edge") or angle != 0.0:
        other = analytic.helmholtz_dlp_real_excess_pair(ta, tb, 1.01 * kappa, n=96, p=6)
        if abs(ref) > 1e-6 * scale:
            assert abs(other - ref) > 1e3 * 1e-12 * scale


def test_real_part_p1(oracle_mod):
    kappa = 8.0
    for case, angle in [("edge", 60.0), ("vertex", 0.0), ("far", 0.0)]:
        verts, tris = _scaled(case, angle, kappa)
        ta, tb = verts[tris[0]], verts[tris[1]]
        scale = max(abs(oracle_mod.pair(verts, tris, 0, 1, la, lb, kernel="helmholtz_dlp",
                                        kappa=kappa, **HIGH)) for la in range(3) for lb in range(3))
        for la, lb in [(0, 0), (1, 2), (2, 1)]:
            helm = oracle_mod.pair(verts, tris, 0, 1, la, lb, kernel="helmholtz_dlp",
                                   kappa=kappa, **HIGH)
            lap = oracle_mod.pair(verts, tris, 0, 1, la, lb, kernel="laplace_dlp", **HIGH)
            ref = analytic.helmholtz_dlp_real_excess_pair(ta, tb, kappa, la, lb, n=96, p=6)
            assert abs((helm.real - lap.real) - ref) <= 1e-12 * scale, (case, la, lb)


def test_small_kappa_is_laplace_and_flat_pairs_vanish(oracle_mod):
    mesh = synth.jitter(synth.icosahedron(), 0.05, 3)
    n = mesh.nt
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    q = dict(q_regular=5, q_identical=5, q_edge=5, q_vertex=5)
    K0 = oracle_mod.entries(mesh.verts, mesh.tris, rows, cols, kernel="laplace_dlp", **q).real
    K1 = oracle_mod.entries(mesh.verts, mesh.tris, rows, cols, kernel="helmholtz_dlp",
                            kappa=1e-9, **q)
    assert np.abs(K1.real - K0).max() < 1e-14 * np.abs(K0).max()
    assert np.abs(K1.imag).max() < 1e-20
    m = synth.two_triangles("identical", 0.0)
    assert oracle_mod.pair(m.verts, m.tris, 0, 1, kernel="helmholtz_dlp", kappa=4.0, **HIGH) == 0
    # the coplanar edge pair is flat up to the rounding of sin(pi) in its vertex
    m = synth.two_triangles("edge", 180.0)
    v = oracle_mod.pair(m.verts, m.tris, 0, 1, kernel="helmholtz_dlp", kappa=4.0, **HIGH)
    s = oracle_mod.pair(m.verts, m.tris, 0, 1, kernel="helmholtz_slp", kappa=4.0, **HIGH)
    assert abs(v) < 1e-14 * abs(s)

"""Pins of the oracle against identities the mathematics fixes.

P2 Gauss's identity: on a closed flat-triangle surface the double layer of a
   constant density is exactly -1/2 at every face-interior point, so the row
   sums of the Galerkin double-layer matrix equal -1/2 times the row sums of
   the mass matrix, up to quadrature error only (which shrinks with the order).
P3 symmetry of the single-layer Galerkin matrix (Laplace; complex-symmetric
   Helmholtz), up to quadrature error.
P5 exponential convergence in the order for every singular case.
P6 Helmholtz: Im k = sin(kappa r)/(4 pi r) is smooth, so the imaginary part of
   any pair integral equals a plain tensor Gauss rule; kappa -> 0 gives Laplace.
P7 invariances: rigid motion; dilation by L scales the single layer by L^3 and
   the double layer by L^2; reversing every orientation flips the double layer.
Plus argument validation and the sphere sum  sum_ij V_ij -> 4 pi.
"""
import numpy as np
import pytest

import synth

Q3 = dict(q_regular=3, q_identical=3, q_edge=3, q_vertex=3)
Q5 = dict(q_regular=5, q_identical=5, q_edge=5, q_vertex=5)
Q8 = dict(q_regular=8, q_identical=8, q_edge=8, q_vertex=8)


def dense(oracle_mod, mesh, basis="p0", **kw):
    n = mesh.nt if basis == "p0" else mesh.nv
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    return oracle_mod.entries(mesh.verts, mesh.tris, rows, cols, basis=basis, **kw).reshape(n, n)


def areas(mesh):
    v = mesh.verts[mesh.tris]
    return 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 1]), axis=1)


def p1_mass_rowsum(mesh):
    out = np.zeros(mesh.nv)
    a = areas(mesh)
    for k in range(3):
        np.add.at(out, mesh.tris[:, k], a / 3.0)
    return out


@pytest.mark.parametrize("meshname", ["octasphere", "cube", "torus"])
def test_gauss_identity_p0(oracle_mod, meshname):
    mesh = {"octasphere": synth.octasphere(3), "cube": synth.cube_surface(3),
            "torus": synth.torus(12, 5)}[meshname]
    res = []
    for q in (Q3, Q5, Q8):
        K = dense(oracle_mod, mesh, kernel="laplace_dlp", **q).real
        res.append(np.abs(K.sum(axis=1) + 0.5 * areas(mesh)).max() / areas(mesh).max())
    assert res[2] < 1e-5
    assert res[2] < res[1] < res[0]


def test_gauss_identity_p1(oracle_mod):
    mesh = synth.octasphere(3)
    res = []
    for q in (Q3, Q5, Q8):
        K = dense(oracle_mod, mesh, basis="p1", kernel="laplace_dlp", **q).real
        m1 = p1_mass_rowsum(mesh)
        res.append(np.abs(K.sum(axis=1) + 0.5 * m1).max() / m1.max())
    assert res[2] < 1e-5
    assert res[2] < res[1] < res[0]


@pytest.mark.parametrize("basis", ["p0", "p1"])
@pytest.mark.parametrize("kernel,kappa", [("laplace_slp", 0.0), ("helmholtz_slp", 3.0)])
def test_slp_symmetry(oracle_mod, basis, kernel, kappa):
    mesh = synth.jitter(synth.icosahedron(), 0.05, 7)
    gaps = []
    for q in (Q3, Q8):
        V = dense(oracle_mod, mesh, basis, kernel=kernel, kappa=kappa, **q)
        gaps.append(np.abs(V - V.T).max() / np.abs(V).max())
    assert gaps[1] < 1e-9
    assert gaps[1] < gaps[0]


@pytest.mark.parametrize("case,angle,aspect", [("identical", 0, 1), ("edge", 30, 1),
                                               ("edge", 90, 1), ("edge", 150, 3),
                                               ("vertex", 0, 1), ("vertex", 0, 6)])
@pytest.mark.parametrize("kernel", ["laplace_slp", "laplace_dlp", "helmholtz_slp"])
def test_exponential_convergence(oracle_mod, case, angle, aspect, kernel):
    m = synth.two_triangles(case, angle, aspect)
    vals = [oracle_mod.pair(m.verts, m.tris, 0, 1, kernel=kernel, kappa=4.0, q_identical=q,
                            q_edge=q, q_vertex=q) for q in range(2, 23, 2)]
    ref = vals[-1]
    err = np.array([abs(v - ref) for v in vals[:-1]]) / max(abs(ref), 1e-3)
    # geometric decay: the error over the first half of the orders shrinks by
    # at least two orders of magnitude, and the last one is small
    assert err[4] < 1e-2 * err[0] + 1e-15
    assert err[-1] < 1e-8


def _plain_imag(ta, tb, kappa, qa=13, qb=12):
    """Im of the pair integral by a plain Duffy tensor Gauss rule in numpy (different
    orders on the two triangles, so no point pair coincides)."""
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
    r = np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=2)
    return float(np.sum(WX[:, None] * WY[None, :] * np.sin(kappa * r) / (4 * np.pi * r)))


def test_helmholtz_imaginary_part_is_smooth(oracle_mod):
    """Im part of any pair (identical included) = plain tensor Gauss of sin(kr)/(4 pi r)."""
    for case, angle in [("identical", 0), ("edge", 60), ("vertex", 0), ("far", 0)]:
        m = synth.two_triangles(case, angle)
        ss = oracle_mod.pair(m.verts, m.tris, 0, 1, kernel="helmholtz_slp", kappa=5.0,
                             q_identical=14, q_edge=14, q_vertex=14, q_regular=14)
        plain = _plain_imag(m.verts[m.tris[0]], m.verts[m.tris[1]], 5.0)
        assert abs(ss.imag - plain) < 1e-13 * abs(plain)


def test_helmholtz_small_kappa_is_laplace(oracle_mod):
    mesh = synth.octahedron()
    V0 = dense(oracle_mod, mesh, kernel="laplace_slp", **Q5)
    V1 = dense(oracle_mod, mesh, kernel="helmholtz_slp", kappa=1e-9, **Q5)
    assert np.abs(V1.real - V0.real).max() < 1e-14 * np.abs(V0).max()
    # Im part ~ kappa/(4 pi) * |T_i||T_j|
    a = areas(mesh)
    assert np.allclose(V1.imag, 1e-9 / (4 * np.pi) * np.outer(a, a), rtol=1e-6, atol=0)


def _rotation(seed):
    rng = synth.SplitMix64(seed)
    A = rng.uniform(9, -1, 1).reshape(3, 3)
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))[None, :]


@pytest.mark.parametrize("kernel", ["laplace_slp", "laplace_dlp", "helmholtz_slp"])
def test_rigid_motion(oracle_mod, kernel):
    mesh = synth.jitter(synth.icosahedron(), 0.05, 3)
    V = dense(oracle_mod, mesh, kernel=kernel, kappa=2.0, **Q5)
    Q = _rotation(11)
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    moved = synth.Mesh(mesh.verts @ Q.T + np.array([1e3, -2e3, 5e2]), mesh.tris)
    W = dense(oracle_mod, moved, kernel=kernel, kappa=2.0, **Q5)
    assert np.abs(W - V).max() < 1e-10 * np.abs(V).max()


def test_dilation_and_orientation(oracle_mod):
    mesh = synth.octasphere(2)
    L = 2.5
    big = synth.Mesh(mesh.verts * L, mesh.tris)
    flipped = synth.Mesh(mesh.verts, mesh.tris[:, [0, 2, 1]].copy())
    V = dense(oracle_mod, mesh, kernel="laplace_slp", **Q5).real
    K = dense(oracle_mod, mesh, kernel="laplace_dlp", **Q5).real
    assert np.abs(dense(oracle_mod, big, kernel="laplace_slp", **Q5).real - L ** 3 * V).max() \
        < 1e-13 * L ** 3 * np.abs(V).max()
    assert np.abs(dense(oracle_mod, big, kernel="laplace_dlp", **Q5).real - L ** 2 * K).max() \
        < 1e-13 * L ** 2 * np.abs(K).max()
    Kf = dense(oracle_mod, flipped, kernel="laplace_dlp", **Q5).real
    Vf = dense(oracle_mod, flipped, kernel="laplace_slp", **Q5).real
    # reversing the orientation reparametrises every triangle, so the rule sees
    # other points: the values agree to quadrature accuracy, the sign flips exactly
    assert np.abs(Kf + K).max() < 1e-5 * np.abs(K).max()
    assert np.abs(Vf - V).max() < 1e-5 * np.abs(V).max()


def test_sphere_single_layer_total(oracle_mod):
    """sum_ij V_ij = int int 1/(4 pi |x-y|) -> 4 pi on the unit sphere, O(h^2)."""
    errs = []
    for k in (1, 2):
        mesh = synth.icosphere(k)
        V = dense(oracle_mod, mesh, kernel="laplace_slp", regular_rule="tri7",
                  q_identical=4, q_edge=4, q_vertex=4).real
        errs.append(abs(V.sum() - 4 * np.pi))
    assert errs[1] < errs[0] / 3.0


def test_argument_validation(oracle_mod):
    m = synth.octahedron()
    with pytest.raises(ValueError):
        oracle_mod.entries(m.verts, m.tris, [0], [8])
    with pytest.raises(ValueError):
        oracle_mod.entries(m.verts, m.tris, [0], [0], q_edge=0)
    bad = m.tris.copy()
    bad[0] = [0, 0, 1]
    with pytest.raises(ValueError):
        oracle_mod.entries(m.verts, bad, [0], [1])
    assert len(oracle_mod.entries(m.verts, m.tris, [], [])) == 0


def test_absolute_sums(oracle_mod):
    """entries_absolute: equal to the entry where the integrand has one sign (single
    layer), never below |entry| (double layer, Helmholtz), and positive."""
    mesh = synth.jitter(synth.cube_surface(2), 0.05, 5)
    n = mesh.nt
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    for kernel, kappa in (("laplace_slp", 0.0), ("laplace_dlp", 0.0), ("helmholtz_slp", 6.0)):
        g = oracle_mod.entries(mesh.verts, mesh.tris, rows, cols, kernel=kernel, kappa=kappa, **Q5)
        A = oracle_mod.entries_absolute(mesh.verts, mesh.tris, rows, cols, kernel=kernel,
                                        kappa=kappa, **Q5)
        assert np.all(A >= np.abs(g) * (1 - 1e-14))
        if kernel == "laplace_slp":
            assert np.allclose(A, g.real, rtol=1e-15, atol=0)
    # P1 single layer: hat functions are nonnegative, so again A = g
    g = oracle_mod.entries(mesh.verts, mesh.tris, [0, 3], [1, 5], basis="p1", **Q5).real
    A = oracle_mod.entries_absolute(mesh.verts, mesh.tris, [0, 3], [1, 5], basis="p1", **Q5)
    assert np.allclose(A, g, rtol=1e-15, atol=0)

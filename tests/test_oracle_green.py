"""Pins of the oracle's Green quadrature entries (Section 2.3: the matrices
A_t of Green's representation formula), independent of the oracle itself:

* piecewise-constant, Laplace: the closed-form potentials of a flat triangle,
  int_T 1/r and int_T (y - z)/r^3 (tests/analytic.py);
* piecewise-linear, Laplace: the closed-form potential of a linear density,
  and its gradient in z by Richardson-extrapolated central differences;
* Helmholtz: the normal derivative equals the z-derivative of the oracle's
  own first entry (a wrong sign, a dropped (1 - i kappa r) factor or a
  transposed argument fails), and kappa -> 0 reproduces Laplace;
* the two triangle rules agree where the integrand is smooth;
* Green's representation formula on the auxiliary box omega_t (Section 2.3,
  G|_{t x s} ~ A_t B_ts): the oracle's entries, scaled as the paper scales
  a_{t+}, a_{t-}, b_{ts+}, b_{ts-}, reproduce the Galerkin entries of an
  admissible block, with an error that falls geometrically as the Gauss rule
  on the box faces is refined; with the minus part's sign flipped it does not."""
import numpy as np
import pytest

import oracle
import synth
from analytic import FOUR_PI, inner, potentials


@pytest.fixture(scope="module")
def mesh():
    return synth.jitter(synth.icosphere(2), 0.05, 19)


def _points(mesh, idx, basis, dist, seed):
    """Points z at distance `dist` (times the support size) outside each
    basis function's support, with random unit normals."""
    rng = np.random.default_rng(seed)
    z, nz = [], []
    for i in idx:
        if basis == "p0":
            c = mesh.verts[mesh.tris[i]].mean(axis=0)
            h = np.linalg.norm(mesh.verts[mesh.tris[i][1]] - mesh.verts[mesh.tris[i][0]])
        else:
            c = mesh.verts[i]
            h = 2.0 * np.linalg.norm(mesh.verts[mesh.tris[np.any(mesh.tris == i, axis=1)]]
                                     .reshape(-1, 3) - c, axis=1).max()
        # outward (the mesh is a sphere about the origin), tilted at random:
        # the point stays more than half of dist * h above the support
        d = rng.normal(size=3)
        u = c / np.linalg.norm(c) + 0.3 * d / np.linalg.norm(d)
        z.append(c + dist * h * u / np.linalg.norm(u))
        n = rng.normal(size=3)
        nz.append(n / np.linalg.norm(n))
    return np.array(z), np.array(nz)


def _support(mesh, i):
    return [(t, list(mesh.tris[t]).index(i)) for t in np.nonzero(np.any(mesh.tris == i, axis=1))[0]]


def _closed_p1_plus(mesh, i, z):
    """int phi_i(y) / (4 pi |y - z|) dy from the closed form, summed over the support."""
    return sum(inner(z[None, :], mesh.verts[mesh.tris[t]], "laplace_slp", lb=k)[0]
               for t, k in _support(mesh, i))


def _fd_gradient(f, z, h):
    """Gradient of f at z by central differences, Richardson-extrapolated."""
    def cd(hh):
        g = np.zeros(3)
        for c in range(3):
            e = np.zeros(3)
            e[c] = hh
            g[c] = (f(z + e) - f(z - e)) / (2 * hh)
        return g
    return (4.0 * cd(h / 2) - cd(h)) / 3.0


@pytest.mark.parametrize("dist", [1.0, 2.0, 4.0])
def test_p0_laplace_against_closed_forms(mesh, dist):
    idx = np.arange(0, mesh.nt, 7)
    z, nz = _points(mesh, idx, "p0", dist, 1)
    plus, minus = oracle.green_entries(mesh.verts, mesh.tris, "p0", idx, z, nz,
                                       rule="duffy", q=40)
    for k, i in enumerate(idx):
        tri = mesh.verts[mesh.tris[i]]
        S, G, D, Dv, w, rho = potentials(z[k][None, :], tri)
        n = np.cross(tri[1] - tri[0], tri[2] - tri[1])
        n /= np.linalg.norm(n)
        # int_T (y - z)/r^3 dy = Dvec - n D (D = w int 1/r^3, w = (z - rho).n)
        vec = Dv[0] - n * D[0]
        assert plus[k].real == pytest.approx(S[0] / FOUR_PI, rel=1e-11)
        assert minus[k].real == pytest.approx(nz[k] @ vec / FOUR_PI, rel=1e-9, abs=1e-13)
        assert plus[k].imag == 0.0 and minus[k].imag == 0.0


@pytest.mark.parametrize("dist", [1.0, 3.0])
def test_p1_laplace_against_closed_forms(mesh, dist):
    idx = np.arange(0, mesh.nv, 9)
    z, nz = _points(mesh, idx, "p1", dist, 2)
    plus, minus = oracle.green_entries(mesh.verts, mesh.tris, "p1", idx, z, nz,
                                       rule="duffy", q=40)
    for k, i in enumerate(idx):
        want = _closed_p1_plus(mesh, i, z[k])
        assert plus[k].real == pytest.approx(want, rel=1e-11)
        grad = _fd_gradient(lambda p: _closed_p1_plus(mesh, i, p), z[k],
                            1e-3 * np.linalg.norm(z[k] - mesh.verts[i]))
        assert minus[k].real == pytest.approx(nz[k] @ grad, rel=1e-7, abs=1e-12)


def test_finite_differences_reproduce_the_p0_closed_form(mesh):
    # the differencing used above, checked where the closed form is known
    tri = mesh.verts[mesh.tris[3]]
    z = tri.mean(axis=0) * 1.4
    n = np.cross(tri[1] - tri[0], tri[2] - tri[1])
    n /= np.linalg.norm(n)
    S = lambda p: potentials(p[None, :], tri)[0][0]
    _, _, D, Dv, _, _ = potentials(z[None, :], tri)
    grad = _fd_gradient(S, z, 1e-3 * np.linalg.norm(z - tri[0]))
    # grad_z int 1/|y - z| = int (y - z)/r^3
    assert np.allclose(grad, Dv[0] - n * D[0], rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("basis", ["p0", "p1"])
@pytest.mark.parametrize("kappa", [1.0, 8.0])
def test_helmholtz_normal_derivative_is_the_z_derivative(mesh, basis, kappa):
    n_idx = mesh.nt if basis == "p0" else mesh.nv
    idx = np.arange(0, n_idx, 23)
    z, nz = _points(mesh, idx, basis, 1.0, 3)
    plus, minus = oracle.green_entries(mesh.verts, mesh.tris, basis, idx, z, nz,
                                       kappa=kappa, rule="duffy", q=20)
    for k, i in enumerate(idx):
        def f(p, part):
            v = oracle.green_entries(mesh.verts, mesh.tris, basis, [i], p[None, :], nz[k:k + 1],
                                     kappa=kappa, rule="duffy", q=20)[0][0]
            return v.real if part == 0 else v.imag
        h = 1e-3 * np.linalg.norm(z[k] - mesh.verts[mesh.tris[i][0]] if basis == "p0"
                                  else z[k] - mesh.verts[i])
        for part in (0, 1):
            g = _fd_gradient(lambda p: f(p, part), z[k], h)
            got = minus[k].real if part == 0 else minus[k].imag
            assert got == pytest.approx(nz[k] @ g, rel=1e-7, abs=1e-12 * abs(minus[k]))


@pytest.mark.parametrize("basis", ["p0", "p1"])
def test_small_wavenumber_reproduces_laplace(mesh, basis):
    n_idx = mesh.nt if basis == "p0" else mesh.nv
    idx = np.arange(0, n_idx, 11)
    z, nz = _points(mesh, idx, basis, 1.0, 4)
    pl, ml = oracle.green_entries(mesh.verts, mesh.tris, basis, idx, z, nz, rule="duffy", q=12)
    ph, mh = oracle.green_entries(mesh.verts, mesh.tris, basis, idx, z, nz, kappa=1e-7,
                                  rule="duffy", q=12)
    assert np.allclose(ph.real, pl.real, rtol=1e-12)
    assert np.allclose(mh.real, ml.real, rtol=1e-12, atol=1e-18)
    # Im exp(i kappa r)/r = kappa + O(kappa^3 r^2): the imaginary part is kappa
    # times the integral of the basis function over 4 pi
    area = []
    for i in idx:
        tris = [mesh.tris[i]] if basis == "p0" else mesh.tris[np.any(mesh.tris == i, axis=1)]
        a = sum(0.5 * np.linalg.norm(np.cross(mesh.verts[t[1]] - mesh.verts[t[0]],
                                              mesh.verts[t[2]] - mesh.verts[t[1]])) for t in tris)
        area.append(a if basis == "p0" else a / 3.0)
    assert np.allclose(ph.imag / 1e-7, np.array(area) / FOUR_PI, rtol=1e-9)


def test_rules_agree_on_smooth_integrands(mesh):
    idx = np.arange(0, mesh.nv, 5)
    z, nz = _points(mesh, idx, "p1", 8.0, 5)
    a = oracle.green_entries(mesh.verts, mesh.tris, "p1", idx, z, nz, kappa=2.0, rule="tri7")
    b = oracle.green_entries(mesh.verts, mesh.tris, "p1", idx, z, nz, kappa=2.0, rule="duffy",
                             q=16)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-6)


def test_bad_index_is_rejected(mesh):
    with pytest.raises(ValueError):
        oracle.green_entries(mesh.verts, mesh.tris, "p1", [mesh.nv], [[3.0, 0, 0]], [[1.0, 0, 0]])


def _box_gap(amin, amax, bmin, bmax):
    gap = np.maximum(0.0, np.maximum(np.asarray(amin) - bmax, np.asarray(bmin) - amax))
    return float(np.linalg.norm(gap))


@pytest.mark.parametrize("basis", ["p0", "p1"])
@pytest.mark.parametrize("kernel,kappa", [("laplace_slp", 0.0), ("helmholtz_slp", 3.0)])
def test_representation_formula_reproduces_admissible_blocks(basis, kernel, kappa):
    """For x in B_t and y outside omega_t, Green's representation formula on
    the boundary of omega_t gives g(x, y) = int [g(x, z) dg/dn(z)(z, y) -
    dg/dn(z)(x, z) g(z, y)] dz; a Gauss rule (z_nu, w_nu) on the faces turns
    it into g_ij ~ sum_nu a_{t+,i nu} b_{ts+,j nu} - a_{t-,i nu} b_{ts-,j nu}
    with a_{t+} = sqrt(w) int phi_i g, a_{t-} = sqrt(w) delta_t int phi_i dg/dn,
    b_{ts+} = sqrt(w) int psi_j dg/dn, b_{ts-} = sqrt(w) / delta_t int psi_j g.
    With Radon's 7 points on every triangle on both sides, the Galerkin entry
    of the admissible block uses the same points, so only the box rule's error
    remains.  Blocks are taken with B_s at least delta_t / 2 away from omega_t
    (the paper's bound on the distance to the boundary)."""
    from synth.structure import build_block_partition, green_box_points
    mesh = synth.jitter(synth.icosphere(3), 0.05, 7)
    part = build_block_partition(mesh, basis, leaf_size=32, eta=2.0)
    tree = part.tree
    best = None
    for t, s in part.far:
        lo, hi = np.asarray(tree.bmin[t]), np.asarray(tree.bmax[t])
        d = float(np.linalg.norm(hi - lo))
        ratio = _box_gap(lo - d / 2, hi + d / 2, tree.bmin[s], tree.bmax[s]) / d
        size = min(len(tree.indices(t)), len(tree.indices(s)))
        if ratio >= 0.5 and size >= 8 and (best is None or size > best[0]):
            best = (size, t, s)
    assert best is not None
    _, t, s = best
    rt, cs = tree.indices(t), tree.indices(s)
    G = oracle.entries(mesh.verts, mesh.tris, np.repeat(rt, len(cs)), np.tile(cs, len(rt)),
                       kernel=kernel, kappa=kappa, basis=basis, q_regular=3,
                       regular_rule="tri7", q_identical=5, q_edge=5, q_vertex=5)
    G = np.asarray(G).reshape(len(rt), len(cs))
    errs, wrong = [], []
    for g in (4, 8, 12):
        z, nz, w, delta = green_box_points(tree.bmin[t], tree.bmax[t], g)
        m = len(z)

        def ent(idx):
            ii = np.repeat(idx, m)
            zz = np.tile(np.arange(m), len(idx))
            P, M = oracle.green_entries(mesh.verts, mesh.tris, basis, ii, z[zz], nz[zz],
                                        kappa=kappa, rule="tri7")
            return P.reshape(len(idx), m), M.reshape(len(idx), m)

        Pt, Mt = ent(rt)
        Ps, Ms = ent(cs)
        sw = np.sqrt(w)
        a_plus, a_minus = Pt * sw, Mt * (sw * delta)
        b_plus, b_minus = Ms * sw, Ps * (sw / delta)
        approx = a_plus @ b_plus.T - a_minus @ b_minus.T
        flipped = a_plus @ b_plus.T + a_minus @ b_minus.T
        if kernel != "helmholtz_slp":
            assert np.abs(approx.imag).max() == 0.0
            approx, flipped = approx.real, flipped.real
        scale = np.abs(G).max()
        errs.append(np.abs(G - approx).max() / scale)
        wrong.append(np.abs(G - flipped).max() / scale)
    assert errs[0] < 5e-2 and errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs
    assert errs[2] < 2e-5, errs
    assert min(wrong) > 0.1, wrong

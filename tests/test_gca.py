"""Host GCA pivots (Sections 2.3-2.4): bem_gca_pivots against a numpy
restatement of the Green quadrature matrix A_t and of cross approximation with
complete pivoting, plus the properties the H^2 form relies on (pivots inside
the cluster, nested in the sons' pivots, rank bound, row skeletons of
admissible blocks close to the SVD optimum).  Host only: no GPU."""
import numpy as np
import pytest

import paper_1510_07244_gb300 as pkg
from paper_1510_07244_gb300 import build as libbuild
from synth import meshes, structure


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return pkg.load()


def supports(tris, basis):
    sup = {}
    if basis == "p0":
        for tr in range(len(tris)):
            sup[tr] = [(tr, -1)]
    else:
        for tr in range(len(tris)):
            for k in range(3):
                sup.setdefault(int(tris[tr, k]), []).append((tr, k))
    return sup


def green_matrix(oracle_mod, verts, tris, sup, rows, cluster, g, kappa):
    """A_t = (A_t+, A_t-) of Section 2.3 at the given rows, written from the
    representation formula: boxes, Gauss points on the faces of omega_t and
    Radon's rule on every support triangle."""
    s, t, w = oracle_mod.radon7()
    v = verts[tris]
    lo = np.min([v[tr].min(0) for i in cluster for tr, _ in sup[i]], axis=0)
    hi = np.max([v[tr].max(0) for i in cluster for tr, _ in sup[i]], axis=0)
    delta = np.linalg.norm(hi - lo)
    lo, hi = lo - delta / 2, hi + delta / 2
    x, wx = np.polynomial.legendre.leggauss(g)
    x, wx = (x + 1) / 2, wx / 2
    Z, N, W = [], [], []
    for ax in range(3):
        for side in range(2):
            a1, a2 = (ax + 1) % 3, (ax + 2) % 3
            for i in range(g):
                for j in range(g):
                    z, n = np.zeros(3), np.zeros(3)
                    z[ax] = hi[ax] if side else lo[ax]
                    z[a1] = lo[a1] + x[i] * (hi[a1] - lo[a1])
                    z[a2] = lo[a2] + x[j] * (hi[a2] - lo[a2])
                    n[ax] = 1.0 if side else -1.0
                    Z.append(z)
                    N.append(n)
                    W.append(wx[i] * wx[j] * (hi[a1] - lo[a1]) * (hi[a2] - lo[a2]))
    Z, N, W = np.array(Z), np.array(N), np.array(W)
    m = len(W)
    A = np.zeros((len(rows), 2 * m), complex)
    for r, i in enumerate(rows):
        for tr, loc in sup[i]:
            a, b, c = v[tr]
            X = a + np.outer(s, b - a) + np.outer(t, c - b)
            area2 = np.linalg.norm(np.cross(b - a, c - b))
            lam = np.ones(len(s)) if loc < 0 else [1 - s, s - t, t][loc]
            D = X[:, None, :] - Z[None, :, :]          # x - z
            R = np.linalg.norm(D, axis=2)
            G = np.exp(1j * kappa * R) / (4 * np.pi * R)
            # n(z) . grad_z g(x, z)
            dG = G * np.einsum("pmk,mk->pm", D, N) / R**2 * (1 - 1j * kappa * R)
            f = (w * area2 * lam)[:, None]
            A[r, :m] += (f * G).sum(0)
            A[r, m:] += (f * dG).sum(0)
    A[:, :m] *= np.sqrt(W)
    A[:, m:] *= np.sqrt(W) * delta
    return A


def cross_approximation(A, eps, kmax):
    A = A.copy()
    piv, first = [], None
    for k in range(min(kmax, *A.shape)):
        i, j = np.unravel_index(np.argmax(np.abs(A)), A.shape)
        if k == 0:
            first = abs(A[i, j])
        elif abs(A[i, j]) <= eps * first:
            break
        piv.append(int(i))
        A = A - np.outer(A[:, j] / A[i, j], A[i, :])
    return piv


def setup(basis, levels=3, leaf=16, kappa=0.0, g=3, eps=1e-6, rank=12, **kw):
    mesh = meshes.jitter(meshes.icosphere(levels), 0.1, 7)
    part = structure.build_block_partition(mesh, basis, leaf, 2.0)
    ptr, idx = part.cluster_csr()
    son = part.son_array()
    pp, pi = pkg.bem_gca_pivots(mesh.verts, mesh.tris, basis, ptr, idx, son, kappa=kappa,
                                gauss_per_face=g, eps=eps, max_rank=rank, **kw)
    piv = [pi[pp[c]:pp[c + 1]] for c in range(len(pp) - 1)]
    return mesh, part, ptr, idx, son, piv


@pytest.mark.parametrize("basis,kappa", [("p0", 0.0), ("p1", 0.0), ("p0", 2.0)])
def test_pivots_match_restatement(oracle_mod, basis, kappa):
    mesh, part, ptr, idx, son, piv = setup(basis, kappa=kappa)
    sup = supports(mesh.tris, basis)
    for c in range(len(piv)):
        cluster = list(idx[ptr[c]:ptr[c + 1]])
        rows = cluster if son[c, 0] < 0 else list(piv[son[c, 0]]) + list(piv[son[c, 1]])
        A = green_matrix(oracle_mod, mesh.verts, mesh.tris, sup, rows, cluster, 3, kappa)
        expect = sorted(rows[k] for k in cross_approximation(A, 1e-6, 12))
        assert list(piv[c]) == expect, c


def test_structure_of_pivots():
    mesh, part, ptr, idx, son, piv = setup("p1", levels=4, leaf=32, rank=16, g=4)
    for c in range(len(piv)):
        cluster = set(idx[ptr[c]:ptr[c + 1]].tolist())
        p = piv[c].tolist()
        assert p == sorted(set(p))
        assert set(p) <= cluster
        assert len(p) == min(16, len(cluster))        # eps never binds at 1e-6, rank 16
        if son[c, 0] >= 0:
            assert set(p) <= set(piv[son[c, 0]].tolist()) | set(piv[son[c, 1]].tolist())


def test_thread_count_does_not_change_result():
    a = setup("p0", n_threads=1)[-1]
    b = setup("p0", n_threads=5)[-1]
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_tolerance_and_rank_bound():
    loose = setup("p0", eps=1e-2, rank=12)[-1]
    tight = setup("p0", eps=1e-9, rank=12)[-1]
    assert sum(map(len, loose)) < sum(map(len, tight))
    assert max(map(len, setup("p0", rank=5)[-1])) == 5


@pytest.mark.parametrize("basis,kernel,kappa,tol", [("p0", "laplace_slp", 0.0, 2e-5),
                                                    ("p1", "laplace_slp", 0.0, 2e-5),
                                                    ("p0", "helmholtz_slp", 6.0, 1e-3)])
def test_row_skeletons_of_admissible_blocks(oracle_mod, basis, kernel, kappa, tol):
    """G|t x s lies close to the span of its pivot rows G|t~ x s: residual
    within a small factor of the best rank-|t~| approximation (SVD)."""
    mesh, part, ptr, idx, son, piv = setup(basis, kappa=kappa)
    checked = 0
    for t, s in part.far[:: max(1, len(part.far) // 30)]:
        it, js = part.tree.indices(t), part.tree.indices(s)
        k = len(piv[t])
        if k >= min(len(it), len(js)):
            continue
        G = oracle_mod.entries(mesh.verts, mesh.tris, np.repeat(it, len(js)), np.tile(js, len(it)),
                               kernel=kernel, kappa=kappa, basis=basis, regular_rule="tri7",
                               q_regular=1, q_identical=4, q_edge=4,
                               q_vertex=4).reshape(len(it), len(js))
        sel = [list(it).index(i) for i in piv[t]]
        Q, _ = np.linalg.qr(G[sel].T)                  # orthonormal basis of the pivot rows
        res = np.linalg.norm(G - G @ Q.conj() @ Q.T) / np.linalg.norm(G)
        sv = np.linalg.svd(G, compute_uv=False)
        best = np.sqrt((sv[k:] ** 2).sum()) / np.linalg.norm(sv)
        assert res <= tol, (t, s, res)
        assert res <= 20 * best, (t, s, res, best)
        checked += 1
    assert checked >= 10


def test_bad_trees_are_rejected():
    mesh = meshes.icosphere(2)
    part = structure.build_block_partition(mesh, "p0", 16, 2.0)
    ptr, idx = part.cluster_csr()
    son = part.son_array()
    bad = son.copy()
    bad[son[0, 0], 0] = 0                               # cycle back to the root
    with pytest.raises(pkg.BemError):
        pkg.bem_gca_pivots(mesh.verts, mesh.tris, "p0", ptr, idx, bad)
    bad = son.copy()
    bad[son[0, 1]] = son[0, 0], -1                     # a cluster with two parents
    with pytest.raises(pkg.BemError):
        pkg.bem_gca_pivots(mesh.verts, mesh.tris, "p0", ptr, idx, bad)
    bad_idx = idx.copy()
    bad_idx[3] = mesh.nt                                # index out of range
    with pytest.raises(pkg.BemError):
        pkg.bem_gca_pivots(mesh.verts, mesh.tris, "p0", ptr, bad_idx, son)
    with pytest.raises(pkg.BemError):
        pkg.bem_gca_pivots(mesh.verts, mesh.tris, "p0", ptr, idx, son, kappa=-1.0)

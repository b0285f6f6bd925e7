"""Pins of the oracle's H2 product and conjugate gradients (oracle/h2.py) and
of the GCA's interpolation matrices (bem_gca_bases, host code), on the CPU.

- bem_gca_bases returns the pivots of bem_gca_pivots, and each matrix
  restricted to its pivot rows is the identity (R_t V_t = I, Section 2.3).
- With every cluster's pivots equal to all its indices and identity bases,
  the H2 product is exactly the dense product (the admissible blocks are then
  the dense blocks themselves): the block bookkeeping of h2_matvec is pinned
  by the plain matrix product.
- With the GCA's bases (rank <= 16) the H2 product of the oracle's dense
  single- and double-layer matrices differs from the dense product by less
  than 1e-2 (the approximation of Section 2.4, not rounding).
- cg() solves a symmetric positive definite system to the requested residual
  and agrees with numpy's direct solve.
- The interior Dirichlet problem of Section 4 with f1 = x1^2 - x3^2 on the
  unit sphere: V a = (1/2 M + K) b has the Neumann data 2 f1 as solution; the
  error of the dense Galerkin solve falls with the mesh size (O(h)).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import h2

Q = dict(q_regular=3, q_identical=4, q_edge=4, q_vertex=4)


def _dense(mesh, kernel):
    n = mesh.nt
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    return oracle.entries(mesh.verts, mesh.tris, rows, cols, kernel=kernel, **Q).real.reshape(n, n)


def _blocks(part, G, ptr, idx, pp, pi):
    near = [(idx[ptr[t]:ptr[t + 1]], idx[ptr[s]:ptr[s + 1]],
             G[np.ix_(idx[ptr[t]:ptr[t + 1]], idx[ptr[s]:ptr[s + 1]])]) for t, s in part.near]
    far = [(t, s, G[np.ix_(pi[pp[t]:pp[t + 1]], pi[pp[s]:pp[s + 1]])]) for t, s in part.far]
    return near, far


@pytest.fixture(scope="module")
def pkg():
    from paper_1510_07244_gb300 import build as libbuild
    libbuild.build()
    import paper_1510_07244_gb300 as p
    return p


def test_gca_bases_interpolate(pkg):
    mesh = synth.jitter(synth.icosphere(3), 0.05, 41)
    for basis in ("p0", "p1"):
        part = synth.structure.build_block_partition(mesh, basis, 32, 2.0)
        ptr, idx = part.cluster_csr()
        son = part.son_array()
        pp, pi, mats = pkg.bem_gca_bases(mesh.verts, mesh.tris, basis, ptr, idx, son)
        pp2, pi2 = pkg.bem_gca_pivots(mesh.verts, mesh.tris, basis, ptr, idx, son)
        assert np.array_equal(pp, pp2) and np.array_equal(pi, pi2)
        for c in range(len(ptr) - 1):
            k = pp[c + 1] - pp[c]
            rows = (idx[ptr[c]:ptr[c + 1]] if son[c, 0] < 0 and son[c, 1] < 0 else
                    np.concatenate([pi[pp[s]:pp[s + 1]] for s in son[c] if s >= 0]))
            assert mats[c].shape == (len(rows), k)
            at = [int(np.where(rows == p)[0][0]) for p in pi[pp[c]:pp[c + 1]]]
            assert np.abs(mats[c][at] - np.eye(k)).max() < 1e-12


def test_h2_product_with_full_pivots_is_dense():
    mesh = synth.jitter(synth.icosphere(2), 0.05, 42)
    n = mesh.nt
    part = synth.structure.build_block_partition(mesh, "p0", 16, 2.0)
    ptr, idx = part.cluster_csr()
    son = part.son_array()
    assert part.far, "the partition needs admissible blocks"
    rng = np.random.default_rng(5)
    G = rng.standard_normal((n, n))
    # pivots = every index of the cluster; leaf bases I, transfer matrices the
    # permutation that takes the sons' index order to the father's
    pp = ptr.copy()
    pi = idx.copy()
    mats = []
    for c in range(len(ptr) - 1):
        own = idx[ptr[c]:ptr[c + 1]]
        if son[c, 0] < 0 and son[c, 1] < 0:
            mats.append(np.eye(len(own)))
        else:
            rows = np.concatenate([idx[ptr[s]:ptr[s + 1]] for s in son[c] if s >= 0])
            mats.append((rows[:, None] == own[None, :]).astype(float))
    bases = h2.full_bases(ptr, idx, son, pp, mats)
    near, far = _blocks(part, G, ptr, idx, pp, pi)
    x = rng.standard_normal(n)
    assert np.allclose(h2.h2_matvec(n, x, near, far, bases, pp), G @ x, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kernel", ["laplace_slp", "laplace_dlp"])
def test_h2_product_approximates_dense(pkg, kernel):
    mesh = synth.icosphere(3)
    n = mesh.nt
    part = synth.structure.build_block_partition(mesh, "p0", 32, 2.0)
    ptr, idx = part.cluster_csr()
    son = part.son_array()
    pp, pi, mats = pkg.bem_gca_bases(mesh.verts, mesh.tris, "p0", ptr, idx, son)
    bases = h2.full_bases(ptr, idx, son, pp, mats)
    G = _dense(mesh, kernel)
    near, far = _blocks(part, G, ptr, idx, pp, pi)
    rng = np.random.default_rng(6)
    for _ in range(3):
        x = rng.standard_normal(n)
        err = np.linalg.norm(h2.h2_matvec(n, x, near, far, bases, pp) - G @ x)
        assert err < 1e-2 * np.linalg.norm(G @ x)


def test_cg_solves_spd_system():
    rng = np.random.default_rng(7)
    B = rng.standard_normal((60, 60))
    A = B @ B.T + 60 * np.eye(60)
    b = rng.standard_normal(60)
    x, it, res = h2.cg(lambda v: A @ v, b, tol=1e-12)
    assert res <= 1e-12 and it <= 60
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-10 * np.abs(x).max())


def _f1_error(mesh):
    """Relative L2-type error of the Galerkin Neumann data against 2 f1 (at the
    centroids), dense solve."""
    n = mesh.nt
    v = mesh.verts[mesh.tris]
    area = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 1]), axis=1)
    c = v.mean(axis=1)
    f1 = c[:, 0] ** 2 - c[:, 2] ** 2
    V = _dense(mesh, "laplace_slp")
    K = _dense(mesh, "laplace_dlp")
    rhs = (0.5 * np.diag(area) + K) @ f1
    a = np.linalg.solve(V, rhs)
    return np.sqrt(np.sum(area * (a - 2 * f1) ** 2) / np.sum(area * (2 * f1) ** 2))


@pytest.mark.slow
def test_dirichlet_problem_converges():
    e1 = _f1_error(synth.octasphere(4))       # 128 triangles
    e2 = _f1_error(synth.octasphere(8))       # 512 triangles
    e3 = _f1_error(synth.octasphere(16))      # 2048 triangles
    assert e1 > e2 > e3
    assert e3 < 0.6 * e2 < 0.36 * e1          # at least O(h^0.7) over two refinements

"""The Green point sets on the clusters' auxiliary boxes (Section 2.3), the
inputs of the Green quadrature matrices: a tensor Gauss-Legendre rule on the
six faces of omega_t = the support box grown by delta_t / 2.  Pinned to exact
surface integrals: the area, the divergence theorem for low-degree fields,
and the distance to the supports."""
import numpy as np
import pytest

import synth
from synth.structure import build_cluster_tree, green_box_points, green_point_sets


@pytest.mark.parametrize("g", [1, 2, 3, 4, 6])
def test_box_rule_integrates_exactly(g):
    bmin = np.array([-0.3, 0.1, 0.7])
    bmax = np.array([0.4, 0.35, 1.9])
    z, n, w, delta = green_box_points(bmin, bmax, g)
    assert z.shape == (6 * g * g, 3) and n.shape == z.shape and w.shape == (6 * g * g,)
    assert delta == pytest.approx(np.linalg.norm(bmax - bmin), rel=1e-15)
    lo, hi = bmin - delta / 2, bmax + delta / 2
    L = hi - lo
    area = 2 * (L[0] * L[1] + L[1] * L[2] + L[0] * L[2])
    vol = np.prod(L)
    assert w.sum() == pytest.approx(area, rel=1e-13)
    # divergence theorem: int n = 0, int z.n = 3 V, int x_k^2 n_k = 2 V c_k
    assert np.abs((w[:, None] * n).sum(0)).max() <= 1e-13 * area
    assert (w * (z * n).sum(1)).sum() == pytest.approx(3 * vol, rel=1e-13)
    c = 0.5 * (lo + hi)
    for k in range(3):
        assert (w * z[:, k] ** 2 * n[:, k]).sum() == pytest.approx(2 * vol * c[k], rel=1e-12)
    # a field of degree 2 g - 1 along each face: int y^(2g-1) n_x over the two
    # x faces cancels; int (x y^(2g-2)) n_x = int y^(2g-2) dV
    p = 2 * g - 2
    ref = L[0] * L[2] * (hi[1] ** (p + 1) - lo[1] ** (p + 1)) / (p + 1)
    assert (w * z[:, 0] * z[:, 1] ** p * n[:, 0]).sum() == pytest.approx(ref, rel=1e-12)


def test_points_lie_on_the_grown_box_with_outward_normals():
    bmin = np.array([0.0, 0.0, 0.0])
    bmax = np.array([1.0, 2.0, 0.5])
    z, n, w, delta = green_box_points(bmin, bmax, 3)
    lo, hi = bmin - delta / 2, bmax + delta / 2
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0)
    assert (w > 0).all()
    for zz, nn in zip(z, n):
        ax = int(np.argmax(np.abs(nn)))
        assert zz[ax] == (hi[ax] if nn[ax] > 0 else lo[ax])
        assert np.all(zz >= lo - 1e-15) and np.all(zz <= hi + 1e-15)
    # every point keeps delta / 2 from the support box
    gap = np.maximum(0.0, np.maximum(bmin - z, z - bmax))
    assert np.linalg.norm(gap, axis=1).min() >= delta / 2 * (1 - 1e-14)


def test_point_sets_in_cluster_csr():
    mesh = synth.icosphere(2)
    tree = build_cluster_tree(mesh, "p1", leaf_size=32)
    clusters = [0, 3, 5]
    pt_ptr, z, nz, sp, sm = green_point_sets(tree, clusters, 2)
    assert pt_ptr.dtype == np.int32 and list(pt_ptr) == [0, 24, 48, 72]
    for k, c in enumerate(clusters):
        zc, nc, wc, delta = green_box_points(tree.bmin[c], tree.bmax[c], 2)
        sl = slice(pt_ptr[k], pt_ptr[k + 1])
        assert np.array_equal(z[sl], zc) and np.array_equal(nz[sl], nc)
        assert np.allclose(sp[sl], np.sqrt(wc), rtol=1e-15)
        assert np.allclose(sm[sl], np.sqrt(wc) * delta, rtol=1e-15)
        # the points keep delta / 2 from every support vertex of the cluster
        idx = tree.indices(c)
        tris = np.where(np.isin(mesh.tris, idx).any(axis=1))[0]
        pts = mesh.verts[np.unique(mesh.tris[tris])]
        d = np.linalg.norm(pts[None, :, :] - zc[:, None, :], axis=2)
        assert d.min() >= delta / 2 * (1 - 1e-12)

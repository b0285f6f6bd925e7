"""Green quadrature matrices A_t = (A_t+, A_t-) of Green's representation
formula (Section 2.3) on the GPU, through the C ABI, against the FP64 oracle
(oracle.green_entries, pinned in test_oracle_green.py) on the same seeded
inputs, element by element.

Tolerance: relative error <= 1e-10 per entry (FP64 on both sides; the same
rule, only the summation order differs: per-triangle partial sums on the GPU,
one running sum in the oracle).  The points stay delta_t / 2 away from the
supports, so no entry is near zero and each is measured against the largest
entry of its block only as a guard.
"""
import numpy as np
import pytest

import oracle
import synth
from synth.structure import build_cluster_tree, green_point_sets

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07244_gb300 as p
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _layout(tree, clusters, gauss_per_face):
    """Rows (cluster CSR), Green points and output offsets of the clusters."""
    row_ptr = [0]
    rows = []
    for c in clusters:
        ind = tree.indices(c)
        rows.append(ind)
        row_ptr.append(row_ptr[-1] + len(ind))
    pt_ptr, z, nz, sp, sm = green_point_sets(tree, clusters, gauss_per_face)
    sizes = [2 * (row_ptr[k + 1] - row_ptr[k]) * (pt_ptr[k + 1] - pt_ptr[k])
             for k in range(len(clusters))]
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    return (np.array(row_ptr, np.int32), np.concatenate(rows).astype(np.int32), pt_ptr, z, nz,
            sp, sm, off, int(np.sum(sizes)))


def _run(ctx, pkg, mid, lay, kernel, kappa, rule, q, unit=False, pad=0):
    import torch
    row_ptr, rows, pt_ptr, z, nz, sp, sm, off, total = lay
    cplx = kernel == "helmholtz_slp"
    out = torch.full((total + pad,), float("nan"),
                     dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    job = pkg.GreenJob(mid, _dev(row_ptr, torch.int32), _dev(rows, torch.int32),
                       _dev(pt_ptr, torch.int32), _dev(z, torch.float64),
                       _dev(nz, torch.float64), _dev(off, torch.int64), out,
                       sp=None if unit else _dev(sp, torch.float64),
                       sm=None if unit else _dev(sm, torch.float64),
                       kernel=pkg.kernel_desc(kernel, kappa), rule=rule, q=q)
    ctx.bem_green_matrices(job)
    ctx.bem_sync()
    return out.cpu().numpy()


def _oracle_blocks(mesh, basis, lay, clusters, kernel, kappa, rule, q, unit=False):
    """Per cluster: (plus, minus) as (n_c, m_c) complex arrays from the oracle."""
    row_ptr, rows, pt_ptr, z, nz, sp, sm, off, total = lay
    res = []
    for k in range(len(clusters)):
        r = rows[row_ptr[k]:row_ptr[k + 1]]
        p = np.arange(pt_ptr[k], pt_ptr[k + 1])
        if len(r) == 0 or len(p) == 0:
            res.append(None)
            continue
        ii = np.repeat(r, len(p))
        pp = np.tile(p, len(r))
        plus, minus = oracle.green_entries(mesh.verts, mesh.tris, basis, ii, z[pp], nz[pp],
                                           kappa=kappa if kernel == "helmholtz_slp" else 0.0,
                                           rule=rule, q=q)
        plus = plus.reshape(len(r), len(p))
        minus = minus.reshape(len(r), len(p))
        if not unit:
            plus = plus * sp[p][None, :]
            minus = minus * sm[p][None, :]
        res.append((plus, minus))
    return res


def _block(out, lay, k):
    row_ptr, rows, pt_ptr, z, nz, sp, sm, off, total = lay
    n = row_ptr[k + 1] - row_ptr[k]
    m = pt_ptr[k + 1] - pt_ptr[k]
    b = out[off[k]:off[k] + 2 * n * m].reshape(2 * m, n).T
    return b[:, :m], b[:, m:]


def _max_rel(got, ref):
    scale = np.abs(ref).max()
    den = np.maximum(np.abs(ref), 1e-3 * scale)
    return float((np.abs(got - ref) / den).max())


def _check(out, ref, lay, clusters, cplx):
    worst = 0.0
    for k in range(len(clusters)):
        if ref[k] is None:
            continue
        gp, gm = _block(out, lay, k)
        rp, rm = ref[k]
        if not cplx:
            assert np.all(np.abs(rp.imag) == 0) and np.all(np.abs(rm.imag) == 0)
            rp, rm = rp.real, rm.real
        worst = max(worst, _max_rel(gp, rp), _max_rel(gm, rm))
    return worst


def _mesh(basis):
    mesh = synth.jitter(synth.icosphere(2), 0.05, 151007244)
    tree = build_cluster_tree(mesh, basis, leaf_size=32)
    return mesh, tree


@pytest.mark.parametrize("basis", ["p0", "p1"])
@pytest.mark.parametrize("kernel,kappa", [("laplace_slp", 0.0), ("helmholtz_slp", 8.0)])
@pytest.mark.parametrize("rule,q,gpf", [("tri7", 0, 3), ("duffy", 3, 2), ("duffy", 5, 4)])
def test_green_matrices_match_oracle(ctx, pkg, basis, kernel, kappa, rule, q, gpf):
    """Every cluster of the tree (leaves of up to 32 rows and the large upper
    clusters, so several warps per CTA and ragged row counts; 24, 54 or 96
    points, so one ragged chunk, a full and a ragged one, or three full
    ones), every entry against the oracle."""
    mesh, tree = _mesh(basis)
    clusters = list(range(tree.n_clusters))
    lay = _layout(tree, clusters, gpf)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, basis)
    try:
        out = _run(ctx, pkg, mid, lay, kernel, kappa, rule, q)
    finally:
        ctx.bem_mesh_free(mid)
    assert not np.isnan(out).any()
    ref = _oracle_blocks(mesh, basis, lay, clusters, kernel, kappa, rule, q)
    assert _check(out, ref, lay, clusters, kernel == "helmholtz_slp") <= TOL


def test_laplace_kinds_share_the_green_function(ctx, pkg):
    """The single- and double-layer Laplace descriptors select the same Green
    function, so the matrices are identical."""
    mesh, tree = _mesh("p1")
    clusters = list(range(tree.n_clusters))
    lay = _layout(tree, clusters, 3)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p1")
    try:
        a = _run(ctx, pkg, mid, lay, "laplace_slp", 0.0, "tri7", 0)
        b = _run(ctx, pkg, mid, lay, "laplace_dlp", 3.0, "tri7", 0)
    finally:
        ctx.bem_mesh_free(mid)
    assert np.array_equal(a, b)


def test_unit_factors_empty_clusters_and_untouched_output(ctx, pkg):
    """Without sp / sm the blocks are the plain integrals; clusters with no
    rows or no points write nothing, and nothing outside the blocks is
    written (the output is NaN-filled beforehand, with spare room at the end)."""
    mesh, tree = _mesh("p0")
    leaves = [c for c in range(tree.n_clusters) if tree.is_leaf(c)][:5]
    row_ptr, rows, pt_ptr, z, nz, sp, sm, off, total = _layout(tree, leaves, 2)
    # cluster 1 keeps its rows but gets no points; cluster 3 gets no rows
    keep_pts = [np.arange(pt_ptr[k], pt_ptr[k + 1]) for k in range(len(leaves))]
    keep_pts[1] = keep_pts[1][:0]
    keep_rows = [rows[row_ptr[k]:row_ptr[k + 1]] for k in range(len(leaves))]
    keep_rows[3] = keep_rows[3][:0]
    pt_ptr = np.concatenate([[0], np.cumsum([len(p) for p in keep_pts])]).astype(np.int32)
    pts = np.concatenate(keep_pts)
    z, nz, sp, sm = z[pts], nz[pts], sp[pts], sm[pts]
    row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in keep_rows])]).astype(np.int32)
    rows = np.concatenate(keep_rows).astype(np.int32)
    sizes = [2 * (row_ptr[k + 1] - row_ptr[k]) * (pt_ptr[k + 1] - pt_ptr[k])
             for k in range(len(leaves))]
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    lay = (row_ptr, rows, pt_ptr, z, nz, sp, sm, off, int(np.sum(sizes)))
    assert sizes[1] == 0 and sizes[3] == 0
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    try:
        out = _run(ctx, pkg, mid, lay, "laplace_slp", 0.0, "tri7", 0, unit=True, pad=17)
    finally:
        ctx.bem_mesh_free(mid)
    total = lay[-1]
    assert not np.isnan(out[:total]).any()
    assert np.isnan(out[total:]).all()
    ref = _oracle_blocks(mesh, "p0", lay, leaves, "laplace_slp", 0.0, "tri7", 0, unit=True)
    assert ref[1] is None and ref[3] is None
    assert _check(out, ref, lay, leaves, False) <= TOL


def test_no_clusters_is_a_no_op(ctx, pkg):
    """An empty cluster list launches nothing and writes nothing."""
    import torch
    mesh, _ = _mesh("p0")
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    try:
        e32 = torch.zeros(1, dtype=torch.int32, device="cuda")
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        pts = torch.zeros((1, 3), dtype=torch.float64, device="cuda") + 5.0
        job = pkg.GreenJob(mid, e32, e32[:0], e32, pts, pts,
                           torch.zeros(0, dtype=torch.int64, device="cuda"), out)
        ctx.bem_green_matrices(job)
        ctx.bem_sync()
    finally:
        ctx.bem_mesh_free(mid)
    assert np.isnan(out.cpu().numpy()).all()


def test_bad_arguments_are_reported(ctx, pkg):
    """A rule outside [1, 5] is refused on the host; a row index out of range
    and a block past the end of the output are found on the device, reported
    by bem_sync, and leave only that row or that cluster unwritten."""
    import torch
    mesh, tree = _mesh("p0")
    leaves = [c for c in range(tree.n_clusters) if tree.is_leaf(c)][:3]
    lay = _layout(tree, leaves, 2)
    row_ptr, rows, pt_ptr, z, nz, sp, sm, off, total = lay
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    try:
        with pytest.raises(pkg.BemError):
            _run(ctx, pkg, mid, lay, "laplace_slp", 0.0, "duffy", 6)
        # row 0 of cluster 0 names a triangle past the end of the mesh
        bad_rows = rows.copy()
        bad_rows[0] = mesh.nt
        out = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        job = pkg.GreenJob(mid, _dev(row_ptr, torch.int32), _dev(bad_rows, torch.int32),
                           _dev(pt_ptr, torch.int32), _dev(z, torch.float64),
                           _dev(nz, torch.float64), _dev(off, torch.int64), out,
                           sp=_dev(sp, torch.float64), sm=_dev(sm, torch.float64))
        ctx.bem_green_matrices(job)
        with pytest.raises(pkg.BemError) as e:
            ctx.bem_sync()
        assert e.value.code == -1
        o = out.cpu().numpy()
        gp, gm = _block(o, lay, 0)
        assert np.isnan(gp[0]).all() and np.isnan(gm[0]).all()
        assert not np.isnan(gp[1:]).any() and not np.isnan(gm[1:]).any()
        for k in (1, 2):
            assert not np.isnan(np.concatenate(_block(o, lay, k))).any()
        # the output is one element too short for the last cluster's block
        out = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        job = pkg.GreenJob(mid, _dev(row_ptr, torch.int32), _dev(rows, torch.int32),
                           _dev(pt_ptr, torch.int32), _dev(z, torch.float64),
                           _dev(nz, torch.float64), _dev(off, torch.int64), out[:total - 1])
        ctx.bem_green_matrices(job)
        with pytest.raises(pkg.BemError):
            ctx.bem_sync()
        o = out.cpu().numpy()
        assert np.isnan(np.concatenate(_block(o, lay, 2))).all()
        assert not np.isnan(np.concatenate(_block(o, lay, 0))).any()
        assert not np.isnan(np.concatenate(_block(o, lay, 1))).any()
    finally:
        ctx.bem_mesh_free(mid)
    ctx.bem_sync()


def test_full_size_sampled(ctx, pkg):
    """The benchmark's configuration: every cluster of the 20480-triangle
    icosphere's tree (piecewise linear, leaf size 32, 4 x 4 points per face,
    Radon's 7 points per support triangle), Laplace and Helmholtz kappa = 8,
    in one launch; the oracle checks the blocks of 12 seeded clusters."""
    mesh = synth.icosphere(5)
    tree = build_cluster_tree(mesh, "p1", leaf_size=32)
    clusters = list(range(tree.n_clusters))
    lay = _layout(tree, clusters, 4)
    rng = np.random.default_rng(151007244)
    pick = sorted(set(rng.integers(0, len(clusters), 12).tolist()) | {len(clusters) - 1})
    pick = [k for k in pick if lay[0][k + 1] - lay[0][k] <= 64]
    assert pick
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p1")
    try:
        for kernel, kappa in (("laplace_slp", 0.0), ("helmholtz_slp", 8.0)):
            out = _run(ctx, pkg, mid, lay, kernel, kappa, "tri7", 0)
            assert not np.isnan(out).any()
            worst = 0.0
            for k in pick:
                one = _layout_one(lay, k)
                ref = _oracle_blocks(mesh, "p1", one, [k], kernel, kappa, "tri7", 0)
                gp, gm = _block(out, lay, k)
                rp, rm = ref[0]
                if kernel != "helmholtz_slp":
                    rp, rm = rp.real, rm.real
                worst = max(worst, _max_rel(gp, rp), _max_rel(gm, rm))
            assert worst <= TOL, (kernel, worst)
    finally:
        ctx.bem_mesh_free(mid)


def _layout_one(lay, k):
    """The layout restricted to cluster k (for the oracle)."""
    row_ptr, rows, pt_ptr, z, nz, sp, sm, off, total = lay
    r = rows[row_ptr[k]:row_ptr[k + 1]]
    p = slice(pt_ptr[k], pt_ptr[k + 1])
    m = pt_ptr[k + 1] - pt_ptr[k]
    return (np.array([0, len(r)], np.int32), r, np.array([0, m], np.int32), z[p], nz[p], sp[p],
            sm[p], np.zeros(1, np.int64), 2 * len(r) * m)


@pytest.mark.parametrize("basis,kappa", [("p0", 0.0), ("p1", 0.0), ("p0", 3.0), ("p1", 3.0)])
def test_gca_with_device_green_matrices(ctx, pkg, basis, kappa):
    """bem_gca_pivots_device (every level's A_t from the device, cross
    approximation on the host) picks the pivots of the host GCA.  The mesh is
    jittered, and on it the host pivots stay the same when every entry of A_t
    is perturbed by 1e-14 relative, so rounding differences decide nothing."""
    from synth.structure import build_block_partition
    mesh = synth.jitter(synth.icosphere(3), 0.1, 11)
    part = build_block_partition(mesh, basis, 16, 2.0)
    ptr, idx = part.cluster_csr()
    son = part.son_array()
    host = pkg.bem_gca_pivots(mesh.verts, mesh.tris, basis, ptr, idx, son, kappa=kappa,
                              gauss_per_face=3)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, basis)
    try:
        dev = ctx.bem_gca_pivots_device(mid, mesh.verts, mesh.tris, basis, ptr, idx, son,
                                        kappa=kappa, gauss_per_face=3)
    finally:
        ctx.bem_mesh_free(mid)
    assert np.array_equal(host[0], dev[0]) and np.array_equal(host[1], dev[1])


def test_gca_device_rejects_another_mesh(ctx, pkg):
    """The uploaded mesh must be the one whose host arrays are passed."""
    from synth.structure import build_block_partition
    mesh = synth.icosphere(2)
    part = build_block_partition(mesh, "p0", 16, 2.0)
    ptr, idx = part.cluster_csr()
    other = synth.icosphere(1)
    mid = ctx.bem_mesh_upload(other.verts, other.tris, "p0")
    # same counts, moved coordinates: caught by the upload's hash
    moved = synth.jitter(mesh, 0.05, 3)
    mid2 = ctx.bem_mesh_upload(moved.verts, moved.tris, "p0")
    try:
        for m in (mid, mid2):
            with pytest.raises(pkg.BemError) as e:
                ctx.bem_gca_pivots_device(m, mesh.verts, mesh.tris, "p0", ptr, idx,
                                          part.son_array())
            assert e.value.code == -1
    finally:
        ctx.bem_mesh_free(mid)
        ctx.bem_mesh_free(mid2)


@pytest.mark.parametrize("basis,kernel,kappa", [("p0", "laplace_slp", 0.0),
                                                ("p1", "helmholtz_slp", 3.0)])
def test_device_matrices_reproduce_galerkin_block(ctx, pkg, basis, kernel, kappa):
    """Section 2.3, G|t x s ~ A_t B_ts: A_t (rows of t, factors sqrt(w) and
    sqrt(w) delta_t) and B_ts (rows of s, factors sqrt(w) / delta_t and
    sqrt(w)) from bem_green_matrices give G|t x s = A_t+ b_ts+^T - A_t- b_ts-^T
    up to the error of the box rule (about 5e-7 with 12 x 12 points per face
    on this block, as the oracle's own pin finds), against the library's
    Galerkin entries with Radon's 7 points; with the minus part's sign flipped
    the error is of order 1."""
    import torch
    from synth.structure import build_block_partition, green_box_points
    mesh = synth.jitter(synth.icosphere(3), 0.05, 7)
    part = build_block_partition(mesh, basis, leaf_size=32, eta=2.0)
    tree = part.tree
    best = None
    for t, s in part.far:
        lo, hi = np.asarray(tree.bmin[t]), np.asarray(tree.bmax[t])
        d = float(np.linalg.norm(hi - lo))
        gap = np.maximum(0.0, np.maximum(lo - d / 2 - tree.bmax[s], tree.bmin[s] - hi - d / 2))
        size = min(len(tree.indices(t)), len(tree.indices(s)))
        if np.linalg.norm(gap) / d >= 0.5 and size >= 8 and (best is None or size > best[0]):
            best = (size, t, s)
    assert best is not None
    _, t, s = best
    rt, cs = tree.indices(t).astype(np.int32), tree.indices(s).astype(np.int32)
    z, nz, w, delta = green_box_points(tree.bmin[t], tree.bmax[t], 12)
    m = len(z)
    sw = np.sqrt(w)
    cplx = kernel == "helmholtz_slp"
    dt = torch.complex128 if cplx else torch.float64
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, basis)
    try:
        def green(rows, sp, sm):
            out = torch.full((2 * len(rows) * m,), float("nan"), dtype=dt, device="cuda")
            job = pkg.GreenJob(mid, _dev([0, len(rows)], torch.int32), _dev(rows, torch.int32),
                               _dev([0, m], torch.int32), _dev(z, torch.float64),
                               _dev(nz, torch.float64), _dev([0], torch.int64), out,
                               sp=_dev(sp, torch.float64), sm=_dev(sm, torch.float64),
                               kernel=pkg.kernel_desc(kernel, kappa), rule="tri7")
            ctx.bem_green_matrices(job)
            ctx.bem_sync()
            b = out.cpu().numpy().reshape(2 * m, len(rows)).T
            return b[:, :m], b[:, m:]

        a_plus, a_minus = green(rt, sw, sw * delta)
        b_minus, b_plus = green(cs, sw / delta, sw)      # plus columns hold int psi g
        rows = np.repeat(rt, len(cs)).astype(np.int32)
        cols = np.tile(cs, len(rt)).astype(np.int32)
        G = torch.full((len(rows),), float("nan"), dtype=dt, device="cuda")
        ctx.bem_pivot_entries(mid, pkg.kernel_desc(kernel, kappa),
                              pkg.quad_desc(q_regular=3, regular_rule="tri7"),
                              _dev(rows, torch.int32), _dev(cols, torch.int32), G)
        ctx.bem_sync()
    finally:
        ctx.bem_mesh_free(mid)
    G = G.cpu().numpy().reshape(len(rt), len(cs))
    approx = a_plus @ b_plus.T - a_minus @ b_minus.T
    flipped = a_plus @ b_plus.T + a_minus @ b_minus.T
    scale = np.abs(G).max()
    assert np.abs(G - approx).max() / scale < 2e-5
    assert np.abs(G - flipped).max() / scale > 0.1

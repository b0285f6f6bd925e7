"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

Tolerance: relative error <= 1e-10 per entry for the FP64 form (measured as
in parity_util.rel_err).  Both sides evaluate the same rule with the same
canonical vertex orders; only the summation order differs (warp trees and a
per-pair scaling on the GPU, plain nested sums in the oracle).
"""
import numpy as np
import pytest

import oracle
import synth
from synth.workloads import BlockSet, h2_blocks
from parity_util import (block_job, oracle_absolute, oracle_entries, rel_err, rel_err_abs,
                         to_dev)

pytestmark = pytest.mark.gpu

TOL = 1e-10
KERNELS = [("laplace_slp", 0.0), ("laplace_dlp", 0.0), ("helmholtz_slp", 4.0)]
QUADS = {"paper": dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5),
         "c1": dict(q_regular=3, regular_rule="tri7", q_identical=4, q_edge=4, q_vertex=4),
         "q4": dict(q_regular=4, regular_rule="duffy", q_identical=6, q_edge=6, q_vertex=6),
         "low": dict(q_regular=2, regular_rule="duffy", q_identical=2, q_edge=3, q_vertex=2)}


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


def _out(n, kernel):
    import torch
    dt = torch.complex128 if kernel == "helmholtz_slp" else torch.float64
    return torch.full((max(n, 1),), float("nan"), dtype=dt, device="cuda")


def _dense(ctx, pkg, mesh, basis, kernel, kappa, quad, lower=0):
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, basis)
    n = mesh.nt if basis == "p0" else mesh.nv
    out = _out(n * n, kernel)
    ctx.bem_assemble_dense(mid, pkg.kernel_desc(kernel, kappa), pkg.quad_desc(**quad), lower, out)
    ctx.bem_sync()
    ctx.bem_mesh_free(mid)
    return out.cpu().numpy()[: n * n].reshape(n, n).T, n


MESHES = {
    "octahedron": lambda: synth.octahedron(),
    "ico2": lambda: synth.jitter(synth.icosphere(2), 0.05, 11),
    "cube3": lambda: synth.jitter(synth.cube_surface(3), 0.05, 12),
    "torus": lambda: synth.jitter(synth.torus(13, 5), 0.05, 13),
}


@pytest.mark.parametrize("meshname", ["octahedron", "ico2", "cube3", "torus"])
@pytest.mark.parametrize("kernel,kappa", KERNELS)
@pytest.mark.parametrize("basis", ["p0", "p1"])
def test_dense_matches_oracle(ctx, pkg, meshname, kernel, kappa, basis):
    mesh = MESHES[meshname]()
    quad = QUADS["paper"]
    got, n = _dense(ctx, pkg, mesh, basis, kernel, kappa, quad)
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    ref = oracle_entries(mesh, basis, rows, cols, kernel, kappa, quad).reshape(n, n)
    assert np.isfinite(got).all()
    assert rel_err(got.ravel(), ref.ravel(), rows).max() <= TOL


@pytest.mark.parametrize("qname", ["c1", "q4", "low"])
@pytest.mark.parametrize("basis", ["p0", "p1"])
def test_dense_other_orders(ctx, pkg, qname, basis):
    mesh = MESHES["cube3"]()
    quad = QUADS[qname]
    for kernel, kappa in KERNELS:
        got, n = _dense(ctx, pkg, mesh, basis, kernel, kappa, quad)
        rows = np.repeat(np.arange(n), n)
        cols = np.tile(np.arange(n), n)
        ref = oracle_entries(mesh, basis, rows, cols, kernel, kappa, quad).reshape(n, n)
        assert rel_err(got.ravel(), ref.ravel(), rows).max() <= TOL, kernel


def test_dense_lower_only(ctx, pkg):
    import torch
    mesh = MESHES["ico2"]()
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    n = mesh.nt
    out = torch.full((n * n,), -7.0, dtype=torch.float64, device="cuda")
    ctx.bem_assemble_dense(mid, pkg.kernel_desc("laplace_slp"), pkg.quad_desc(**QUADS["c1"]),
                           1, out)
    ctx.bem_sync()
    full, _ = _dense(ctx, pkg, mesh, "p0", "laplace_slp", 0.0, QUADS["c1"])
    got = out.cpu().numpy().reshape(n, n).T
    il = np.tril_indices(n)
    iu = np.triu_indices(n, 1)
    assert np.array_equal(got[il], full[il])
    assert np.all(got[iu] == -7.0)


@pytest.mark.parametrize("basis", ["p0", "p1"])
@pytest.mark.parametrize("kernel,kappa", KERNELS)
def test_near_field_and_coupling(ctx, pkg, basis, kernel, kappa):
    quad = QUADS["paper"]
    if basis == "p0":
        mesh = synth.jitter(synth.icosphere(2), 0.05, 21)
        part, near, far = h2_blocks(mesh, basis, leaf_size=12, eta=1.0, rank=6, pivot_seed=5)
    else:
        mesh = synth.jitter(synth.icosphere(3), 0.05, 21)
        part, near, far = h2_blocks(mesh, basis, leaf_size=16, eta=2.0, rank=6, pivot_seed=5)
    assert len(near.blk_row) > 4 and len(far.blk_row) > 4
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, basis)
    out_n = _out(near.n_entries, kernel)
    out_f = _out(far.n_entries, kernel)
    ctx.bem_near_field([block_job(pkg, mid, near, kernel, kappa, quad, out_n)])
    ctx.bem_coupling_blocks([block_job(pkg, mid, far, kernel, kappa, quad, out_f)])
    ctx.bem_sync()
    for bs, out in ((near, out_n), (far, out_f)):
        r, c = bs.entry_indices()
        got = out.cpu().numpy()[: bs.n_entries]
        ref = oracle_entries(mesh, basis, r, c, kernel, kappa, quad)
        assert np.isfinite(got).all()
        assert rel_err(got, ref, r).max() <= TOL
    ctx.bem_mesh_free(mid)


@pytest.mark.parametrize("basis", ["p0", "p1"])
@pytest.mark.parametrize("kernel,kappa", KERNELS)
def test_pivot_entries(ctx, pkg, basis, kernel, kappa):
    import torch
    mesh = synth.jitter(synth.cube_surface(4), 0.05, 31)
    quad = QUADS["paper"]
    n = mesh.nt if basis == "p0" else mesh.nv
    rng = synth.SplitMix64(77)
    rows = rng.integers(400, n)
    cols = rng.integers(400, n)
    # include every touching configuration explicitly
    t = mesh.tris
    if basis == "p0":
        extra_r = [0, 0, 0, 1]
        extra_c = [0, 1, int(np.where((t == t[0, 0]).any(1))[0][-1]), 1]
    else:
        extra_r = [t[0, 0], t[0, 0], t[0, 1]]
        extra_c = [t[0, 0], t[0, 1], t[0, 1]]
    rows = np.concatenate([rows, extra_r]).astype(np.int32)
    cols = np.concatenate([cols, extra_c]).astype(np.int32)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, basis)
    out = _out(len(rows), kernel)
    ctx.bem_pivot_entries(mid, pkg.kernel_desc(kernel, kappa), pkg.quad_desc(**quad),
                          to_dev(rows, torch.int32), to_dev(cols, torch.int32), out)
    ctx.bem_sync()
    got = out.cpu().numpy()[: len(rows)]
    ref = oracle_entries(mesh, basis, rows, cols, kernel, kappa, quad)
    assert rel_err(got, ref, rows).max() <= TOL
    ctx.bem_mesh_free(mid)


def test_results_are_deterministic(ctx, pkg):
    mesh = synth.jitter(synth.icosphere(2), 0.05, 41)
    a, _ = _dense(ctx, pkg, mesh, "p1", "helmholtz_slp", 3.0, QUADS["paper"])
    b, _ = _dense(ctx, pkg, mesh, "p1", "helmholtz_slp", 3.0, QUADS["paper"])
    assert np.array_equal(a, b)


def test_empty_and_ragged_inputs(ctx, pkg):
    import torch
    mesh = synth.octahedron()
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    kd, qd = pkg.kernel_desc("laplace_slp"), pkg.quad_desc(**QUADS["paper"])
    # zero entries / zero blocks are no-ops
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    ctx.bem_pivot_entries(mid, kd, qd, e, e, torch.zeros(1, dtype=torch.float64, device="cuda"))
    # clusters of sizes 1, 3 and 8 (ragged tiles), a block with an empty cluster
    bs = BlockSet(np.array([0, 1, 4, 12, 12]), np.array([5, 0, 2, 7] + list(range(8))),
                  np.array([0, 1, 4, 12, 12]), np.array([5, 0, 2, 7] + list(range(8))),
                  np.array([0, 1, 2, 2, 3]), np.array([2, 1, 0, 2, 1]),
                  np.array([0, 8, 17, 25, 89]), 89)
    out = torch.full((89,), float("nan"), dtype=torch.float64, device="cuda")
    ctx.bem_near_field([block_job(pkg, mid, bs, "laplace_slp", 0.0, QUADS["paper"], out)])
    ctx.bem_sync()
    r, c = bs.entry_indices()
    ref = oracle_entries(mesh, "p0", r, c, "laplace_slp", 0.0, QUADS["paper"])
    got = out.cpu().numpy()
    assert rel_err(got, ref, r).max() <= TOL
    ctx.bem_mesh_free(mid)


def test_device_detected_errors(ctx, pkg):
    import torch
    mesh = synth.octahedron()
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    kd, qd = pkg.kernel_desc("laplace_slp"), pkg.quad_desc(**QUADS["paper"])
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    bad = torch.tensor([0, 99], dtype=torch.int32, device="cuda")
    ctx.bem_pivot_entries(mid, kd, qd, bad, bad, out)
    with pytest.raises(pkg.BemError) as ei:
        ctx.bem_sync()
    assert ei.value.code == -1
    ctx.bem_sync()   # the status word was cleared
    # a touching pair inside a coupling block is rejected
    bs = BlockSet(np.array([0, 2]), np.array([0, 1]), np.array([0, 2]), np.array([0, 1]),
                  np.array([0]), np.array([0]), np.array([0]), 4)
    ctx.bem_coupling_blocks([block_job(pkg, mid, bs, "laplace_slp", 0.0, QUADS["paper"], out)])
    with pytest.raises(pkg.BemError):
        ctx.bem_sync()
    ctx.bem_mesh_free(mid)


def test_host_detected_errors(ctx, pkg):
    mesh = synth.octahedron()
    with pytest.raises(pkg.BemError) as ei:
        bad = mesh.tris.copy()
        bad[0] = [0, 0, 1]
        ctx.bem_mesh_upload(mesh.verts, bad, "p0")
    assert ei.value.code == -5
    with pytest.raises(pkg.BemError):
        ctx.bem_mesh_upload(mesh.verts, mesh.tris + 100, "p0")
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    import torch
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.BemError) as ei:
        ctx.bem_assemble_dense(mid, pkg.kernel_desc("laplace_slp"),
                               pkg.quad_desc(q_regular=7), 0, out)
    assert ei.value.code == -6
    ctx.bem_mesh_free(mid)


def test_c2_full_size_sampled(ctx, pkg):
    """The benchmark's 20480-triangle P1 workload in its launch configuration:
    all near-field and coupling entries on the GPU, a seeded sample of each
    checked against the oracle."""
    w = synth.workloads.config2()
    quad = w.quad.kw()
    mid = ctx.bem_mesh_upload(w.mesh.verts, w.mesh.tris, w.basis)
    rng = synth.SplitMix64(99)
    for op in w.operators:
        out_n = _out(w.near.n_entries, op.kernel)
        out_f = _out(w.far.n_entries, op.kernel)
        ctx.bem_near_field([block_job(pkg, mid, w.near, op.kernel, op.kappa, quad, out_n)])
        ctx.bem_coupling_blocks([block_job(pkg, mid, w.far, op.kernel, op.kappa, quad, out_f)])
        ctx.bem_sync()
        for bs, out in ((w.near, out_n), (w.far, out_f)):
            got_all = out.cpu().numpy()[: bs.n_entries]
            assert np.isfinite(got_all).all()
            r, c = bs.entry_indices()
            pick = rng.integers(1500, bs.n_entries)
            ref = oracle_entries(w.mesh, w.basis, r[pick], c[pick], op.kernel, op.kappa, quad)
            # row scale from the full row set of the sample
            assert rel_err(got_all[pick], ref, r[pick]).max() <= TOL
    ctx.bem_mesh_free(mid)


# --------------------------------------------------------------------------
# Mixed-precision form: FP32 regular and common-vertex pairs (Laplace), FP64
# identical and common-edge pairs.  Bar: 1e-6, the tolerance of the mixed
# form, measured against the sum of term magnitudes (rel_err_abs), which is
# the plain relative error wherever the integrand has one sign.
# --------------------------------------------------------------------------
MIXED_TOL = 1e-6
LAPLACE = [("laplace_slp", 0.0), ("laplace_dlp", 0.0)]
# "mixed": FP64 identical and common-edge pairs; "mixed_full": those in FP32 too
MIXED_FORMS = ["mixed", "mixed_full"]


@pytest.mark.parametrize("form", MIXED_FORMS)
@pytest.mark.parametrize("meshname", ["ico2", "cube3", "torus"])
@pytest.mark.parametrize("kernel,kappa", LAPLACE)
@pytest.mark.parametrize("basis", ["p0", "p1"])
def test_mixed_dense_matches_oracle(ctx, pkg, meshname, kernel, kappa, basis, form):
    mesh = MESHES[meshname]()
    quad = dict(QUADS["paper"], precision=form)
    got, n = _dense(ctx, pkg, mesh, basis, kernel, kappa, quad)
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    ref = oracle_entries(mesh, basis, rows, cols, kernel, kappa, QUADS["paper"]).reshape(n, n)
    absint = oracle_absolute(mesh, basis, rows, cols, kernel, kappa, QUADS["paper"])
    err = rel_err_abs(got.ravel(), ref.ravel(), absint, rows)
    assert err.max() <= MIXED_TOL
    # the row-scaled measure too: the single layer has no cancellation, and
    # the piecewise-constant double layer has the cancellation guard
    if kernel == "laplace_slp" or basis == "p0":
        assert rel_err(got.ravel(), ref.ravel(), rows).max() <= MIXED_TOL
    # and it is not the FP64 result in disguise
    assert err.max() > 1e-12


@pytest.mark.parametrize("form", MIXED_FORMS)
@pytest.mark.parametrize("basis", ["p0", "p1"])
@pytest.mark.parametrize("kernel,kappa", LAPLACE)
def test_mixed_near_field_and_coupling(ctx, pkg, basis, kernel, kappa, form):
    quad = dict(QUADS["paper"], precision=form)
    mesh = synth.jitter(synth.icosphere(3), 0.05, 23)
    part, near, far = h2_blocks(mesh, basis, leaf_size=16, eta=2.0, rank=6, pivot_seed=7)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, basis)
    out_n = _out(near.n_entries, kernel)
    out_f = _out(far.n_entries, kernel)
    ctx.bem_near_field([block_job(pkg, mid, near, kernel, kappa, quad, out_n)])
    ctx.bem_coupling_blocks([block_job(pkg, mid, far, kernel, kappa, quad, out_f)])
    ctx.bem_sync()
    for bs, out in ((near, out_n), (far, out_f)):
        r, c = bs.entry_indices()
        got = out.cpu().numpy()[: bs.n_entries]
        ref = oracle_entries(mesh, basis, r, c, kernel, kappa, QUADS["paper"])
        absint = oracle_absolute(mesh, basis, r, c, kernel, kappa, QUADS["paper"])
        assert rel_err_abs(got, ref, absint, r).max() <= MIXED_TOL
        if kernel == "laplace_slp" or basis == "p0":
            assert rel_err(got, ref.real, r).max() <= MIXED_TOL
    ctx.bem_mesh_free(mid)


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_cancellation_guard_row_scaled(ctx, pkg, form):
    """Jittered flat faces make many double-layer pairs straddle each other's
    planes.  With the guard the float forms meet the row-scaled bar on every
    near-field and coupling entry, through the per-call entry points and
    through a plan (batched, CUDA graph), and they agree bit for bit."""
    import torch
    quad = dict(QUADS["paper"], precision=form)
    mesh = synth.jitter(synth.cube_surface(8), 0.05, 29)
    part, near, far = h2_blocks(mesh, "p0", leaf_size=32, eta=2.0, rank=8, pivot_seed=5)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    outs = {nm: (_out(bs.n_entries, "laplace_dlp"), _out(bs.n_entries, "laplace_dlp"))
            for nm, bs in (("near", near), ("far", far))}
    ctx.bem_near_field([block_job(pkg, mid, near, "laplace_dlp", 0.0, quad, outs["near"][0])])
    ctx.bem_coupling_blocks([block_job(pkg, mid, far, "laplace_dlp", 0.0, quad, outs["far"][0])])
    plan = ctx.bem_plan_create([block_job(pkg, mid, near, "laplace_dlp", 0.0, quad, outs["near"][1])],
                               [block_job(pkg, mid, far, "laplace_dlp", 0.0, quad, outs["far"][1])],
                               pkg.PLAN_GRAPH)
    ctx.bem_plan_run(plan)
    ctx.bem_plan_run(plan)          # a second replay starts from clean guard state
    ctx.bem_sync()
    stats = ctx.bem_plan_guard_stats(plan)
    ctx.bem_plan_destroy(plan)
    assert stats["recomputed"] > 0 and stats["recomputed"] < stats["entries"] // 16
    for nm, bs in (("near", near), ("far", far)):
        r, c = bs.entry_indices()
        ref = oracle_entries(mesh, "p0", r, c, "laplace_dlp", 0.0, QUADS["paper"])
        a = outs[nm][0].cpu().numpy()[: bs.n_entries]
        b = outs[nm][1].cpu().numpy()[: bs.n_entries]
        assert np.array_equal(a, b), nm
        assert rel_err(a, ref, r).max() <= MIXED_TOL, nm
    ctx.bem_mesh_free(mid)


@pytest.mark.parametrize("kernel", ["laplace_slp", "laplace_dlp"])
def test_coupling_engine_ragged_and_errors(ctx, pkg, kernel):
    """Piecewise-linear coupling blocks of the mixed form (one entry per lane,
    16 x 2 warp tiles): pivot sets of 1, 3, 17 (two row tiles) and 0 entries,
    against the oracle; a touching pair or an index out of range sets the
    status word and zeroes the entry."""
    import torch
    mesh = synth.jitter(synth.icosphere(3), 0.05, 29)
    quad = dict(QUADS["paper"], precision="mixed_full")
    rng = synth.SplitMix64(3)
    # four clusters of far-apart vertices: around the poles +-z and +-x
    v = mesh.verts
    groups = [np.where(v[:, 2] > 0.97)[0][:1], np.where(v[:, 2] < -0.9)[0][:3],
              np.where(v[:, 0] > 0.7)[0][:17], np.zeros(0, np.int64)]
    ptr = np.concatenate([[0], np.cumsum([len(g) for g in groups])])
    idx = np.concatenate(groups)
    pairs = [(0, 1), (1, 0), (2, 1), (1, 2), (0, 2), (2, 3), (3, 0)]
    sizes = [len(groups[a]) * len(groups[b]) for a, b in pairs]
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    bs = BlockSet(ptr, idx, ptr, idx, np.array([p[0] for p in pairs]),
                  np.array([p[1] for p in pairs]), off, int(sum(sizes)))
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p1")
    out = torch.full((bs.n_entries,), float("nan"), dtype=torch.float64, device="cuda")
    ctx.bem_coupling_blocks([block_job(pkg, mid, bs, kernel, 0.0, quad, out)])
    ctx.bem_sync()
    r, c = bs.entry_indices()
    ref = oracle_entries(mesh, "p1", r, c, kernel, 0.0, QUADS["paper"])
    absint = oracle_absolute(mesh, "p1", r, c, kernel, 0.0, QUADS["paper"])
    got = out.cpu().numpy()
    assert rel_err_abs(got, ref, absint, r).max() <= MIXED_TOL
    # a block whose supports touch (vertex 0 against its neighbour) is not admissible
    nb = int(mesh.tris[np.where((mesh.tris == 0).any(axis=1))[0][0]][1:].max())
    for pair in ([0, nb], [0, mesh.nv + 5]):
        bad = BlockSet(np.array([0, 1, 2]), np.array(pair), np.array([0, 1, 2]), np.array(pair),
                       np.array([0]), np.array([1]), np.array([0]), 1)
        one = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.bem_coupling_blocks([block_job(pkg, mid, bad, kernel, 0.0, quad, one)])
        with pytest.raises(pkg.BemError) as ei:
            ctx.bem_sync()
        assert ei.value.code == -1
        assert one.item() == 0.0
    ctx.bem_mesh_free(mid)


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_mixed_translated_far_from_origin(ctx, pkg, form):
    """The double-float anchors keep the mixed form accurate when the mesh sits
    far from the origin (coordinates ~1e3, triangles ~0.1)."""
    mesh = MESHES["cube3"]()
    moved = synth.Mesh(mesh.verts + np.array([1e3, -7e2, 3e2]), mesh.tris)
    quad = dict(QUADS["paper"], precision=form)
    for kernel in ("laplace_slp", "laplace_dlp"):
        got, n = _dense(ctx, pkg, moved, "p1", kernel, 0.0, quad)
        rows = np.repeat(np.arange(n), n)
        cols = np.tile(np.arange(n), n)
        ref = oracle_entries(mesh, "p1", rows, cols, kernel, 0.0, QUADS["paper"]).reshape(n, n)
        absint = oracle_absolute(mesh, "p1", rows, cols, kernel, 0.0, QUADS["paper"])
        assert rel_err_abs(got.ravel(), ref.ravel(), absint, rows).max() <= MIXED_TOL, kernel


def test_mixed_full_size_against_fp64(ctx, pkg):
    """Every entry of the 20480-triangle P1 workload: both mixed forms vs FP64 form."""
    w = synth.workloads.config2()
    mid = ctx.bem_mesh_upload(w.mesh.verts, w.mesh.tris, w.basis)
    q64 = w.quad.kw()
    for op in w.operators:
        res = {}
        for name, q in [("fp64", q64)] + [(f, dict(q64, precision=f)) for f in MIXED_FORMS]:
            out_n = _out(w.near.n_entries, op.kernel)
            out_f = _out(w.far.n_entries, op.kernel)
            ctx.bem_near_field([block_job(pkg, mid, w.near, op.kernel, op.kappa, q, out_n)])
            ctx.bem_coupling_blocks([block_job(pkg, mid, w.far, op.kernel, op.kappa, q, out_f)])
            ctx.bem_sync()
            res[name] = (out_n.cpu().numpy(), out_f.cpu().numpy())
        for k, bs in enumerate((w.near, w.far)):
            r, _ = bs.entry_indices()
            for f in MIXED_FORMS:
                err = rel_err(res[f][k], res["fp64"][k], r)
                assert err.max() <= MIXED_TOL, (op.kernel, f, k, err.max())
    ctx.bem_mesh_free(mid)


@pytest.mark.parametrize("form", MIXED_FORMS)
@pytest.mark.parametrize("meshname,kappa", [("cube3", 4.0), ("torus", 8.0), ("ico2", 16.0)])
def test_mixed_helmholtz_p0(ctx, pkg, meshname, kappa, form):
    """Mixed Helmholtz (P0): FP32 disjoint and common-vertex pairs with the
    double-float reference phase; within 1e-6 of the oracle."""
    mesh = MESHES[meshname]()
    quad = dict(QUADS["paper"], precision=form)
    got, n = _dense(ctx, pkg, mesh, "p0", "helmholtz_slp", kappa, quad)
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    ref = oracle_entries(mesh, "p0", rows, cols, "helmholtz_slp", kappa, QUADS["paper"]).reshape(n, n)
    absint = oracle_absolute(mesh, "p0", rows, cols, "helmholtz_slp", kappa, QUADS["paper"])
    err = rel_err_abs(got.ravel(), ref.ravel(), absint, rows)
    assert 1e-12 < err.max() <= MIXED_TOL


def test_mixed_helmholtz_far_phase(ctx, pkg):
    """kappa = 16 on a 2048-triangle sphere: far pairs with kappa r up to 32."""
    mesh = synth.jitter(synth.octasphere(16), 0.05, 77)
    quad = dict(QUADS["paper"], precision="mixed")
    got, n = _dense(ctx, pkg, mesh, "p0", "helmholtz_slp", 16.0, quad)
    rng = synth.SplitMix64(5)
    rows = rng.integers(3000, n)
    cols = rng.integers(3000, n)
    ref = oracle_entries(mesh, "p0", rows, cols, "helmholtz_slp", 16.0, QUADS["paper"])
    absint = oracle_absolute(mesh, "p0", rows, cols, "helmholtz_slp", 16.0, QUADS["paper"])
    assert rel_err_abs(got[rows, cols], ref, absint, rows).max() <= MIXED_TOL


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_c3_full_size_sampled(ctx, pkg, form):
    """The 49152-triangle jittered cube, Helmholtz kappa = 8, both float forms:
    all near-field and coupling blocks on the GPU, whole sampled blocks checked
    against the FP64 oracle (the error of the float forms on this workload)."""
    from parity_util import sample_block_entries
    w = synth.workloads.config3()
    op = w.operators[0]
    q = w.quad.kw()
    mid = ctx.bem_mesh_upload(w.mesh.verts, w.mesh.tris, w.basis)
    rng = synth.SplitMix64(31)
    for bs, call in ((w.near, ctx.bem_near_field), (w.far, ctx.bem_coupling_blocks)):
        out = _out(bs.n_entries, op.kernel)
        call([block_job(pkg, mid, bs, op.kernel, op.kappa, dict(q, precision=form), out)])
        ctx.bem_sync()
        got_all = out.cpu().numpy()
        assert np.isfinite(got_all).all()
        pos = sample_block_entries(bs, 8, rng)
        r, c = bs.entry_indices()
        ref = oracle_entries(w.mesh, "p0", r[pos], c[pos], op.kernel, op.kappa, q)
        A = oracle_absolute(w.mesh, "p0", r[pos], c[pos], op.kernel, op.kappa, q)
        assert rel_err_abs(got_all[pos], ref, A, r[pos]).max() <= MIXED_TOL
    ctx.bem_mesh_free(mid)

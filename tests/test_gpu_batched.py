"""Persistent batched driver (bem_plan_*): one launch per kernel bucket over
many meshes and kernels, optionally captured in a CUDA graph and autotuned.
Its results must equal those of the per-job calls bit for bit (the same tile
bodies run in both), and sampled entries must match the oracle."""
import numpy as np
import pytest

import synth
from parity_util import block_job, oracle_entries, rel_err, sample_block_entries

pytestmark = pytest.mark.gpu

QUAD = dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07244_gb300 as pkg
    ctx = pkg.Context(0)
    yield pkg, ctx
    ctx.close()


@pytest.fixture(scope="module")
def small_batch():
    return synth.workloads.config4(count=6, lo=200.0, hi=1200.0, leaf_size=16, eta=2.0, rank=6)


def _jobs(pkg, ctx, w, precision):
    import torch
    mids, near, far, outs = [], [], [], []
    q = dict(QUAD, precision=precision)
    for it in w.items:
        mid = ctx.bem_mesh_upload(it.mesh.verts, it.mesh.tris, w.basis)
        mids.append(mid)
        for op in it.operators:
            dt = torch.complex128 if op.kernel == "helmholtz_slp" else torch.float64
            on = torch.full((max(1, it.near.n_entries),), float("nan"), dtype=dt, device="cuda")
            of = torch.full((max(1, it.far.n_entries),), float("nan"), dtype=dt, device="cuda")
            near.append(block_job(pkg, mid, it.near, op.kernel, op.kappa, q, on))
            far.append(block_job(pkg, mid, it.far, op.kernel, op.kappa, q, of))
            outs.append((it, op, on, of))
    return mids, near, far, outs


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_full"])
@pytest.mark.parametrize("flags", [0, 1, 3, 7, 9, 11])
def test_plan_equals_per_job_calls(env, small_batch, precision, flags):
    pkg, ctx = env
    mids, near, far, outs = _jobs(pkg, ctx, small_batch, precision)
    for j in near:
        ctx.bem_near_field([j])
    for j in far:
        ctx.bem_coupling_blocks([j])
    ctx.bem_sync()
    ref = [(on.clone(), of.clone()) for _, _, on, of in outs]
    for _, _, on, of in outs:
        on.fill_(float("nan"))
        of.fill_(float("nan"))
    plan = ctx.bem_plan_create(near, far, flags)
    ctx.bem_plan_run(plan)
    ctx.bem_plan_run(plan)
    ctx.bem_sync()
    info = ctx.bem_plan_info(plan)
    # one launch per (kernel, precision) bucket: far fewer than one per job
    assert info["block_launches"] <= 2 < len(near) + len(far)
    for (r_on, r_of), (_, _, on, of) in zip(ref, outs):
        assert torch_equal(on, r_on) and torch_equal(of, r_of)
    ctx.bem_plan_destroy(plan)
    for m in mids:
        ctx.bem_mesh_free(m)


def torch_equal(a, b):
    import torch
    return bool(torch.equal(a, b))


def test_plan_matches_oracle(env, small_batch):
    pkg, ctx = env
    mids, near, far, outs = _jobs(pkg, ctx, small_batch, "fp64")
    plan = ctx.bem_plan_create(near, far, 3)
    ctx.bem_plan_run(plan)
    ctx.bem_sync()
    rng = synth.SplitMix64(17)
    for it, op, on, of in outs:
        for bs, out in ((it.near, on), (it.far, of)):
            if bs.n_entries == 0:
                continue
            r, c = bs.entry_indices()
            pick = sample_block_entries(bs, 12, rng)
            got = out.cpu().numpy()[pick]
            ref = oracle_entries(it.mesh, "p0", r[pick], c[pick], op.kernel, op.kappa, QUAD)
            assert rel_err(got, ref, r[pick]).max() <= 1e-10
    ctx.bem_plan_destroy(plan)
    for m in mids:
        ctx.bem_mesh_free(m)


@pytest.mark.parametrize("precision,leaf", [("fp64", 16), ("mixed_full", 16), ("mixed_full", 64)])
def test_plan_p1_and_profile(env, precision, leaf):
    """Piecewise-linear jobs of two meshes in one plan; the launch profile
    counts every bucket launch of every run.  In the mixed form the coupling
    jobs run in their own bucket (coupling engine).  The plan's near-field
    tiles read support records built once per run (clusters of up to 64
    indices: several 32-index slices each), the per-job calls build them per
    tile: the results agree bit for bit."""
    import torch
    pkg, ctx = env
    quad = dict(QUAD, precision=precision)
    jobs_n, jobs_f, outs, mids = [], [], [], []
    for lv, seed in ((2, 3), (3, 4)):
        mesh = synth.jitter(synth.icosphere(lv), 0.05, seed)
        _, near, far = synth.workloads.h2_blocks(mesh, "p1", leaf, 2.0, 6, seed)
        mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p1")
        mids.append(mid)
        for kernel in ("laplace_slp", "laplace_dlp"):
            on = torch.zeros(max(1, near.n_entries), dtype=torch.float64, device="cuda")
            of = torch.zeros(max(1, far.n_entries), dtype=torch.float64, device="cuda")
            jobs_n.append(block_job(pkg, mid, near, kernel, 0.0, quad, on))
            jobs_f.append(block_job(pkg, mid, far, kernel, 0.0, quad, of))
            outs.append((on, of))
    for j in jobs_n:
        ctx.bem_near_field([j])
    for j in jobs_f:
        ctx.bem_coupling_blocks([j])
    ctx.bem_sync()
    ref = [(a.clone(), b.clone()) for a, b in outs]
    plan = ctx.bem_plan_create(jobs_n, jobs_f, 7)
    ctx.bem_profile_reset()
    ctx.bem_profile_enable(True)
    for _ in range(3):
        ctx.bem_plan_run(plan)
    prof = ctx.bem_profile_read()
    ctx.bem_profile_enable(False)
    for (ra, rb), (a, b) in zip(ref, outs):
        assert torch.equal(a, ra) and torch.equal(b, rb)
    info = ctx.bem_plan_info(plan)
    engines = [k for k in ("block_p1", "coupling_p1") if k in prof]
    assert "block_p1" in engines and (precision != "fp64" or len(engines) == 1)
    assert sum(prof[k][0] for k in engines) == 3 * info["block_launches"]
    assert info["block_launches"] == len(engines) * 2      # per engine: SLP and DLP buckets
    # one support build per distinct cluster list (rows = columns here) per run
    # (jobs without blocks need none)
    tables = info["aux_launches"] // 2 - info["block_launches"]
    assert 2 <= tables <= len(jobs_n) + len(jobs_f)
    assert prof["supports"][0] == 3 * tables
    assert all(v[1] > 0 for v in prof.values())
    ctx.bem_plan_destroy(plan)
    for m in mids:
        ctx.bem_mesh_free(m)


def test_shards_reproduce_unsharded_run(env):
    """Multi-GPU sharding rehearsed on one GPU: the block lists cut into three
    cost-balanced shards, run one after another into one output, give the
    unsharded FP64 result bit for bit (whole blocks, no exchange)."""
    import torch
    import bench
    from synth.workloads import BlockSet
    pkg, ctx = env
    w = synth.workloads.config2(levels=3)
    mid = ctx.bem_mesh_upload(w.mesh.verts, w.mesh.tris, w.basis)
    for bs, call in ((w.near, ctx.bem_near_field), (w.far, ctx.bem_coupling_blocks)):
        full = torch.zeros(bs.n_entries, dtype=torch.float64, device="cuda")
        call([block_job(pkg, mid, bs, "laplace_dlp", 0.0, QUAD, full)])
        sharded = torch.zeros_like(full)
        bounds = pkg.bem_shard_blocks(bench.block_costs(bs), 3)
        for k in range(3):
            lo, hi = int(bounds[k]), int(bounds[k + 1])
            part = BlockSet(bs.row_ptr, bs.row_idx, bs.col_ptr, bs.col_idx, bs.blk_row[lo:hi],
                            bs.blk_col[lo:hi], bs.blk_off[lo:hi], bs.n_entries)
            if hi > lo:
                call([block_job(pkg, mid, part, "laplace_dlp", 0.0, QUAD, sharded)])
        ctx.bem_sync()
        assert torch.equal(full, sharded)
    ctx.bem_mesh_free(mid)


def test_plan_rejects_learned_orders_without_model(env, small_batch):
    """A learned-order job needs an order model: without one the plan is
    refused, not silently evaluated at the fixed orders."""
    pkg, ctx = env
    ctx.bem_set_order_model(None, 0.0)
    mids, near, far, outs = _jobs(pkg, ctx, small_batch, "mixed_full")
    near[0].quad = pkg.quad_desc(**QUAD, precision="mixed_full", order_mode="learned")
    with pytest.raises(pkg.BemError) as ei:
        ctx.bem_plan_create(near, far, 0)
    assert ei.value.code == -1
    for m in mids:
        ctx.bem_mesh_free(m)


def test_plan_fuses_single_and_double_layer(env):
    """Jobs of both layers over the same device block arrays run fused (near
    field: one tile engine launch; coupling: one coupling launch), sharing the
    distances, and give the per-job results bit for bit."""
    import torch
    from parity_util import oracle_absolute, rel_err_abs, to_dev
    pkg, ctx = env
    mesh = synth.jitter(synth.icosphere(3), 0.05, 5)
    _, near, far = synth.workloads.h2_blocks(mesh, "p1", 16, 2.0, 6, 5)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p1")
    quad = dict(QUAD, precision="mixed_full")
    jobs = {"near": [], "far": []}
    outs = []
    for name, bs in (("near", near), ("far", far)):
        arr = [to_dev(a, torch.int32) for a in (bs.row_ptr, bs.row_idx, bs.blk_row, bs.blk_col)]
        off = to_dev(bs.blk_off, torch.int64)
        for kernel in ("laplace_slp", "laplace_dlp"):
            o = torch.full((bs.n_entries,), float("nan"), dtype=torch.float64, device="cuda")
            jobs[name].append(pkg.BlockJob(mid, arr[0], arr[1], arr[0], arr[1], arr[2], arr[3], off,
                                           o, pkg.kernel_desc(kernel), pkg.quad_desc(**quad)))
            outs.append((name, kernel, bs, o))
    ctx.bem_near_field(jobs["near"])
    ctx.bem_coupling_blocks(jobs["far"])
    ctx.bem_sync()
    ref = [o.clone() for *_, o in outs]
    for *_, o in outs:
        o.fill_(float("nan"))
    plan = ctx.bem_plan_create(jobs["near"], jobs["far"], pkg.PLAN_GRAPH | pkg.PLAN_PROFILE)
    ctx.bem_profile_reset()
    ctx.bem_profile_enable(True)
    ctx.bem_plan_run(plan)
    prof = ctx.bem_profile_read()
    ctx.bem_profile_enable(False)
    assert ctx.bem_plan_info(plan)["block_launches"] == 2
    assert prof["coupling_p1"][0] == 1 and prof["block_p1"][0] == 1
    for (name, kernel, bs, o), r in zip(outs, ref):
        assert torch.equal(o, r), (name, kernel)
        rows, cols = bs.entry_indices()
        want = oracle_entries(mesh, "p1", rows, cols, kernel, 0.0, QUAD)
        A = oracle_absolute(mesh, "p1", rows, cols, kernel, 0.0, QUAD)
        assert rel_err_abs(o.cpu().numpy(), want, A, rows).max() <= 1e-6, (name, kernel)
    ctx.bem_plan_destroy(plan)
    ctx.bem_mesh_free(mid)


def test_static_plan_skips_list_passes(env):
    """BEM_PLAN_STATIC_LISTS: the support records and prefix sums are built once
    at creation; the runs issue only the quadrature and guard passes, with the
    same results bit for bit (P1, fused layers, near field and coupling)."""
    import torch
    from parity_util import to_dev
    pkg, ctx = env
    mesh = synth.jitter(synth.icosphere(3), 0.05, 6)
    _, near, far = synth.workloads.h2_blocks(mesh, "p1", 16, 2.0, 6, 5)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p1")
    quad = dict(QUAD, precision="mixed_full")
    res = {}
    for flags in (pkg.PLAN_GRAPH | pkg.PLAN_PROFILE,
                  pkg.PLAN_GRAPH | pkg.PLAN_PROFILE | pkg.PLAN_STATIC_LISTS):
        jobs = {"near": [], "far": []}
        outs = []
        for name, bs in (("near", near), ("far", far)):
            arr = [to_dev(a, torch.int32) for a in (bs.row_ptr, bs.row_idx, bs.blk_row, bs.blk_col)]
            off = to_dev(bs.blk_off, torch.int64)
            for kernel in ("laplace_slp", "laplace_dlp"):
                o = torch.full((bs.n_entries,), float("nan"), dtype=torch.float64, device="cuda")
                jobs[name].append(pkg.BlockJob(mid, arr[0], arr[1], arr[0], arr[1], arr[2], arr[3],
                                               off, o, pkg.kernel_desc(kernel), pkg.quad_desc(**quad)))
                outs.append(o)
        plan = ctx.bem_plan_create(jobs["near"], jobs["far"], flags)
        for o in outs:
            o.fill_(float("nan"))
        ctx.bem_profile_reset()
        ctx.bem_profile_enable(True)
        ctx.bem_plan_run(plan)
        ctx.bem_plan_run(plan)
        prof = ctx.bem_profile_read()
        ctx.bem_profile_enable(False)
        ctx.bem_sync()
        res[flags] = ([o.cpu() for o in outs], prof, ctx.bem_plan_info(plan)["aux_launches"])
        ctx.bem_plan_destroy(plan)
    (a, pa, na), (b, pb, nb) = res.values()
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    assert "supports" in pa and "tile_prefix" in pa
    assert "supports" not in pb and "tile_prefix" not in pb
    assert nb < na
    ctx.bem_mesh_free(mid)

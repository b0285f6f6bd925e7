"""The allocation-free near-field entry point (bem_near_field_noalloc).

It serves callers that cannot allocate device memory (their device memory is
owned by a pool allocator, or they cannot afford the device synchronisation an
allocation may cause): the same kernels as bem_near_field, scratch in a static
device array.  Its output must agree with bem_near_field within the parity
tolerance of the other GPU tests, on two calls in a row (the static array
keeps the previous call's contents), including a list of exactly 65536 blocks
(every tile prefix slot of the array in use); once the touching pass and its
kernels are warm, further calls leave the device's free memory unchanged.
This file is collected last so that a run stopping at the first failure has
run every other test already; it also passes when run alone in a fresh
process.
"""
import numpy as np
import pytest

import synth
from synth.workloads import BlockSet, h2_blocks
from parity_util import block_job, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10
QUAD = dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07244_gb300 as pkg
    ctx = pkg.Context(0)
    yield pkg, ctx
    ctx.close()


@pytest.mark.parametrize("basis,kernel,kappa", [("p0", "laplace_slp", 0.0),
                                                ("p1", "laplace_dlp", 0.0),
                                                ("p1", "helmholtz_slp", 3.0)])
def test_noalloc_matches_near_field_twice(setup, basis, kernel, kappa):
    import torch
    pkg, ctx = setup
    mesh = synth.jitter(synth.icosphere(3), 0.05, 61)
    _, near, _ = h2_blocks(mesh, basis, leaf_size=16, eta=2.0, rank=4, pivot_seed=1)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, basis)
    dt = torch.complex128 if kernel == "helmholtz_slp" else torch.float64
    ref = torch.full((near.n_entries,), float("nan"), dtype=dt, device="cuda")
    ctx.bem_near_field([block_job(pkg, mid, near, kernel, kappa, QUAD, ref)])
    ctx.bem_sync()
    ref_h = ref.cpu().numpy()
    rows, _ = near.entry_indices()
    for _ in range(2):
        out = torch.full((near.n_entries,), float("nan"), dtype=dt, device="cuda")
        ctx.bem_near_field_noalloc(block_job(pkg, mid, near, kernel, kappa, QUAD, out))
        ctx.bem_sync()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_err(got, ref_h, rows).max() <= TOL
    ctx.bem_mesh_free(mid)


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    import torch
    pkg, ctx = setup
    mesh = synth.octahedron()
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    _, near, _ = h2_blocks(mesh, "p0", leaf_size=4, eta=2.0, rank=2, pivot_seed=1)
    out = torch.zeros(max(near.n_entries, 1), dtype=torch.float64, device="cuda")
    too_high = dict(QUAD, q_identical=7)
    with pytest.raises(pkg.BemError) as ei:
        ctx.bem_near_field_noalloc(block_job(pkg, mid, near, "laplace_slp", 0.0, too_high, out))
    assert ei.value.code == -1 and "static scratch" in str(ei.value)
    ctx.bem_mesh_free(mid)


def _one_triangle_blocks(nt, n_blocks):
    """P0 blocks of one triangle each: block k pairs triangle k mod nt with a
    seeded partner (identical, touching and disjoint pairs all occur)."""
    ptr = np.arange(nt + 1, dtype=np.int32)
    idx = np.arange(nt, dtype=np.int32)
    k = np.arange(n_blocks, dtype=np.int64)
    rows = (k % nt).astype(np.int32)
    cols = ((k // nt) * 37 + k * 5 + synth.SplitMix64(3).integers(n_blocks, 3)) % nt
    return BlockSet(ptr, idx, ptr, idx, rows, cols.astype(np.int32), k, n_blocks)


def test_noalloc_at_its_block_limit_allocates_nothing(setup):
    import torch
    pkg, ctx = setup
    mesh = synth.jitter(synth.icosphere(3), 0.05, 62)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    bs = _one_triangle_blocks(mesh.nt, 65536)
    ref = torch.full((bs.n_entries,), float("nan"), dtype=torch.float64, device="cuda")
    ctx.bem_near_field([block_job(pkg, mid, bs, "laplace_slp", 0.0, QUAD, ref)])
    ctx.bem_sync()
    ref_h = ref.cpu().numpy()
    rows = bs.blk_row
    outs = [torch.full((bs.n_entries,), float("nan"), dtype=torch.float64, device="cuda")
            for _ in range(3)]
    jobs = [block_job(pkg, mid, bs, "laplace_slp", 0.0, QUAD, o) for o in outs]
    ctx.bem_near_field_noalloc(jobs[0])          # warm: set-up and kernel loading
    ctx.bem_sync()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for j in jobs[1:]:
        ctx.bem_near_field_noalloc(j)
    ctx.bem_sync()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0
    for o in outs:
        got = o.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_err(got, ref_h, rows).max() <= TOL
    # one block more than the array holds is refused before anything runs
    over = _one_triangle_blocks(mesh.nt, 65537)
    big = torch.zeros(over.n_entries, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.BemError) as ei:
        ctx.bem_near_field_noalloc(block_job(pkg, mid, over, "laplace_slp", 0.0, QUAD, big))
    assert ei.value.code == -1 and "65536 blocks" in str(ei.value)
    ctx.bem_mesh_free(mid)

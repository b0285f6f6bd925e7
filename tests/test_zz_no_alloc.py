"""The allocation-free near-field entry point (bem_near_field_noalloc).

It serves callers that cannot allocate device memory (their device memory is
owned by a pool allocator, or they cannot afford the device synchronisation an
allocation may cause): the same kernels as bem_near_field, scratch in a static
device array.  Its output must agree with bem_near_field within the parity
tolerance of the other GPU tests, on two calls in a row (the static array
keeps the previous call's contents).  This file is collected last so that a
run stopping at the first failure has run every other test already; it also
passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import synth
from synth.workloads import h2_blocks
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

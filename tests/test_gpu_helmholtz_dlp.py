"""GPU parity of the Helmholtz double layer and the Brakhage-Werner combination
(Section 4's exterior problem: K - i eta V) against the oracle.

BEM_HELMHOLTZ_DLP is compared with the oracle's Helmholtz double layer entry
by entry; BEM_HELMHOLTZ_BW with the oracle's K - i eta V, which is its
definition.  Both kernels run in FP64 in every precision: a float-form request
gives the FP64 result bit for bit.
"""
import numpy as np
import pytest

import synth
from synth.workloads import h2_blocks
from parity_util import block_job, oracle_entries, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-10
Q = dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)
KAPPA, ETA = 3.0, 3.0


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


def _oracle(mesh, basis, rows, cols, kernel):
    if kernel == "helmholtz_dlp":
        return oracle_entries(mesh, basis, rows, cols, "helmholtz_dlp", KAPPA, Q)
    K = oracle_entries(mesh, basis, rows, cols, "helmholtz_dlp", KAPPA, Q)
    V = oracle_entries(mesh, basis, rows, cols, "helmholtz_slp", KAPPA, Q)
    return K - 1j * ETA * V


@pytest.mark.parametrize("basis", ["p0", "p1"])
@pytest.mark.parametrize("kernel", ["helmholtz_dlp", "helmholtz_bw"])
def test_dense_matches_oracle(env, basis, kernel):
    import torch
    pkg, ctx = env
    mesh = synth.jitter(synth.icosphere(2 if basis == "p0" else 1), 0.05, 81)
    n = mesh.nt if basis == "p0" else mesh.nv
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, basis)
    out = torch.full((n * n,), complex("nan"), dtype=torch.complex128, device="cuda")
    ctx.bem_assemble_dense(mid, pkg.kernel_desc(kernel, KAPPA, ETA), pkg.quad_desc(**Q), 0, out)
    ctx.bem_sync()
    got = out.cpu().numpy().reshape(n, n).T
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    ref = _oracle(mesh, basis, rows, cols, kernel).reshape(n, n)
    assert rel_err(got.ravel(), ref.ravel(), rows).max() <= TOL
    ctx.bem_mesh_free(mid)


@pytest.mark.parametrize("kernel", ["helmholtz_dlp", "helmholtz_bw"])
def test_near_coupling_plan_and_pivots(env, kernel):
    """Near field and coupling blocks (per call and in a plan, a float-form
    request included) and arbitrary pivot entries."""
    import torch
    pkg, ctx = env
    mesh = synth.jitter(synth.icosphere(3), 0.05, 82)
    _, near, far = h2_blocks(mesh, "p0", 16, 2.0, 6, 3)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    res = {}
    for how in ("calls", "plan"):
        outs = {}
        for nm, bs in (("near", near), ("far", far)):
            outs[nm] = torch.full((bs.n_entries,), complex("nan"), dtype=torch.complex128,
                                  device="cuda")
        q = Q if how == "calls" else dict(Q, precision="mixed_full")
        jn = block_job(pkg, mid, near, kernel, KAPPA, q, outs["near"])
        jf = block_job(pkg, mid, far, kernel, KAPPA, q, outs["far"])
        for j in (jn, jf):
            j.kernel = pkg.kernel_desc(kernel, KAPPA, ETA)
        if how == "calls":
            ctx.bem_near_field([jn])
            ctx.bem_coupling_blocks([jf])
        else:
            plan = ctx.bem_plan_create([jn], [jf], pkg.PLAN_GRAPH)
            ctx.bem_plan_run(plan)
            ctx.bem_sync()
            ctx.bem_plan_destroy(plan)
        ctx.bem_sync()
        res[how] = {k: v.cpu() for k, v in outs.items()}
    for nm, bs in (("near", near), ("far", far)):
        assert torch.equal(res["calls"][nm], res["plan"][nm]), nm
        r, c = bs.entry_indices()
        ref = _oracle(mesh, "p0", r, c, kernel)
        assert rel_err(res["calls"][nm].numpy(), ref, r).max() <= TOL, nm
    # pivot entries, touching pairs included
    rng = np.random.default_rng(8)
    rows = rng.integers(0, mesh.nt, 300).astype(np.int32)
    cols = rng.integers(0, mesh.nt, 300).astype(np.int32)
    cols[:20] = rows[:20]
    out = torch.empty(300, dtype=torch.complex128, device="cuda")
    ctx.bem_pivot_entries(mid, pkg.kernel_desc(kernel, KAPPA, ETA), pkg.quad_desc(**Q),
                          to_dev(rows, torch.int32), to_dev(cols, torch.int32), out)
    ctx.bem_sync()
    ref = _oracle(mesh, "p0", rows, cols, kernel)
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL * np.abs(ref).max()
    ctx.bem_mesh_free(mid)


def test_new_kinds_reject_learned_orders(env):
    import torch
    pkg, ctx = env
    mesh = synth.octahedron()
    _, near, _ = h2_blocks(mesh, "p0", 4, 2.0, 2, 1)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    out = torch.zeros(max(1, near.n_entries), dtype=torch.complex128, device="cuda")
    j = block_job(pkg, mid, near, "helmholtz_dlp", KAPPA, dict(Q, order_mode="learned"), out)
    with pytest.raises(pkg.BemError) as ei:
        ctx.bem_near_field([j])
    assert ei.value.code == -6
    ctx.bem_mesh_free(mid)

"""GPU: the H2 matrix-vector product and conjugate gradients (bem_h2_*) against
the oracle's plain definitions (oracle/h2.py) on the same blocks, and the
interior Dirichlet problem of Section 4 solved through them.

- The product matches the oracle's H2 product of the same near-field and
  coupling entries (copied back from the device) and the same bases to 1e-12
  relative, and repeats bit for bit.
- Conjugate gradients reach the requested residual and agree with the
  oracle's conjugate gradients on the same operator.
- With f1 = x1^2 - x3^2 on the paper's octahedral spheres, V a = (1/2 M + K) b
  (near field and coupling blocks from the library, GCA bases) gives Neumann
  data whose error against 2 f1 falls with the mesh size.
"""
import numpy as np
import pytest

import synth
from oracle import h2 as oh2
from parity_util import block_job, to_dev

pytestmark = pytest.mark.gpu

FP64 = dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)


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


def _h2_operator(pkg, ctx, mesh, kernel, leaf=32, diag=None, bases=None, rank=16, eps=1e-6):
    """Near and coupling blocks of one kernel on the GPU, the GCA bases on the
    host (at most `rank` pivots per cluster, cross-approximation tolerance
    eps), and the H2 handle over them."""
    import torch
    part = synth.structure.build_block_partition(mesh, "p0", leaf, 2.0)
    ptr, idx = part.cluster_csr()
    son = part.son_array()
    if bases is None:
        bases = pkg.bem_gca_bases(mesh.verts, mesh.tris, "p0", ptr, idx, son, eps=eps,
                                  max_rank=rank)
    pp, pi, mats = bases
    nr, nc, no, ntot = part.near_blocks()
    fr, fc, fo, ftot = synth.structure.coupling_blocks(part, pp)
    near = synth.workloads.BlockSet(ptr, idx, ptr, idx, nr, nc, no, ntot)
    far = synth.workloads.BlockSet(pp, pi, pp, pi, fr, fc, fo, ftot)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    nv = torch.zeros(max(1, ntot), dtype=torch.float64, device="cuda")
    fv = torch.zeros(max(1, ftot), dtype=torch.float64, device="cuda")
    ctx.bem_near_field([block_job(pkg, mid, near, kernel, 0.0, FP64, nv)])
    if len(fr):
        ctx.bem_coupling_blocks([block_job(pkg, mid, far, kernel, 0.0, FP64, fv)])
    ctx.bem_sync()
    ctx.bem_mesh_free(mid)
    h = ctx.bem_h2_create(mesh.nt, ptr, idx, son, pp, pi, mats, (nr, nc, no), nv, (fr, fc, fo),
                          fv, diag=diag)
    return dict(h=h, nv=nv, fv=fv, part=part, ptr=ptr, idx=idx, son=son, pp=pp, pi=pi,
                mats=mats, near=(nr, nc, no), far=(fr, fc, fo), bases=bases)


def _oracle_blocks(op):
    nvh = op["nv"].cpu().numpy()
    fvh = op["fv"].cpu().numpy()
    ptr, idx, pp, pi = op["ptr"], op["idx"], op["pp"], op["pi"]
    near = []
    for t, s, o in zip(*op["near"]):
        rt, rs = idx[ptr[t]:ptr[t + 1]], idx[ptr[s]:ptr[s + 1]]
        near.append((rt, rs, nvh[o:o + len(rt) * len(rs)].reshape(len(rs), len(rt)).T))
    far = []
    for t, s, o in zip(*op["far"]):
        kt, ks = pp[t + 1] - pp[t], pp[s + 1] - pp[s]
        far.append((t, s, fvh[o:o + kt * ks].reshape(ks, kt).T))
    bases = oh2.full_bases(ptr, idx, op["son"], pp, op["mats"])
    return near, far, bases


@pytest.mark.parametrize("kernel", ["laplace_slp", "laplace_dlp"])
def test_h2_matvec_matches_oracle(env, kernel):
    import torch
    pkg, ctx = env
    mesh = synth.jitter(synth.icosphere(3), 0.05, 71)
    n = mesh.nt
    diag = np.linspace(0.5, 1.5, n) if kernel == "laplace_dlp" else None
    op = _h2_operator(pkg, ctx, mesh, kernel, diag=diag)
    near, far, bases = _oracle_blocks(op)
    rng = np.random.default_rng(3)
    for _ in range(2):
        x = rng.standard_normal(n)
        xd = to_dev(x, torch.float64)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        y2 = torch.empty_like(y)
        ctx.bem_h2_matvec(op["h"], xd, y)
        ctx.bem_h2_matvec(op["h"], xd, y2)
        ctx.bem_sync()
        ref = oh2.h2_matvec(n, x, near, far, bases, op["pp"])
        if diag is not None:
            ref = ref + diag * x
        got = y.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        assert torch.equal(y, y2)
    ctx.bem_h2_destroy(op["h"])


def test_h2_cg_matches_oracle(env):
    import torch
    pkg, ctx = env
    mesh = synth.jitter(synth.icosphere(3), 0.05, 72)
    n = mesh.nt
    op = _h2_operator(pkg, ctx, mesh, "laplace_slp")
    near, far, bases = _oracle_blocks(op)
    b = np.random.default_rng(4).standard_normal(n)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    it, res = ctx.bem_h2_cg(op["h"], to_dev(b, torch.float64), x, tol=1e-10, maxit=500)
    ctx.bem_sync()
    assert res <= 1e-10 and 0 < it < 500
    xo, ito, reso = oh2.cg(lambda v: oh2.h2_matvec(n, v, near, far, bases, op["pp"]), b,
                           tol=1e-10)
    assert abs(it - ito) <= 2
    got = x.cpu().numpy()
    assert np.abs(got - xo).max() <= 1e-8 * np.abs(xo).max()
    ctx.bem_h2_destroy(op["h"])


def test_h2_rejects_bad_input(env):
    import torch
    pkg, ctx = env
    mesh = synth.octahedron()
    part = synth.structure.build_block_partition(mesh, "p0", 4, 2.0)
    ptr, idx = part.cluster_csr()
    son = part.son_array()
    pp, pi, mats = pkg.bem_gca_bases(mesh.verts, mesh.tris, "p0", ptr, idx, son)
    v = torch.zeros(64, dtype=torch.float64, device="cuda")
    bad = [np.zeros((1, 1))] * len(mats)          # basis matrices of the wrong shape
    with pytest.raises(pkg.BemError):
        ctx.bem_h2_create(mesh.nt, ptr, idx, son, pp, pi, bad, part.near_blocks()[:3], v,
                          ([], [], []), v)


def _neumann_error(pkg, ctx, k):
    """The Galerkin Neumann data of f1 on the octahedral sphere with 8 k^2
    triangles, solved by H2 conjugate gradients; relative error vs 2 f1.  The
    GCA keeps up to 32 pivots per cluster at tolerance 1e-8: as the paper
    notes (Section 4), the compression must become more accurate as the mesh
    is refined, and 16 pivots no longer keep the H2 error below the
    discretisation error of the 8192-triangle sphere."""
    import torch
    mesh = synth.octasphere(k)
    n = mesh.nt
    v = mesh.verts[mesh.tris]
    area = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 1]), axis=1)
    c = v.mean(axis=1)
    f1 = c[:, 0] ** 2 - c[:, 2] ** 2
    V = _h2_operator(pkg, ctx, mesh, "laplace_slp", rank=32, eps=1e-8)
    K = _h2_operator(pkg, ctx, mesh, "laplace_dlp", diag=0.5 * area, bases=V["bases"])
    rhs = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.bem_h2_matvec(K["h"], to_dev(f1, torch.float64), rhs)
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    it, res = ctx.bem_h2_cg(V["h"], rhs, a, tol=1e-8, maxit=2000)
    ctx.bem_sync()
    assert res <= 1e-8
    an = a.cpu().numpy()
    ctx.bem_h2_destroy(V["h"])
    ctx.bem_h2_destroy(K["h"])
    return np.sqrt(np.sum(area * (an - 2 * f1) ** 2) / np.sum(area * (2 * f1) ** 2)), it


def test_dirichlet_problem_by_h2_cg_converges(env):
    pkg, ctx = env
    errs = [_neumann_error(pkg, ctx, k)[0] for k in (8, 16, 32)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.6 * errs[1] < 0.36 * errs[0]

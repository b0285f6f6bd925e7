"""GPU: the exterior Helmholtz problem of Section 4 in the Brakhage-Werner form.

- bem_potentials against plain numpy tensor Gauss of the same integrands
  (points off the surface: smooth integrands) for every kernel kind.
- bem_dense_gmres against numpy's direct solve of the same complex system.
- The exterior Dirichlet problem with f(x) = g(x, (0, 0, 0.2)) (kappa = 3):
  (1/2 M + K - i eta V) w = F on the paper's octahedral spheres, the field
  u = (W - i eta S) w at exterior points against f itself; the error falls
  under refinement.
"""
import numpy as np
import pytest

import synth
from parity_util import to_dev

pytestmark = pytest.mark.gpu

KAPPA, ETA = 3.0, 3.0
Z0 = np.array([0.0, 0.0, 0.2])


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


def _green(z, y, kappa):
    r = np.linalg.norm(z - y, axis=-1)
    return np.exp(1j * kappa * r) / (4 * np.pi * r)


def _plain_potential(mesh, w, z, kind, q=12):
    """numpy tensor Gauss (Duffy square, q x q) of sum_j w_j int_Tj k(z, y) dy."""
    g, gw = np.polynomial.legendre.leggauss(q)
    g, gw = (g + 1) / 2, gw / 2
    S, T = np.meshgrid(g, g, indexing="ij")
    W = (np.outer(gw, gw) * S).ravel()
    s, t = S.ravel(), (S * T).ravel()
    v = mesh.verts[mesh.tris]
    e1, e2 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 1]
    cr = np.cross(e1, e2)
    sg = np.linalg.norm(cr, axis=1)
    n = cr / sg[:, None]
    Y = v[:, None, 0] + s[None, :, None] * e1[:, None] + t[None, :, None] * e2[:, None]
    out = np.zeros(len(z), complex)
    for k, zk in enumerate(z):
        d = zk - Y
        r = np.linalg.norm(d, axis=2)
        kr = KAPPA * r
        if kind == "laplace_slp":
            f = 1 / r
        elif kind == "laplace_dlp":
            f = np.einsum("jpc,jc->jp", d, n) / r ** 3
        elif kind == "helmholtz_slp":
            f = np.exp(1j * kr) / r
        else:
            f = np.einsum("jpc,jc->jp", d, n) * (1 - 1j * kr) * np.exp(1j * kr) / r ** 3
            if kind == "helmholtz_bw":
                f = f - 1j * ETA * np.exp(1j * kr) / r
        out[k] = np.sum(w * sg * (f @ W)) / (4 * np.pi)
    return out


@pytest.mark.parametrize("kind", ["laplace_slp", "laplace_dlp", "helmholtz_slp", "helmholtz_dlp",
                                  "helmholtz_bw"])
def test_potentials_match_plain_gauss(env, kind):
    import torch
    pkg, ctx = env
    mesh = synth.jitter(synth.icosphere(2), 0.05, 91)
    rng = np.random.default_rng(1)
    w = rng.standard_normal(mesh.nt) + 1j * rng.standard_normal(mesh.nt)
    d = rng.standard_normal((37, 3))
    z = d / np.linalg.norm(d, axis=1)[:, None] * rng.uniform(1.6, 3.0, 37)[:, None]
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    out = torch.empty(37, dtype=torch.complex128, device="cuda")
    ctx.bem_potentials(mid, pkg.kernel_desc(kind, KAPPA, ETA), to_dev(z, torch.float64),
                       to_dev(w, torch.complex128), out, q=5)
    ctx.bem_sync()
    got = out.cpu().numpy()
    ref = _plain_potential(mesh, w, z, kind, q=5)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    ctx.bem_mesh_free(mid)


def test_gmres_matches_direct_solve(env):
    import torch
    pkg, ctx = env
    rng = np.random.default_rng(2)
    n = 300
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A / np.sqrt(n) + 3 * np.eye(n)
    d = 0.5 + 0.1j * rng.standard_normal(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = torch.empty(n, dtype=torch.complex128, device="cuda")
    it, res = ctx.bem_dense_gmres(to_dev(A.T.ravel(), torch.complex128), to_dev(b, torch.complex128),
                                  x, diag=to_dev(d, torch.complex128), tol=1e-12, restart=20)
    ctx.bem_sync()
    ref = np.linalg.solve(A + np.diag(d), b)
    assert res <= 1e-12 and it > 20           # restarted at least once
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


def _exterior_error(pkg, ctx, k):
    """Brakhage-Werner solve on the octahedral sphere with 8 k^2 triangles;
    relative max error of u at exterior points against f."""
    import torch
    mesh = synth.octasphere(k)
    n = mesh.nt
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    quad = pkg.quad_desc(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)
    A = torch.empty(n * n, dtype=torch.complex128, device="cuda")
    ctx.bem_assemble_dense(mid, pkg.kernel_desc("helmholtz_bw", KAPPA, ETA), quad, 0, A)
    v = mesh.verts[mesh.tris]
    area = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 1]), axis=1)
    # F_i = int_Ti f = int_Ti g(x, z0) dx: the Green matrix entry of the point z0
    rows = torch.arange(n, dtype=torch.int32, device="cuda")
    F = torch.empty(2 * n, dtype=torch.complex128, device="cuda")
    job = pkg.GreenJob(mid, to_dev(np.array([0, n]), torch.int32), rows,
                       to_dev(np.array([0, 1]), torch.int32), to_dev(Z0[None, :], torch.float64),
                       to_dev(np.array([[0.0, 0.0, 1.0]]), torch.float64),
                       to_dev(np.array([0]), torch.int64), F,
                       kernel=pkg.kernel_desc("helmholtz_slp", KAPPA), rule="duffy", q=5)
    ctx.bem_green_matrices(job)
    w = torch.empty(n, dtype=torch.complex128, device="cuda")
    it, res = ctx.bem_dense_gmres(A, F[:n].contiguous(), w,
                                  diag=to_dev(0.5 * area + 0j, torch.complex128), tol=1e-10,
                                  restart=100)
    assert res <= 1e-10
    rng = np.random.default_rng(3)
    d = rng.standard_normal((24, 3))
    z = d / np.linalg.norm(d, axis=1)[:, None] * rng.uniform(1.5, 3.0, 24)[:, None]
    u = torch.empty(24, dtype=torch.complex128, device="cuda")
    ctx.bem_potentials(mid, pkg.kernel_desc("helmholtz_bw", KAPPA, ETA), to_dev(z, torch.float64),
                       w, u, q=5)
    ctx.bem_sync()
    f = _green(z, Z0, KAPPA)
    ctx.bem_mesh_free(mid)
    return np.abs(u.cpu().numpy() - f).max() / np.abs(f).max(), it


def test_exterior_problem_converges(env):
    pkg, ctx = env
    errs = [_exterior_error(pkg, ctx, k)[0] for k in (8, 16, 32)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.5 * errs[0]
    assert errs[2] < 2e-2

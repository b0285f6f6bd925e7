"""The library against the stored oracle values of tests/golden/oracle_entries.txt
(no oracle call at run time): FP64 form at 1e-10, float forms at 1e-6, relative to
max(|g|, 1e-3 max |g| of the group)."""
import numpy as np
import pytest

from test_golden import golden_mesh, read_entries

pytestmark = pytest.mark.gpu

QUAD = dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07244_gb300 as p
    return p


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6), ("mixed_full", 1e-6)])
def test_library_matches_stored_oracle_values(pkg, precision, tol):
    import torch
    ctx = pkg.Context(0)
    for (name, basis, kernel, kappa), rows in read_entries().items():
        if precision != "fp64" and kernel == "helmholtz_slp" and basis == "p1":
            continue
        m = golden_mesh(name)
        n = m.nt if basis == "p0" else m.nv
        mid = ctx.bem_mesh_upload(m.verts, m.tris, basis)
        dt = torch.complex128 if kernel == "helmholtz_slp" else torch.float64
        out = torch.full((n * n,), float("nan"), dtype=dt, device="cuda")
        ctx.bem_assemble_dense(mid, pkg.kernel_desc(kernel, kappa),
                               pkg.quad_desc(**QUAD, precision=precision), 0, out)
        ctx.bem_sync()
        G = out.cpu().numpy().reshape(n, n).T          # column-major -> [row, col]
        want = np.array([x[2] for x in rows])
        got = np.array([G[x[0], x[1]] for x in rows])
        scale = np.maximum(np.abs(want), 1e-3 * np.abs(want).max())
        assert (np.abs(got - want) / scale).max() <= tol, (name, basis, kernel, precision)
        ctx.bem_mesh_free(mid)
    ctx.close()

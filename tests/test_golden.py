"""Stored fixtures (tests/golden/): the paper's mesh family and the oracle's
regression values.  Host only."""
import os

import numpy as np

from synth import meshes

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_sizes():
    vals = []
    for line in open(os.path.join(GOLDEN, "paper_sphere_sizes.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            vals.append(int(line))
    return vals


def read_entries():
    groups = {}
    for line in open(os.path.join(GOLDEN, "oracle_entries.txt")):
        if line.startswith("#"):
            continue
        name, basis, kernel, kappa, r, c, re, im = line.split()
        key = (name, basis, kernel, float(kappa))
        groups.setdefault(key, []).append((int(r), int(c), float(re) + 1j * float(im)))
    return groups


def golden_mesh(name):
    if name == "octahedron":
        return meshes.octahedron()
    return meshes.jitter(meshes.icosphere(1), 0.05, 151007244)


def test_paper_sphere_family():
    """The octahedral sphere generator yields the DoF counts of Section 4's tables:
    8 n^2 triangles for n = 16, 32, ..., 512, closed (Euler characteristic 2), on
    the unit sphere."""
    sizes = read_sizes()
    assert len(sizes) == 6
    for k, dofs in enumerate(sizes):
        n = 16 * 2 ** k
        assert 8 * n * n == dofs
    for n in (16, 32):
        m = meshes.octasphere(n)
        assert m.nt == sizes[n // 32]
        assert np.allclose(np.linalg.norm(m.verts, axis=1), 1.0, atol=1e-14)
        edges = {tuple(sorted((int(t[a]), int(t[(a + 1) % 3])))) for t in m.tris for a in range(3)}
        assert m.nv - len(edges) + m.nt == 2


def test_oracle_reproduces_its_stored_values(oracle_mod):
    quad = dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)
    for (name, basis, kernel, kappa), rows in read_entries().items():
        m = golden_mesh(name)
        r = np.array([x[0] for x in rows])
        c = np.array([x[1] for x in rows])
        want = np.array([x[2] for x in rows])
        got = oracle_mod.entries(m.verts, m.tris, r, c, kernel=kernel, kappa=kappa, basis=basis,
                                 **quad)
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max(), (name, basis, kernel)

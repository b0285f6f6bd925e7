"""Writes oracle_entries.txt: Galerkin entries computed by the oracle alone, for
small seeded meshes, as regression values for the oracle (CPU test) and as
expected values for the library that need no oracle at run time (GPU test).

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import meshes  # noqa: E402

QUAD = dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)
CASES = [
    # (mesh name, basis, kernel, kappa)
    ("octahedron", "p0", "laplace_slp", 0.0),
    ("octahedron", "p0", "laplace_dlp", 0.0),
    ("icosphere1_jitter", "p1", "laplace_slp", 0.0),
    ("icosphere1_jitter", "p1", "laplace_dlp", 0.0),
    ("icosphere1_jitter", "p0", "helmholtz_slp", 2.0),
]


def mesh(name):
    if name == "octahedron":
        return meshes.octahedron()
    return meshes.jitter(meshes.icosphere(1), 0.05, 151007244)


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_entries.txt")
    with open(out, "w") as f:
        f.write("# Galerkin entries g_ij of the oracle (oracle/bem_oracle.c), written by\n")
        f.write("# tests/golden/make_golden.py; quadrature: Duffy q=3 for disjoint pairs,\n")
        f.write("# Sauter-Schwab q=5 for touching pairs (Section 2.2).\n")
        f.write("# mesh basis kernel kappa row col re im\n")
        for name, basis, kernel, kappa in CASES:
            m = mesh(name)
            n = m.nt if basis == "p0" else m.nv
            rng = np.random.default_rng(7)
            if n <= 8:
                rows, cols = np.repeat(np.arange(n), n), np.tile(np.arange(n), n)
            else:
                rows, cols = rng.integers(0, n, 24), rng.integers(0, n, 24)
                rows[:4] = cols[:4] = np.arange(4)          # some diagonal entries too
            z = oracle.entries(m.verts, m.tris, rows, cols, kernel=kernel, kappa=kappa,
                               basis=basis, **QUAD)
            for r, c, v in zip(rows, cols, z):
                f.write(f"{name} {basis} {kernel} {kappa:g} {r} {c} {v.real:.17e} {v.imag:.17e}\n")
    print(out)


if __name__ == "__main__":
    main()

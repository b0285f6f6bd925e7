"""The host case test of mesh upload (bem_touching_pairs): touching pairs,
their case and the vertex orders the Sauter-Schwab maps use (Section 2.2),
against the oracle's classification of every pair by brute force, and the
pair counts against closed forms in the vertex degrees."""
import numpy as np
import pytest

import oracle
import paper_1510_07244_gb300 as pkg
import synth.meshes as sm

CASE_ID = {"vertex": 1, "edge": 2, "identical": 3}


def _variants(m, seed):
    """The mesh, with every triangle's vertices rotated and the vertices
    relabelled, and with shuffled triangles of which some are reversed."""
    rng = np.random.default_rng(seed)
    t = np.stack([np.roll(row, k) for row, k in zip(m.tris, rng.integers(0, 3, m.nt))])
    relabel = rng.permutation(m.nv)[t]
    shuffled = t[rng.permutation(m.nt)].copy()
    flip = rng.random(m.nt) < 0.3
    shuffled[flip] = shuffled[flip][:, ::-1]
    return [m.tris, relabel, shuffled]


def _fin():
    # three triangles on one edge, a fan continuing from one of them, an
    # isolated triangle: not a manifold, every case still defined
    return np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4], [2, 5, 6], [7, 8, 9], [0, 2, 3]]), 10


SMALL = [("icosphere2", sm.icosphere(2)), ("cube4", sm.cube_surface(4)),
         ("torus", sm.torus(12, 6)), ("octasphere4", sm.octasphere(4))]


def _brute_force(tris):
    nt = len(tris)
    out = []
    for a in range(nt):
        share = np.isin(tris, tris[a]).any(axis=1)
        for b in np.nonzero(share)[0]:
            case, oa, ob = oracle.classify_orders(tris[a], tris[b])
            assert case != "regular"
            out.append((a, int(b), CASE_ID[case], *oa, *ob))
    return np.array(out, np.int64)


@pytest.mark.parametrize("name,mesh", SMALL, ids=[n for n, _ in SMALL])
def test_pairs_match_oracle_classification(name, mesh):
    for k, tris in enumerate(_variants(mesh, 11)):
        got = pkg.bem_touching_pairs(tris, mesh.nv)
        lib = np.column_stack([got["src"], got["dst"], got["case"], got["ord"]]).astype(np.int64)
        want = _brute_force(np.asarray(tris))
        assert lib.shape == want.shape, (name, k)
        assert np.array_equal(lib, want), (name, k)


def test_non_manifold_and_isolated_triangles():
    tris, nv = _fin()
    got = pkg.bem_touching_pairs(tris, nv)
    lib = np.column_stack([got["src"], got["dst"], got["case"], got["ord"]]).astype(np.int64)
    assert np.array_equal(lib, _brute_force(tris))
    # the isolated triangle 4 touches only itself
    assert list(got["dst"][got["src"] == 4]) == [4]


def test_orders_put_shared_vertices_first():
    m = sm.icosphere(3)
    tris = _variants(m, 5)[2]
    got = pkg.bem_touching_pairs(tris, m.nv)
    A = tris[got["src"][:, None], got["ord"][:, :3]]
    B = tris[got["dst"][:, None], got["ord"][:, 3:]]
    for c in (1, 2, 3):
        sel = got["case"] == c
        # the c shared vertices occupy positions 0 .. c-1 on both sides
        assert np.array_equal(A[sel, :c], B[sel, :c])
        # and no other vertex of a is one of b's (row by row)
        assert not (A[sel, c:, None] == B[sel, None, :]).any()
    # a's order is always a rotation of its own (orientation kept); so is b's,
    # except for a common edge, which b takes in the direction it has in a
    def rotation(o):
        return (o[:, 1] == (o[:, 0] + 1) % 3) & (o[:, 2] == (o[:, 0] + 2) % 3)
    assert rotation(got["ord"][:, :3]).all()
    assert rotation(got["ord"][got["case"] != 2, 3:]).all()
    # on a consistently oriented mesh every common edge runs the other way in b
    g = pkg.bem_touching_pairs(m.tris, m.nv)
    assert not rotation(g["ord"][g["case"] == 2, 3:]).any()


def test_counts_from_vertex_degrees():
    """On a closed manifold mesh: nt identical pairs, 3 nt ordered common-edge
    pairs, and sum_v deg(v) (deg(v) - 1) - 2 (3 nt) common-vertex pairs."""
    for m in (sm.icosphere(5), sm.cube_surface(24), sm.torus(40, 12)):
        got = pkg.bem_touching_pairs(m.tris, m.nv)
        deg = np.bincount(m.tris.ravel(), minlength=m.nv)
        n = np.bincount(got["case"], minlength=4)
        assert n[3] == m.nt and n[2] == 3 * m.nt
        assert n[1] == int(np.sum(deg * (deg - 1))) - 6 * m.nt
        # ascending (a, b)
        key = got["src"].astype(np.int64) * m.nt + got["dst"]
        assert np.all(np.diff(key) > 0)


def test_icosphere_20480_counts():
    # the 20480-triangle sphere: 20480 / 61440 / 184260 ordered pairs per case
    m = sm.icosphere(5)
    n = np.bincount(pkg.bem_touching_pairs(m.tris, m.nv)["case"], minlength=4)
    assert list(n[1:]) == [184260, 61440, 20480]


def test_bad_meshes_are_rejected():
    with pytest.raises(pkg.BemError) as e:
        pkg.bem_touching_pairs(np.array([[0, 1, 2], [2, 1, 0]]), 3)   # same three vertices
    assert e.value.code == -5
    with pytest.raises(pkg.BemError) as e:
        pkg.bem_touching_pairs(np.array([[0, 1, 1]]), 3)             # repeated vertex
    assert e.value.code == -5
    with pytest.raises(pkg.BemError) as e:
        pkg.bem_touching_pairs(np.array([[0, 1, 3]]), 3)             # index out of range
    assert e.value.code == -1


def _fan_reference(tris, nv):
    """Every touching pair in ascending (a, b), found through the vertex fans
    and classified by the oracle (for meshes too large for _brute_force)."""
    fans = [[] for _ in range(nv)]
    for t, row in enumerate(tris):
        for v in row:
            fans[v].append(t)
    out = []
    for a, row in enumerate(tris):
        for b in sorted(set(fans[row[0]]) | set(fans[row[1]]) | set(fans[row[2]])):
            case, oa, ob = oracle.classify_orders(row, tris[b])
            out.append((a, b, CASE_ID[case], *oa, *ob))
    return np.array(out, np.int64)


def test_large_mesh_split_over_host_threads():
    """5120 triangles are planned in contiguous triangle ranges on host
    threads; shuffled and relabelled variants put neighbours in other ranges.
    The joined result equals the oracle's classification of every pair."""
    m = sm.icosphere(4)
    for k, tris in enumerate(_variants(m, 5)):
        tris = np.asarray(tris)
        got = pkg.bem_touching_pairs(tris, m.nv)
        lib = np.column_stack([got["src"], got["dst"], got["case"], got["ord"]]).astype(np.int64)
        want = _fan_reference(tris, m.nv)
        assert np.array_equal(lib, want), k


def test_duplicate_found_in_any_range():
    """Two triangles with the same vertices at the end of a large mesh (both
    in the last host range) are rejected like the small case."""
    m = sm.icosphere(4)
    tris = np.vstack([m.tris, m.tris[-1][::-1]])
    with pytest.raises(pkg.BemError) as e:
        pkg.bem_touching_pairs(tris, m.nv)
    assert e.value.code == -5


def test_duplicate_vertex_finder_against_brute_force(tmp_path):
    """The upload's test for two vertex indices with equal coordinates (a
    hash of the exact triples) agrees with a pairwise comparison on seeded
    random vertex sets with planted duplicates and signed zeros
    (tests/dup_vertex_check.cpp, built here with the host compiler)."""
    import os
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_1510_07244_gb300", "csrc")
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.exists("/usr/local/cuda/include/cuda_runtime.h"):
        pytest.skip("no host C++ compiler or CUDA headers")
    exe = str(tmp_path / "dup_vertex_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(root, "include"), "-I", csrc,
                    "-I", "/usr/local/cuda/include", os.path.join(root, "tests", "dup_vertex_check.cpp"),
                    os.path.join(csrc, "bem_mesh_plan.cpp"), os.path.join(csrc, "bem_rules.cpp"),
                    "-o", exe, "-lpthread"], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr

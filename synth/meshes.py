"""Seeded flat-triangle surface meshes (vertices float64 (nv,3), triangles int32 (nt,3)).

Every closed mesh is outward oriented: for a triangle (v0, v1, v2) the normal
(v1-v0) x (v2-v1) points out of the enclosed volume, and each undirected edge
is shared by exactly two triangles that traverse it in opposite directions.

Recipes (all distances in the mesh's own units):
  icosphere(k)     icosahedron, k times 4-fold midpoint refinement, every new
                   vertex projected to the unit sphere: 20*4^k triangles.
  octasphere(n)    the double pyramid |x|_1 = 1, each face split regularly
                   into n^2 triangles, vertices projected to the unit sphere
                   (the paper's test surface): 8*n^2 triangles.
  cube_surface(n)  surface of [0,1]^3, n x n squares per face, each square
                   split along one fixed diagonal: 12*n^2 triangles.
  torus(nu, nv)    major radius R, minor radius r, nu x nv quad grid, each
                   quad split in two: 2*nu*nv triangles.
  jitter(mesh, f)  adds i.i.d. uniform noise in [-f*h, f*h] to every
                   coordinate, h = mean edge length before the jitter.
"""
from dataclasses import dataclass
import itertools
import numpy as np

from .rng import SplitMix64


@dataclass
class Mesh:
    verts: np.ndarray   # (nv, 3) float64
    tris: np.ndarray    # (nt, 3) int32
    name: str = ""

    @property
    def nv(self):
        return int(self.verts.shape[0])

    @property
    def nt(self):
        return int(self.tris.shape[0])


def _orient_outward(verts, tris, center_fn):
    v = verts[tris]
    n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 1])
    c = v.mean(axis=1)
    flip = np.einsum("ij,ij->i", n, c - center_fn(c)) < 0
    tris = tris.copy()
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def mean_edge_length(mesh: Mesh) -> float:
    v = mesh.verts[mesh.tris]
    e = np.concatenate([v[:, 1] - v[:, 0], v[:, 2] - v[:, 1], v[:, 0] - v[:, 2]])
    return float(np.linalg.norm(e, axis=1).mean())


def icosahedron() -> Mesh:
    p = (1.0 + 5.0 ** 0.5) / 2.0
    pts = []
    for a, b in itertools.product((-1.0, 1.0), repeat=2):
        pts += [(0.0, a, b * p), (a, b * p, 0.0), (b * p, 0.0, a)]
    verts = np.array(pts, dtype=np.float64)
    faces = []
    for i, j, k in itertools.combinations(range(12), 3):
        d = [np.linalg.norm(verts[i] - verts[j]), np.linalg.norm(verts[j] - verts[k]),
             np.linalg.norm(verts[k] - verts[i])]
        if all(abs(x - 2.0) < 1e-9 for x in d):
            faces.append((i, j, k))
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    tris = np.array(faces, dtype=np.int32)
    return Mesh(verts, _orient_outward(verts, tris, lambda c: 0.0 * c), "icosahedron")


def octahedron() -> Mesh:
    verts = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)],
                     dtype=np.float64)
    faces = [(a, b, c) for a in (0, 1) for b in (2, 3) for c in (4, 5)]
    tris = np.array(faces, dtype=np.int32)
    return Mesh(verts, _orient_outward(verts, tris, lambda c: 0.0 * c), "octahedron")


def icosphere(levels: int) -> Mesh:
    m = icosahedron()
    verts = [tuple(v) for v in m.verts]
    tris = [tuple(t) for t in m.tris]
    for _ in range(levels):
        cache = {}
        new = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                p = (np.array(verts[a]) + np.array(verts[b])) * 0.5
                p /= np.linalg.norm(p)
                cache[key] = len(verts)
                verts.append(tuple(p))
            return cache[key]

        for a, b, c in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = new
    return Mesh(np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32),
                f"icosphere{levels}")


def octasphere(n: int) -> Mesh:
    """Paper's test surface: the 8 faces of |x|_1 = 1 split regularly into n^2 triangles."""
    index = {}
    verts = []

    def vid(key):
        if key not in index:
            index[key] = len(verts)
            p = np.array(key, dtype=np.float64) / n
            verts.append(p / np.linalg.norm(p))
        return index[key]

    tris = []
    for sx, sy, sz in itertools.product((-1, 1), repeat=3):
        # face points (sx*i, sy*j, sz*(n-i-j)) with i + j <= n
        def P(i, j):
            return vid((sx * i, sy * j, sz * (n - i - j)))
        for i in range(n):
            for j in range(n - i):
                tris.append((P(i, j), P(i + 1, j), P(i, j + 1)))
                if i + j + 1 < n:
                    tris.append((P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)))
    verts = np.array(verts, dtype=np.float64)
    tris = np.array(tris, dtype=np.int32)
    return Mesh(verts, _orient_outward(verts, tris, lambda c: 0.0 * c), f"octasphere{n}")


def subdivided_sphere(base: Mesh, n: int, name: str) -> Mesh:
    """Each face of a convex polyhedron inscribed in the unit sphere split
    regularly into n^2 triangles, vertices projected to the unit sphere."""
    index = {}
    verts = []

    def vid(key, p):
        if key not in index:
            index[key] = len(verts)
            verts.append(p / np.linalg.norm(p))
        return index[key]

    def key_of(face, i, j):
        # a point (i, j, n-i-j) on a face, made canonical across shared edges by
        # its exact barycentric weights on the sorted vertex ids
        a, b, c = face
        w = {a: n - i - j, b: i, c: j}
        return tuple(sorted((v, k) for v, k in w.items() if k > 0))

    tris = []
    for face in base.tris:
        A, B, C = (base.verts[v] for v in face)

        def P(i, j):
            return vid(key_of(face, i, j), (A * (n - i - j) + B * i + C * j) / n)
        for i in range(n):
            for j in range(n - i):
                tris.append((P(i, j), P(i + 1, j), P(i, j + 1)))
                if i + j + 1 < n:
                    tris.append((P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)))
    verts = np.array(verts, dtype=np.float64)
    tris = np.array(tris, dtype=np.int32)
    return Mesh(verts, _orient_outward(verts, tris, lambda c: 0.0 * c), name)


def icosphere_n(n: int) -> Mesh:
    """Icosahedron with every face split into n^2 triangles (20 n^2 triangles)."""
    return subdivided_sphere(icosahedron(), n, f"icosphere_n{n}")


def cube_surface(n: int) -> Mesh:
    index = {}
    verts = []

    def vid(p):
        if p not in index:
            index[p] = len(verts)
            verts.append(np.array(p, dtype=np.float64) / n)
        return index[p]

    tris = []
    for axis in range(3):
        for side in (0, n):
            for i in range(n):
                for j in range(n):
                    def P(a, b):
                        q = [0, 0, 0]
                        q[axis] = side
                        q[(axis + 1) % 3] = a
                        q[(axis + 2) % 3] = b
                        return vid(tuple(q))
                    a, b, c, d = P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)
                    tris.append((a, b, c))
                    tris.append((a, c, d))
    verts = np.array(verts, dtype=np.float64)
    tris = np.array(tris, dtype=np.int32)
    return Mesh(verts, _orient_outward(verts, tris, lambda c: 0.0 * c + 0.5), f"cube{n}")


def torus(nu: int, nv: int, R: float = 1.0, r: float = 0.3) -> Mesh:
    u = 2.0 * np.pi * np.arange(nu) / nu
    v = 2.0 * np.pi * np.arange(nv) / nv
    U, V = np.meshgrid(u, v, indexing="ij")
    verts = np.stack([(R + r * np.cos(V)) * np.cos(U), (R + r * np.cos(V)) * np.sin(U),
                      r * np.sin(V)], axis=-1).reshape(-1, 3)

    def vid(i, j):
        return (i % nu) * nv + (j % nv)

    tris = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tris.append((a, b, c))
            tris.append((a, c, d))
    tris = np.array(tris, dtype=np.int32)

    def tube_center(c):
        phi = np.arctan2(c[:, 1], c[:, 0])
        return np.stack([R * np.cos(phi), R * np.sin(phi), 0.0 * phi], axis=-1)
    return Mesh(verts.astype(np.float64), _orient_outward(verts, tris, tube_center),
                f"torus{nu}x{nv}")


def jitter(mesh: Mesh, frac: float, seed: int) -> Mesh:
    h = mean_edge_length(mesh)
    rng = SplitMix64(seed)
    noise = rng.uniform(mesh.nv * 3, -frac * h, frac * h).reshape(mesh.nv, 3)
    return Mesh(mesh.verts + noise, mesh.tris.copy(), mesh.name + f"+jitter{frac}")


def two_triangles(case: str, angle_deg: float = 90.0, aspect: float = 1.0) -> Mesh:
    """Two flat triangles in a chosen touching configuration (not a closed surface).

    case 'identical': one triangle listed twice with the same vertex ids.
    case 'edge':   common edge (0,1); the second triangle is the first rotated
                   about the edge by angle_deg (180 = coplanar).
    case 'vertex': common vertex 0 only.
    case 'far':    disjoint triangles one unit apart.
    """
    a = np.array([0.0, 0.0, 0.0])
    b = np.array([1.0, 0.0, 0.0])
    c = np.array([0.35, 0.8 * aspect, 0.0])
    th = np.deg2rad(angle_deg)
    # rotate c (relative to the edge a-b) about the x axis by th, then reflect so the
    # second triangle sits on the other side of the edge when th = 180
    d = np.array([0.6, 0.7 * aspect * np.cos(th), 0.7 * aspect * np.sin(th)])
    if case == "identical":
        return Mesh(np.stack([a, b, c]), np.array([[0, 1, 2], [0, 1, 2]], np.int32), "identical")
    if case == "edge":
        return Mesh(np.stack([a, b, c, d]), np.array([[0, 1, 2], [1, 0, 3]], np.int32), "edge")
    if case == "vertex":
        e = np.array([-0.8, 0.3, 0.45])
        f = np.array([-0.5, -0.6, 0.2])
        return Mesh(np.stack([a, b, c, e, f]), np.array([[0, 1, 2], [0, 3, 4]], np.int32),
                    "vertex")
    if case == "far":
        e = c + np.array([0.2, 0.3, 1.0])
        return Mesh(np.stack([a, b, c, a + [0.1, 0.2, 1.0], b + [0.0, 0.3, 1.1], e]),
                    np.array([[0, 1, 2], [3, 4, 5]], np.int32), "far")
    raise ValueError(case)

"""Index-set structure for H2-style block partitions (no quadrature arithmetic).

build_cluster_tree: geometric bisection of the index set (triangles for the
  piecewise-constant basis, vertices for the piecewise-linear basis): a
  cluster's index points are split at the middle of the longest side of their
  bounding box, recursively, until at most `leaf_size` indices remain.
build_block_partition: the recursive block tree over (root, root) with the
  admissibility test  max(diam B_t, diam B_s) <= eta * dist(B_t, B_s),  where
  B_t bounds the supports of all basis functions of t.  Admissible leaves are
  far blocks, leaf x leaf inadmissible blocks are near blocks.
seeded_pivots: a seeded stand-in for the cross-approximation pivots, at most
  `rank` indices per cluster.
green_box_points: the point sets of the Green quadrature matrices (Section
  2.3): points, outward normals and weights of a tensor Gauss-Legendre rule
  (numpy's nodes) on the six faces of a cluster's auxiliary box omega_t.  They
  are inputs of the library's call; the integrals over the mesh are not here.

Everything is returned as plain int32/int64 numpy arrays in the cluster-CSR
form that the library's block-list calls take: clusters (ptr, idx), blocks
(row cluster, column cluster, output offset).
"""
from dataclasses import dataclass, field
import numpy as np

from .rng import SplitMix64


@dataclass
class ClusterTree:
    perm: np.ndarray                 # indices in cluster order
    start: list = field(default_factory=list)
    end: list = field(default_factory=list)
    sons: list = field(default_factory=list)
    bmin: list = field(default_factory=list)
    bmax: list = field(default_factory=list)

    @property
    def n_clusters(self):
        return len(self.start)

    def indices(self, c):
        return self.perm[self.start[c]:self.end[c]]

    def is_leaf(self, c):
        return len(self.sons[c]) == 0


def _support_boxes(mesh, basis):
    v = mesh.verts[mesh.tris]                  # (nt,3,3)
    tmin, tmax = v.min(axis=1), v.max(axis=1)
    if basis == "p0":
        return v.mean(axis=1), tmin, tmax
    nv = mesh.nv
    bmin = np.full((nv, 3), np.inf)
    bmax = np.full((nv, 3), -np.inf)
    for k in range(3):
        np.minimum.at(bmin, mesh.tris[:, k], tmin)
        np.maximum.at(bmax, mesh.tris[:, k], tmax)
    return mesh.verts.copy(), bmin, bmax


def build_cluster_tree(mesh, basis: str = "p0", leaf_size: int = 32) -> ClusterTree:
    pts, smin, smax = _support_boxes(mesh, basis)
    n = pts.shape[0]
    tree = ClusterTree(perm=np.arange(n, dtype=np.int64))

    def make(lo, hi):
        cid = len(tree.start)
        tree.start.append(lo)
        tree.end.append(hi)
        tree.sons.append([])
        idx = tree.perm[lo:hi]
        tree.bmin.append(smin[idx].min(axis=0))
        tree.bmax.append(smax[idx].max(axis=0))
        if hi - lo > leaf_size:
            p = pts[idx]
            lo_b, hi_b = p.min(axis=0), p.max(axis=0)
            ax = int(np.argmax(hi_b - lo_b))
            mid = 0.5 * (lo_b[ax] + hi_b[ax])
            left = p[:, ax] <= mid
            if left.all() or not left.any():      # coincident points: split by count
                order = np.argsort(p[:, ax], kind="stable")
                left = np.zeros(len(idx), bool)
                left[order[: len(idx) // 2]] = True
            tree.perm[lo:hi] = np.concatenate([idx[left], idx[~left]])
            m = lo + int(left.sum())
            tree.sons[cid] = [make(lo, m), make(m, hi)]
        return cid

    make(0, n)
    return tree


def _diam(bmin, bmax):
    return float(np.linalg.norm(bmax - bmin))


def _dist(amin, amax, bmin, bmax):
    gap = np.maximum(0.0, np.maximum(amin - bmax, bmin - amax))
    return float(np.linalg.norm(gap))


@dataclass
class BlockPartition:
    tree: ClusterTree
    near: list          # [(t, s)]
    far: list           # [(t, s)]

    def cluster_csr(self, clusters=None):
        """(ptr, idx) of the index sets of all clusters, int32."""
        t = self.tree
        sizes = [t.end[c] - t.start[c] for c in range(t.n_clusters)]
        ptr = np.zeros(t.n_clusters + 1, np.int32)
        ptr[1:] = np.cumsum(sizes)
        idx = np.concatenate([t.indices(c) for c in range(t.n_clusters)]).astype(np.int32)
        return ptr, idx

    def son_array(self):
        """int32 (n_clusters, 2): the sons of every cluster, -1 where absent."""
        t = self.tree
        out = np.full((t.n_clusters, 2), -1, np.int32)
        for c in range(t.n_clusters):
            for k, s in enumerate(t.sons[c]):
                out[c, k] = s
        return out

    def near_blocks(self):
        """(blk_row, blk_col, blk_off, total) for the near blocks, column-major |t| x |s|."""
        return _blocks(self.near, lambda c: self.tree.end[c] - self.tree.start[c])

    def n_near_entries(self):
        return int(self.near_blocks()[3])


def _blocks(pairs, size):
    r = np.array([p[0] for p in pairs], np.int32)
    c = np.array([p[1] for p in pairs], np.int32)
    n = np.array([size(a) * size(b) for a, b in pairs], np.int64)
    off = np.zeros(len(pairs), np.int64)
    if len(pairs):
        off[1:] = np.cumsum(n)[:-1]
    return r, c, off, int(n.sum())


def build_block_partition(mesh, basis: str = "p0", leaf_size: int = 32,
                          eta: float = 2.0) -> BlockPartition:
    tree = build_cluster_tree(mesh, basis, leaf_size)
    near, far = [], []
    stack = [(0, 0)]
    while stack:
        t, s = stack.pop()
        bt = (tree.bmin[t], tree.bmax[t])
        bs = (tree.bmin[s], tree.bmax[s])
        if max(_diam(*bt), _diam(*bs)) <= eta * _dist(bt[0], bt[1], bs[0], bs[1]):
            far.append((t, s))
        elif tree.is_leaf(t) and tree.is_leaf(s):
            near.append((t, s))
        else:
            st = tree.sons[t] if not tree.is_leaf(t) else [t]
            ss = tree.sons[s] if not tree.is_leaf(s) else [s]
            for a in reversed(st):
                for b in reversed(ss):
                    stack.append((a, b))
    near.sort()
    far.sort()
    return BlockPartition(tree, near, far)


def seeded_pivots(part: BlockPartition, rank: int, seed: int):
    """At most `rank` seeded indices per cluster, as cluster CSR (ptr, idx) int32."""
    rng = SplitMix64(seed)
    t = part.tree
    ptr = [0]
    idx = []
    for c in range(t.n_clusters):
        ind = t.indices(c)
        k = min(rank, len(ind))
        pick = np.sort(ind[rng.permutation(len(ind))[:k]])
        idx.append(pick)
        ptr.append(ptr[-1] + k)
    return np.array(ptr, np.int32), np.concatenate(idx).astype(np.int32)


def coupling_blocks(part: BlockPartition, piv_ptr):
    """(blk_row, blk_col, blk_off, total) for the far blocks over pivot sets."""
    return _blocks(part.far, lambda c: int(piv_ptr[c + 1] - piv_ptr[c]))


def green_box_points(bmin, bmax, gauss_per_face: int):
    """Points on the boundary of the auxiliary box omega_t of a cluster whose
    supports lie in the box [bmin, bmax] (Section 2.3): omega_t is that box
    grown by delta / 2 on every side, delta = diam [bmin, bmax], so the points
    stay delta / 2 away from the supports.  Each face carries the tensor
    product of two gauss_per_face-point Gauss-Legendre rules.

    Returns (z (m, 3), outward unit normals (m, 3), weights (m,), delta) with
    m = 6 gauss_per_face^2, faces in the order -x, +x, -y, +y, -z, +z."""
    bmin = np.asarray(bmin, np.float64)
    bmax = np.asarray(bmax, np.float64)
    delta = float(np.linalg.norm(bmax - bmin))
    lo, hi = bmin - 0.5 * delta, bmax + 0.5 * delta
    x, w = np.polynomial.legendre.leggauss(int(gauss_per_face))
    z, nz, wt = [], [], []
    for ax in range(3):
        a, b = [d for d in range(3) if d != ax]
        ua = 0.5 * (lo[a] + hi[a]) + 0.5 * (hi[a] - lo[a]) * x
        ub = 0.5 * (lo[b] + hi[b]) + 0.5 * (hi[b] - lo[b]) * x
        wab = np.outer(w * 0.5 * (hi[a] - lo[a]), w * 0.5 * (hi[b] - lo[b])).ravel()
        for side, val in ((-1.0, lo[ax]), (1.0, hi[ax])):
            p = np.zeros((len(x) * len(x), 3))
            p[:, ax] = val
            p[:, a] = np.repeat(ua, len(x))
            p[:, b] = np.tile(ub, len(x))
            n = np.zeros_like(p)
            n[:, ax] = side
            z.append(p)
            nz.append(n)
            wt.append(wab)
    return np.concatenate(z), np.concatenate(nz), np.concatenate(wt), delta


def green_point_sets(tree: ClusterTree, clusters, gauss_per_face: int):
    """Green point sets of the given clusters in the CSR form the library's
    Green-matrix call takes: (pt_ptr int32, z (m, 3), nz (m, 3), sp, sm) with
    sp = sqrt(w) and sm = sqrt(w) delta_t, the factors of A_t+ and A_t-."""
    ptr = [0]
    zs, ns, sps, sms = [], [], [], []
    for c in clusters:
        z, n, w, delta = green_box_points(tree.bmin[c], tree.bmax[c], gauss_per_face)
        zs.append(z)
        ns.append(n)
        sps.append(np.sqrt(w))
        sms.append(np.sqrt(w) * delta)
        ptr.append(ptr[-1] + len(z))
    return (np.array(ptr, np.int32), np.concatenate(zs), np.concatenate(ns),
            np.concatenate(sps), np.concatenate(sms))

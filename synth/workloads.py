"""Synthetic workloads of the benchmark configurations (inputs only).

Seeds: 151007244 + 1000 * config + mesh index.  Each workload lists its mesh,
basis, kernels, quadrature orders and, for the H2 configurations, the block
partition (near blocks over cluster index sets, far blocks over pivot sets).
"""
from dataclasses import dataclass, field

import numpy as np

from . import meshes, structure

SEED0 = 151007244


def seed(config: int, mesh_index: int = 0) -> int:
    return SEED0 + 1000 * config + mesh_index


@dataclass
class Operator:
    kernel: str
    kappa: float = 0.0


@dataclass
class Quad:
    q_regular: int = 3
    regular_rule: str = "duffy"
    q_identical: int = 5
    q_edge: int = 5
    q_vertex: int = 5

    def kw(self):
        return dict(q_regular=self.q_regular, regular_rule=self.regular_rule,
                    q_identical=self.q_identical, q_edge=self.q_edge, q_vertex=self.q_vertex)


@dataclass
class BlockSet:
    """Cluster CSR (ptr, idx) for rows and columns, and blocks (row, col, off)."""
    row_ptr: np.ndarray
    row_idx: np.ndarray
    col_ptr: np.ndarray
    col_idx: np.ndarray
    blk_row: np.ndarray
    blk_col: np.ndarray
    blk_off: np.ndarray
    n_entries: int

    def entry_indices(self):
        """(rows, cols) of every output entry in output order (column-major blocks)."""
        R, C = [], []
        for t, s in zip(self.blk_row, self.blk_col):
            ri = self.row_idx[self.row_ptr[t]:self.row_ptr[t + 1]]
            ci = self.col_idx[self.col_ptr[s]:self.col_ptr[s + 1]]
            R.append(np.tile(ri, len(ci)))
            C.append(np.repeat(ci, len(ri)))
        if not R:
            return np.zeros(0, np.int64), np.zeros(0, np.int64)
        return np.concatenate(R).astype(np.int64), np.concatenate(C).astype(np.int64)


@dataclass
class Workload:
    name: str
    mesh: meshes.Mesh
    basis: str
    operators: list
    quad: Quad
    dense: bool = False
    near: BlockSet = None
    far: BlockSet = None
    meta: dict = field(default_factory=dict)
    partition: object = None         # structure.BlockPartition of the H2 blocks

    @property
    def n_entries_per_operator(self):
        if self.dense:
            n = self.mesh.nt if self.basis == "p0" else self.mesh.nv
            return n * n
        return self.near.n_entries + self.far.n_entries


def h2_blocks(mesh, basis, leaf_size=32, eta=2.0, rank=16, pivot_seed=0):
    part = structure.build_block_partition(mesh, basis, leaf_size, eta)
    cptr, cidx = part.cluster_csr()
    r, c, off, tot = part.near_blocks()
    near = BlockSet(cptr, cidx, cptr, cidx, r, c, off, tot)
    pptr, pidx = structure.seeded_pivots(part, rank, pivot_seed)
    fr, fc, foff, ftot = structure.coupling_blocks(part, pptr)
    far = BlockSet(pptr, pidx, pptr, pidx, fr, fc, foff, ftot)
    return part, near, far


def config1() -> Workload:
    """Laplace single layer, P0, 1280-triangle icosphere, dense; SS q=4, Radon 7x7."""
    mesh = meshes.icosphere(3)
    return Workload("C1 icosphere1280 laplace_slp p0 dense", mesh, "p0",
                    [Operator("laplace_slp")],
                    Quad(q_regular=3, regular_rule="tri7", q_identical=4, q_edge=4, q_vertex=4),
                    dense=True)


def config2(levels: int = 5) -> Workload:
    """Laplace SLP + DLP, P1, 20480-triangle icosphere, H2 leaf 32, eta 2, rank <= 16;
    SS q=5, Duffy q=3, FP64."""
    mesh = meshes.icosphere(levels)
    part, near, far = h2_blocks(mesh, "p1", 32, 2.0, 16, seed(2))
    return Workload(f"C2 icosphere{mesh.nt} laplace_slp+dlp p1 h2", mesh, "p1",
                    [Operator("laplace_slp"), Operator("laplace_dlp")], Quad(3, "duffy", 5, 5, 5),
                    near=near, far=far, partition=part,
                    meta={"leaf_size": 32, "eta": 2.0, "rank": 16,
                          "n_near_blocks": len(near.blk_row), "n_far_blocks": len(far.blk_row)})


def config3(n: int = 64) -> Workload:
    """Helmholtz single layer, kappa = 8, P0, surface of the unit cube with n x n
    squares per face (12 n^2 triangles; n = 64: 49152), vertices jittered by 5%
    of the mean edge length (seeded); H2 blocks (leaf 32, eta 2, <= 16 pivots);
    SS q=5, Duffy q=3; mixed precision."""
    mesh = meshes.jitter(meshes.cube_surface(n), 0.05, seed(3))
    part, near, far = h2_blocks(mesh, "p0", 32, 2.0, 16, seed(3, 1))
    return Workload(f"C3 cube{mesh.nt} helmholtz_slp k8 p0 h2 mixed", mesh, "p0",
                    [Operator("helmholtz_slp", 8.0)], Quad(3, "duffy", 5, 5, 5),
                    near=near, far=far, partition=part,
                    meta={"leaf_size": 32, "eta": 2.0, "rank": 16, "precision": "mixed"})


def config5(n: int = 128) -> Workload:
    """Learned quadrature orders: the paper's octahedral sphere with 8 n^2 triangles
    (n = 128: 131072), vertices jittered by 5% of the mean edge length (seeded);
    Laplace double layer and Helmholtz single layer with kappa = 16, P0, H2 blocks
    (leaf 32, eta 2, <= 16 pivots); SS q=5, Duffy q=3 as the fixed orders."""
    mesh = meshes.jitter(meshes.octasphere(n), 0.05, seed(5))
    part, near, far = h2_blocks(mesh, "p0", 32, 2.0, 16, seed(5, 1))
    return Workload(f"C5 octasphere{mesh.nt} laplace_dlp+helmholtz_slp k16 p0 h2 learned", mesh,
                    "p0", [Operator("laplace_dlp"), Operator("helmholtz_slp", 16.0)],
                    Quad(3, "duffy", 5, 5, 5), near=near, far=far, partition=part,
                    meta={"leaf_size": 32, "eta": 2.0, "rank": 16, "order_mode": "learned"})


def order_training_meshes():
    """Smaller meshes of the same family on which the order model's labels are
    generated: jittered octahedral spheres with 2048, 4608 and 8192 triangles."""
    return [meshes.jitter(meshes.octasphere(n), 0.05, seed(5, 10 + k))
            for k, n in enumerate((16, 24, 32))]


@dataclass
class BatchItem:
    """One mesh of a batched workload with its operators and block sets."""
    mesh: meshes.Mesh
    operators: list
    near: BlockSet
    far: BlockSet
    partition: object = None         # structure.BlockPartition of the H2 blocks


@dataclass
class BatchWorkload:
    name: str
    basis: str
    quad: Quad
    items: list
    meta: dict = field(default_factory=dict)

    @property
    def n_entries(self):
        return sum(len(it.operators) * (it.near.n_entries + it.far.n_entries) for it in self.items)


def _nearest(target, sizes):
    """(n, size) minimising |log size - log target| over the candidates."""
    best = min(sizes, key=lambda ns: abs(np.log(ns[1]) - np.log(target)))
    return best


def config4(count: int = 48, lo: float = 500.0, hi: float = 30000.0, leaf_size: int = 32,
            eta: float = 2.0, rank: int = 16) -> BatchWorkload:
    """48 closed meshes of uneven size (16 spheres, 16 cubes, 16 tori with radii
    1 and 0.3), target sizes log-uniform in [500, 30000] triangles (seeded),
    jitter 5%; per mesh the Laplace double layer and the Helmholtz single layer
    with kappa ~ U[1, 10]; P0, H2 blocks (leaf 32, eta 2, <= 16 pivots)."""
    from .rng import SplitMix64
    rng = SplitMix64(seed(4))
    targets = np.exp(rng.uniform(count, np.log(lo), np.log(hi)))
    kappas = rng.uniform(count, 1.0, 10.0)
    items = []
    for k in range(count):
        kind = ("sphere", "cube", "torus")[k % 3]
        t = targets[k]
        if kind == "sphere":
            n, _ = _nearest(t, [(n, 20 * n * n) for n in range(3, 40)])
            mesh = meshes.icosphere_n(n)
        elif kind == "cube":
            n, _ = _nearest(t, [(n, 12 * n * n) for n in range(3, 51)])
            mesh = meshes.cube_surface(n)
        else:
            cands = []
            for nv_ in range(4, 60):
                nu_ = max(6, int(round(3.3 * nv_)))
                cands.append(((nu_, nv_), 2 * nu_ * nv_))
            (nu_, nv_), _ = _nearest(t, cands)
            mesh = meshes.torus(nu_, nv_)
        mesh = meshes.jitter(mesh, 0.05, seed(4, k))
        part, near, far = h2_blocks(mesh, "p0", leaf_size, eta, rank, seed(4, 100 + k))
        items.append(BatchItem(mesh, [Operator("laplace_dlp"),
                                      Operator("helmholtz_slp", float(kappas[k]))], near, far,
                               part))
    return BatchWorkload(f"C4 {count} meshes (spheres/cubes/tori) laplace_dlp+helmholtz_slp p0 h2",
                         "p0", Quad(3, "duffy", 5, 5, 5), items,
                         meta={"triangles": int(sum(it.mesh.nt for it in items))})

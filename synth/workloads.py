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
                    near=near, far=far,
                    meta={"leaf_size": 32, "eta": 2.0, "rank": 16,
                          "n_near_blocks": len(near.blk_row), "n_far_blocks": len(far.blk_row)})

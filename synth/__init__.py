"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds mesh generators, a counter-free splitmix64 stream, and
purely structural index-set builders (cluster trees, block partitions and
seeded pivot subsets), and the point sets on the clusters' auxiliary boxes that
the Green quadrature matrices take as input.  It contains none of the
quadrature arithmetic over the mesh: no triangle or Sauter-Schwab rules, no
kernels, no integrals.
"""
from .rng import SplitMix64
from .meshes import (Mesh, icosphere, icosphere_n, octasphere, cube_surface, torus,
                     jitter, icosahedron, octahedron, two_triangles,
                     mean_edge_length)
from . import workloads
from .structure import (ClusterTree, build_cluster_tree, build_block_partition,
                        seeded_pivots, BlockPartition, green_box_points,
                        green_point_sets)

__all__ = ["SplitMix64", "Mesh", "icosphere", "icosphere_n", "octasphere", "cube_surface",
           "torus", "jitter", "icosahedron", "octahedron", "two_triangles",
           "mean_edge_length", "ClusterTree", "build_cluster_tree",
           "build_block_partition", "seeded_pivots", "BlockPartition", "workloads",
           "green_box_points", "green_point_sets"]

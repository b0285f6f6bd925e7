"""GB300 (sm_103a) Galerkin boundary-element quadrature: Sauter-Schwab near
field and H2 coupling/pivot entries behind the C ABI of include/bem.h.

The compute path is the CUDA library built by ``paper_1510_07244_gb300.build``;
this package only marshals arguments to it (``_binding``) and orchestrates the
training of the quadrature-order model (``order_model``).  The synthetic
inputs live in the separate ``synth`` package.
"""
from ._binding import (Context, BlockJob, GreenJob, BemError, kernel_desc, quad_desc, load,
                       LIB_PATH, EXPORTS, KERNELS, BASES, RULES, bem_rule_points, bem_rule_points_xi, PLAN_GRAPH,
                       PLAN_AUTOTUNE, PLAN_PROFILE, PLAN_STATIC_LISTS, ORDER_CLASSES,
                       ORDER_CLASS_POINTS, bem_shard_blocks, bem_gca_pivots,
                       bem_touching_pairs, bem_gca_bases)

__all__ = ["Context", "BlockJob", "GreenJob", "BemError", "kernel_desc", "quad_desc", "load",
           "LIB_PATH", "EXPORTS", "KERNELS", "BASES", "RULES", "bem_rule_points", "bem_rule_points_xi",
           "PLAN_GRAPH", "PLAN_AUTOTUNE", "PLAN_PROFILE", "PLAN_STATIC_LISTS", "ORDER_CLASSES",
           "ORDER_CLASS_POINTS", "bem_shard_blocks", "bem_gca_pivots",
           "bem_touching_pairs", "bem_gca_bases"]

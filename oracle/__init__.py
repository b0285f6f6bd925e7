"""Plain FP64 CPU oracle for Galerkin BEM matrix entries -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library (``paper_1510_07244_gb300``) never
imports it and shares no code with it.
"""
from .oracle import (build, gauss_legendre01, radon7, rule_points, classify, classify_orders,
                     entries, entries_absolute, pair, green_entries, CASES, KERNELS, BASES,
                     RULES)

__all__ = ["build", "gauss_legendre01", "radon7", "rule_points", "classify", "classify_orders",
           "entries", "green_entries",
           "entries_absolute", "pair", "CASES", "KERNELS", "BASES", "RULES"]

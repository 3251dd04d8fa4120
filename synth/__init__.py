"""Seeded synthetic workloads shared by the oracle tests, the CUDA-path tests and the bench.

This module only draws random inputs and prepares them (label rule, min-max scaling). It holds
none of the method's arithmetic: no kernel sums, no Fourier coefficients, no solver steps.

Workloads stand in for the paper's datasets (HIGGS, SUSY, cod-rna; Sec. 6), which are not
available here: the dimensions d (6-12) and window counts P (2-4) lie in the paper's range
(d 8-28, P 3-10) and n reaches its "large" regime (n > 1e5).
"""
from .data import (SEED_BASE, minmax_scale, consecutive_windows, config1, config2, config3,
                   config4, config5, matvec_vectors, subsample_rows, small_problem, C_GRID, SIGMA_GRID)

__all__ = ["SEED_BASE", "minmax_scale", "consecutive_windows", "config1", "config2", "config3",
           "config4", "config5", "matvec_vectors", "subsample_rows", "small_problem", "C_GRID", "SIGMA_GRID"]

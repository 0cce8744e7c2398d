"""CPU FP64 oracle for the RFD graph-field integrator (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs may import this package.  The library never does.
"""
from .rfd import *  # noqa: F401,F403
from .rfd import (SplitMix64, sample_frequencies, tau, density, weights, features,
                  column_scales, factors, phi1, rfd_gfi, rfd_gfi_from_plan,
                  dense_lowrank_gfi, exact_adjacency, dense_exact_gfi,
                  smoothed_kernel, smoothed_adjacency, rel_frobenius,
                  default_sigma, default_radius)

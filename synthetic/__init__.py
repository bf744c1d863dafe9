"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds only input generation (random hole layouts, random vectors, the
named workload presets and the network's initial weights).  It contains none of the method's arithmetic: no basis
functions, quadrature, assembly, multigrid or Krylov steps.
"""
from .geometry import HoleLayout, random_holes, config1_disc, config_layout
from .configs import PRESETS, Preset, preset
from .vectors import random_grid_vector
from .network import initial_weights, random_error

__all__ = ["HoleLayout", "random_holes", "config1_disc", "config_layout", "PRESETS",
           "Preset", "preset", "random_grid_vector", "initial_weights", "random_error"]

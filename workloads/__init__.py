"""Seeded synthetic inputs shared by the GPU path's harness and by the oracle.

This package holds no arithmetic of the solver itself: no metric, no spectral
operator, no conserved-variable map.  It defines the workload configurations
(grid sizes, spin, equation-of-state index, seeds) and evaluates the primitive
profiles (density, pressure, velocity, vector potential) at node coordinates that
the caller computes on its own side.
"""
from .synth import (  # noqa: F401
    Config, CONFIGS, config, batch_configs, splitmix64, noise, primitive_profiles,
    global_node_index,
)

"""Seeded synthetic instances of the multi-agent collision-avoidance QP.

This module only *draws* problem data (starts, goals, model matrices,
linearization halfspaces and the initial consensus positions). It holds none
of the solver's arithmetic, and both the CPU oracle and the GPU path read the
same arrays from it.
"""
from .generator import (  # noqa: F401
    Batch,
    SplitMix64,
    make_workload,
    WORKLOADS,
    make_batch,
    double_integrator,
    pair_list,
    random_scenario,
    build_scenario,
    nearest_neighbour_pairs,
    heterogeneous_agents,
)

"""Seeded synthetic tree tensor networks shared by the oracle, the tests and the bench.

This module only draws random numbers and fixes shapes. It holds none of the CBC
arithmetic (no contraction, no decomposition), so the CPU oracle and the CUDA path
can both consume its output without sharing any of the method's code.
"""
from .networks import (  # noqa: F401
    Network,
    Problem,
    binary_tree_topology,
    chain_topology,
    children_of,
    clamp_bonds,
    make_problem,
    random_network,
    sketch_matrices,
    CONFIGS,
)

"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package draws random numbers and packs them into plain data records
(task durations, demands, capacities, precedence edges, bound restrictions on
start variables, random generic constraint rows).  It holds none of the
method's arithmetic: no propagation, no branching rule, no model expansion.
Both sides build their own stores and constraint tables from these records.
"""
from .rng import SplitMix64
from .rcpsp import RcpspInstance, draw_rcpsp, config_instance, CONFIGS
from .nodes import draw_partial_assignments
from .generic import GenericModel, draw_generic_model, draw_generic_store

__all__ = [
    "SplitMix64", "RcpspInstance", "draw_rcpsp", "config_instance", "CONFIGS",
    "draw_partial_assignments", "GenericModel", "draw_generic_model", "draw_generic_store",
]

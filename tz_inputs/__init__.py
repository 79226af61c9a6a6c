"""Seeded synthetic inputs shared by the oracle and the GPU library.

This package only *describes problems*: lattices, the random-circuit
prescription of Sec. 1 (which gate goes where; gate names only) and random
output bitstrings. It holds none of the method's arithmetic: no gate matrix,
no tensor, no contraction. Both the oracle and the product consume the
circuit through its plain-text spec.
"""
from .splitmix64 import SplitMix64
from .lattice import Lattice, grid, bristlecone
from .generate import generate_circuit, circuit_to_spec, cz_pattern_edges, PATTERN_ORDER
from .bitstrings import random_bitstrings

__all__ = [
    "SplitMix64", "Lattice", "grid", "bristlecone", "generate_circuit",
    "circuit_to_spec", "cz_pattern_edges", "PATTERN_ORDER", "random_bitstrings",
]

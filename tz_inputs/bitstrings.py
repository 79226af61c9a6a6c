"""Seeded uniform random output bitstrings.

Row j of the result is bitstring x_j; column q is the bit of qubit q (0/1,
uint8). Bits are drawn row by row, qubit by qubit, each the top bit of one
SplitMix64 draw.
"""
import numpy as np

from .splitmix64 import SplitMix64


def random_bitstrings(n_qubits: int, count: int, seed: int) -> np.ndarray:
    rng = SplitMix64(seed)
    out = np.empty((count, n_qubits), dtype=np.uint8)
    for j in range(count):
        for q in range(n_qubits):
            out[j, q] = rng.next_bit()
    return out

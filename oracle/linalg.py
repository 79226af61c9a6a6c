"""Plain definitions of the per-step operations of a contraction (FP64).

These are the textbook definitions the GPU kernels must reproduce:

* bit permutation: a tensor whose indices all have dimension 2 is stored as
  a vector of 2^r entries; transposing it permutes the bits of the entry
  offset. out[j] = in[i] where bit perm[p] of i equals bit p of j.
* batched complex matrix product C[z] = A[z] B[z]^T (the contraction of one
  tree node once the operands are laid out as [batch, m, k] and
  [batch, n, k]); numpy's matmul in complex128 is the primitive.
* FP64 sum of partial amplitudes (Sec. 1: subtask results add up to the
  amplitude): acc + scale * part, in complex128.
"""
import numpy as np


def bit_permute(x: np.ndarray, perm) -> np.ndarray:
    r = len(perm)
    x = np.asarray(x).reshape(-1)
    assert x.size == 1 << r
    j = np.arange(1 << r, dtype=np.int64)
    i = np.zeros_like(j)
    for p, q in enumerate(perm):
        i |= ((j >> p) & 1) << q
    return x[i]


def cgemm(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A: (batch, m, k), B: (batch, n, k) -> (batch, m, n), complex128."""
    return np.matmul(A.astype(np.complex128), np.swapaxes(B.astype(np.complex128), 1, 2))


def accumulate(acc: np.ndarray, part: np.ndarray, scale: complex = 1.0) -> np.ndarray:
    return acc.astype(np.complex128) + complex(scale) * part.astype(np.complex128)

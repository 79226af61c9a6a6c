"""FP64 state-vector simulation (oracle part 1).

a(x) = <x| U_C |0^n>, U_C the gates of the spec applied in file order.
Indexing: bit q of the basis-state index is qubit q, i.e. the state index of
bitstring x is sum_q x_q 2^q.
"""
import numpy as np

from .gates import ONE_QUBIT, CZ
from .spec import parse_spec


def _axis(n, q):
    # psi is reshaped C-order to (2,)*n, so axis 0 carries the highest bit.
    return n - 1 - q


def final_state(n, gates):
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    for (_, name, qs) in gates:
        if name == "cz":
            a, b = _axis(n, qs[0]), _axis(n, qs[1])
            idx = [slice(None)] * n
            idx[a] = 1
            idx[b] = 1
            psi[tuple(idx)] *= -1.0
        else:
            ax = _axis(n, qs[0])
            psi = np.moveaxis(np.tensordot(ONE_QUBIT[name], psi, axes=([1], [ax])), 0, ax)
    return psi.reshape(-1)


def basis_index(bits):
    return int(sum(int(b) << q for q, b in enumerate(bits)))


def amplitudes(spec_text: str, bitstrings) -> np.ndarray:
    n, gates = parse_spec(spec_text)
    psi = final_state(n, gates)
    return np.array([psi[basis_index(x)] for x in np.asarray(bitstrings)], dtype=np.complex128)


def dense_unitary(n, gates):
    """The full 2^n x 2^n matrix of the circuit from Kronecker products
    (small n only). Qubit q is the factor at Kronecker position n-1-q, so the
    matrix acts on the same little-endian index as `final_state`."""
    I2 = np.eye(2, dtype=np.complex128)
    U = np.eye(1 << n, dtype=np.complex128)
    for (_, name, qs) in gates:
        if name == "cz":
            d = np.ones(1 << n, dtype=np.complex128)
            for i in range(1 << n):
                if (i >> qs[0]) & 1 and (i >> qs[1]) & 1:
                    d[i] = -1.0
            G = np.diag(d)
        else:
            G = np.array([[1.0]], dtype=np.complex128)
            for pos in range(n):
                q = n - 1 - pos
                G = np.kron(G, ONE_QUBIT[name] if q == qs[0] else I2)
        U = G @ U
    return U

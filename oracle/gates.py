"""FP64 gate matrices of the circuit family of Sec. 1.

The paper names the gates (H, CZ, T, sqrt(X), sqrt(Y)) but prints no matrix;
these are the standard definitions, with the principal square roots:

  H       = (1/sqrt2) [[1, 1], [1, -1]]
  T       = diag(1, exp(i pi/4))
  sqrt(X) = (1/2) [[1+i, 1-i], [1-i, 1+i]]      (squares to X exactly)
  sqrt(Y) = (1/2) [[1+i, -1-i], [1+i, 1+i]]     (squares to Y exactly)
  CZ      = diag(1, 1, 1, -1)

Matrices act on column vectors (|0>, |1>): U[out, in].
"""
import numpy as np

S2 = 1.0 / np.sqrt(2.0)
H = np.array([[S2, S2], [S2, -S2]], dtype=np.complex128)
T = np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128)
SQRT_X = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
SQRT_Y = 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128)
CZ = np.diag(np.array([1, 1, 1, -1], dtype=np.complex128))
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)

ONE_QUBIT = {"h": H, "t": T, "x_1_2": SQRT_X, "y_1_2": SQRT_Y}


def cz_tensor():
    """CZ as a rank-4 tensor [o0, o1, i0, i1] (out legs first)."""
    return CZ.reshape(2, 2, 2, 2)

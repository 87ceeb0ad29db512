"""FP64 gate matrices of the oracle, written from the standard definitions.

Conventions: qubit q is bit q of the amplitude index (Sec. 2).  Matrices act on
column vectors; for multi-qubit matrices the row/column index is
r = sum_t b(q_t) 2^t over the gate's listed qubits (first listed = least
significant).  No global phase is dropped: amplitudes are compared exactly.
"""
import math

import numpy as np

SQ2 = 1.0 / math.sqrt(2.0)


def one_qubit_matrix(kind: str, param: float = 0.0, matrix=None) -> np.ndarray:
    """2x2 matrix of a single-qubit gate kind."""
    if kind == "U1":
        return np.asarray(matrix, dtype=np.complex128).reshape(2, 2)
    if kind == "H":
        return np.array([[SQ2, SQ2], [SQ2, -SQ2]], dtype=np.complex128)
    if kind == "X":
        return np.array([[0, 1], [1, 0]], dtype=np.complex128)
    if kind == "Y":
        return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    if kind == "Z":
        return np.array([[1, 0], [0, -1]], dtype=np.complex128)
    if kind == "S":
        return np.array([[1, 0], [0, 1j]], dtype=np.complex128)
    if kind == "T":
        return np.array([[1, 0], [0, complex(SQ2, SQ2)]], dtype=np.complex128)
    h = 0.5 * param
    if kind == "RZ":   # exp(-i theta Z / 2)
        return np.array([[complex(math.cos(h), -math.sin(h)), 0], [0, complex(math.cos(h), math.sin(h))]],
                        dtype=np.complex128)
    if kind == "RX":   # exp(-i theta X / 2)
        return np.array([[math.cos(h), complex(0, -math.sin(h))], [complex(0, -math.sin(h)), math.cos(h)]],
                        dtype=np.complex128)
    if kind == "RY":   # exp(-i theta Y / 2)
        return np.array([[math.cos(h), -math.sin(h)], [math.sin(h), math.cos(h)]], dtype=np.complex128)
    if kind == "P":    # diag(1, e^{i theta})
        return np.array([[1, 0], [0, complex(math.cos(param), math.sin(param))]], dtype=np.complex128)
    raise ValueError(kind)


def controlled_target_matrix(kind: str, param: float = 0.0, matrix=None) -> np.ndarray:
    """The 2x2 applied to the target when the control is 1."""
    if kind == "CNOT":
        return one_qubit_matrix("X")
    if kind == "CZ":
        return one_qubit_matrix("Z")
    if kind == "CP":
        return one_qubit_matrix("P", param)
    if kind == "CU":
        return np.asarray(matrix, dtype=np.complex128).reshape(2, 2)
    raise ValueError(kind)


SWAP4 = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def gate_full_matrix(g) -> np.ndarray:
    """The gate as a 2^k x 2^k matrix over its listed qubits (r = sum b(q_t) 2^t)."""
    k = g.kind
    if k in ("U2", "UK"):
        return np.asarray(g.matrix, dtype=np.complex128)
    if len(g.qubits) == 1:
        return one_qubit_matrix(k, g.param, g.matrix)
    if k in ("CNOT", "CZ", "CP", "CU"):
        u = controlled_target_matrix(k, g.param, g.matrix)
        m = np.eye(4, dtype=np.complex128)
        # qubits = (control, target): r = b(c) + 2 b(t); control=1 rows are r = 1, 3
        m[1, 1], m[1, 3], m[3, 1], m[3, 3] = u[0, 0], u[0, 1], u[1, 0], u[1, 1]
        return m
    if k in ("SWAP", "RELABEL"):   # an Emulated-SWAP acts as a SWAP on hardware (Appendix B)
        return SWAP4.copy()
    raise ValueError(k)


def is_diagonal_on(g, q: int) -> bool:
    """True if the gate acts diagonally on qubit q (it commutes with Z on q)."""
    k = g.kind
    if k in ("RZ", "Z", "S", "T", "P", "CZ", "CP"):
        return True
    if k in ("CNOT", "CU"):
        return q == g.qubits[0] or (k == "CU" and _is_diag2(g.matrix))
    if k == "U1":
        return _is_diag2(g.matrix)
    return False


def _is_diag2(m) -> bool:
    m = np.asarray(m).reshape(2, 2)
    return m[0, 1] == 0 and m[1, 0] == 0

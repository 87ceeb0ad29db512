"""Python driver of the FP64 C oracle (test infrastructure only).

`OracleState` keeps 2^n complex128 amplitudes in a numpy array and applies the
workload's gates through the C routines of sv_oracle.c.  By default the state
is in logical order (alpha_i at index i, Sec. 2).  `run_storage_program`
executes a compiled instruction list in storage order: a gate on logical qubit
q acts on storage bit sigma(q) and PermuteQubits(sigma') rewrites the vector
from sigma to sigma' (Sec. 2, Appendix A).
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence

import numpy as np

from . import build as _build
from .gates import controlled_target_matrix, gate_full_matrix, one_qubit_matrix

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_init_zero.argtypes = [dp, ctypes.c_int]
        L.or_apply_1q.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int]
        L.or_apply_ctrl.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int]
        L.or_apply_2q.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int]
        L.or_apply_dense.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ip]
        L.or_permute.argtypes = [dp, dp, ctypes.c_int, ip, ip]
        L.or_to_logical.argtypes = [dp, dp, ctypes.c_int, ip]
        L.or_probabilities.argtypes = [dp, ctypes.c_int, dp]
        L.or_norm2.argtypes = [dp, ctypes.c_int]
        L.or_norm2.restype = ctypes.c_double
        L.or_inner.argtypes = [dp, dp, ctypes.c_int, dp]
        L.or_num_threads.restype = ctypes.c_int
        for f in ("or_init_zero", "or_apply_1q", "or_apply_ctrl", "or_apply_2q", "or_apply_dense",
                  "or_permute", "or_to_logical", "or_probabilities", "or_inner"):
            getattr(L, f).restype = None
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _mat(m: np.ndarray) -> np.ndarray:
    """complex matrix -> contiguous (re, im) doubles, row-major."""
    return np.ascontiguousarray(np.asarray(m, dtype=np.complex128)).view(np.float64).copy()


def num_threads() -> int:
    return int(lib().or_num_threads())


class OracleState:
    def __init__(self, n: int, psi: Optional[np.ndarray] = None):
        self.n = n
        if psi is None:
            self.psi = np.empty(1 << n, dtype=np.complex128)
            lib().or_init_zero(_dp(self.psi.view(np.float64)), n)
        else:
            self.psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()

    # -- primitive routines -------------------------------------------------
    def apply_1q(self, U, q: int, bit_of=None):
        lib().or_apply_1q(_dp(self.psi.view(np.float64)), self.n, _dp(_mat(U)), int(q))

    def apply_ctrl(self, U, c: int, t: int):
        lib().or_apply_ctrl(_dp(self.psi.view(np.float64)), self.n, _dp(_mat(U)), int(c), int(t))

    def apply_dense(self, U, qubits: Sequence[int]):
        qs = np.asarray(qubits, dtype=np.int32)
        lib().or_apply_dense(_dp(self.psi.view(np.float64)), self.n, _dp(_mat(U)), len(qs), _ip(qs))

    # -- gates ----------------------------------------------------------------
    def apply_gate(self, g, sigma: Optional[Sequence[int]] = None):
        """Apply one workload gate.  With `sigma`, the vector is in storage order
        under sigma and logical qubit q lives at storage bit sigma[q]."""
        pos = (lambda q: q) if sigma is None else (lambda q: int(sigma[q]))
        k = g.kind
        if len(g.qubits) == 1 and k != "UK":
            self.apply_1q(one_qubit_matrix(k, g.param, g.matrix), pos(g.qubits[0]))
        elif k in ("CNOT", "CZ", "CP", "CU"):
            self.apply_ctrl(controlled_target_matrix(k, g.param, g.matrix), pos(g.qubits[0]), pos(g.qubits[1]))
        else:
            self.apply_dense(gate_full_matrix(g), [pos(q) for q in g.qubits])

    def run(self, circuit: Iterable) -> "OracleState":
        for g in circuit:
            self.apply_gate(g)
        return self

    # -- read-outs -------------------------------------------------------------
    def probabilities(self) -> np.ndarray:
        p = np.empty(1 << self.n, dtype=np.float64)
        lib().or_probabilities(_dp(self.psi.view(np.float64)), self.n, _dp(p))
        return p

    def norm2(self) -> float:
        return float(lib().or_norm2(_dp(self.psi.view(np.float64)), self.n))


def simulate(n: int, circuit: Iterable) -> np.ndarray:
    """Logical-order FP64 amplitudes after `circuit` applied to |0...0>."""
    return OracleState(n).run(circuit).psi


def permute_storage(stored: np.ndarray, n: int, sigma: Sequence[int], sigma_new: Sequence[int]) -> np.ndarray:
    """PermuteQubits: the vector stored under sigma rewritten under sigma'."""
    a = np.ascontiguousarray(stored, dtype=np.complex128)
    out = np.empty_like(a)
    s0 = np.asarray(sigma, dtype=np.int32)
    s1 = np.asarray(sigma_new, dtype=np.int32)
    lib().or_permute(_dp(a.view(np.float64)), _dp(out.view(np.float64)), n, _ip(s0), _ip(s1))
    return out


def to_logical(stored: np.ndarray, n: int, sigma: Sequence[int]) -> np.ndarray:
    a = np.ascontiguousarray(stored, dtype=np.complex128)
    out = np.empty_like(a)
    s = np.asarray(sigma, dtype=np.int32)
    lib().or_to_logical(_dp(a.view(np.float64)), _dp(out.view(np.float64)), n, _ip(s))
    return out


def inner(a: np.ndarray, b: np.ndarray, n: int) -> complex:
    out = np.empty(2, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    lib().or_inner(_dp(a.view(np.float64)), _dp(b.view(np.float64)), n, _dp(out))
    return complex(out[0], out[1])


def logical_index(j: np.ndarray, sigma: Sequence[int]) -> np.ndarray:
    """Sec. 2's index map read backwards: the storage position j holds the amplitude of the
    logical index i with i_q = bit sigma(q) of j, i.e. j = j(i, sigma) = sum_q i_q 2^sigma(q).
    Vectorised over an array of positions (uint64)."""
    j = np.asarray(j, dtype=np.uint64)
    i = np.zeros_like(j)
    for q, p in enumerate(sigma):
        i |= ((j >> np.uint64(p)) & np.uint64(1)) << np.uint64(q)
    return i


def run_storage_program(n: int, program: Sequence, identity_start: bool = True) -> np.ndarray:
    """Execute a compiled instruction list in storage order and return the
    logical-order state.  Instructions: ("gate", Gate) or ("permute", sigma')."""
    sigma: List[int] = list(range(n))
    st = OracleState(n)   # |0..0> is the same vector under every sigma
    for ins in program:
        if ins[0] == "gate":
            st.apply_gate(ins[1], sigma)
        elif ins[0] == "permute":
            new = list(ins[1])
            st.psi = permute_storage(st.psi, n, sigma, new)
            sigma = new
        else:
            raise ValueError(ins[0])
    return to_logical(st.psi, n, sigma)


def fidelity_loss(a: np.ndarray, b: np.ndarray) -> float:
    """1 - |<a|b>|^2 for unit vectors, accumulated in FP64 (numpy vdot)."""
    ov = np.vdot(np.asarray(a, dtype=np.complex128), np.asarray(b, dtype=np.complex128))
    return float(1.0 - abs(ov) ** 2)

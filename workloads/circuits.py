"""Seeded synthetic circuit generators.

This module produces *inputs* only: lists of gates with logical qubit indices,
angles and (for randomly drawn unitaries) explicit matrices.  It applies no
gate to any state and holds none of the simulation arithmetic; both the FP64
oracle (``oracle/``) and the CUDA library consume the same ``Gate`` lists and
each interprets named gates through its own definitions.

Conventions (readings of the paper where it is silent):

* qubit ``q`` is bit ``q`` of the amplitude index, i = sum_q i_q 2^q (Sec. 2,
  representation of the state).
* two-qubit controlled gates list ``(control, target)``.
* ``U2`` / ``UK`` matrices use the row/column index r = sum_t b(q_t) 2^t, so the
  first listed qubit is the least significant bit of r.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Gate kinds understood by both the oracle and the library.
KINDS_1Q_NAMED = ("H", "X", "Y", "Z", "S", "T")       # fixed 1-qubit gates
KINDS_1Q_PARAM = ("RZ", "RX", "RY", "P")              # 1-qubit rotations / phase
KINDS = (
    "U1",      # arbitrary 2x2 unitary (matrix given)
    *KINDS_1Q_NAMED, *KINDS_1Q_PARAM,
    "CNOT",    # controlled-X, qubits (control, target)
    "CZ",      # controlled-Z, symmetric
    "CP",      # controlled phase diag(1,1,1,e^{i param}), qubits (control, target)
    "CU",      # controlled arbitrary 2x2 (matrix given), qubits (control, target)
    "SWAP",    # exchange of two qubits
    "U2",      # arbitrary 4x4 on (q0, q1), matrix given
    "UK",      # arbitrary 2^k x 2^k on k qubits, matrix given
    "RELABEL", # Emulated-SWAP (Appendix B): exchange two qubits' storage positions, no data moved
)


@dataclass
class Gate:
    kind: str
    qubits: Tuple[int, ...]
    param: float = 0.0
    matrix: Optional[np.ndarray] = field(default=None, repr=False)

    def __post_init__(self):
        if self.kind not in KINDS:
            raise ValueError(f"unknown gate kind {self.kind}")
        self.qubits = tuple(int(q) for q in self.qubits)
        if self.matrix is not None:
            self.matrix = np.ascontiguousarray(self.matrix, dtype=np.complex128)


Circuit = List[Gate]


def _uniform_angle(rng: np.random.Generator) -> float:
    return float(rng.uniform(0.0, 2.0 * math.pi))


def haar_2x2(rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(2) element, Zyczkowski-Kus parametrisation.

    U = e^{i a} [[e^{i p} cos f, e^{i c} sin f], [-e^{-i c} sin f, e^{-i p} cos f]]
    with sin^2 f ~ U(0,1) and a, p, c ~ U(0, 2 pi), drawn in that order.
    """
    u = rng.uniform(0.0, 1.0)
    a = _uniform_angle(rng)
    p = _uniform_angle(rng)
    c = _uniform_angle(rng)
    f = math.asin(math.sqrt(u))
    ea = complex(math.cos(a), math.sin(a))
    m = np.array(
        [[complex(math.cos(p), math.sin(p)) * math.cos(f), complex(math.cos(c), math.sin(c)) * math.sin(f)],
         [-complex(math.cos(c), -math.sin(c)) * math.sin(f), complex(math.cos(p), -math.sin(p)) * math.cos(f)]],
        dtype=np.complex128)
    return ea * m


def haar_unitary(dim: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(dim) via QR of a complex Ginibre matrix with phase fix."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return np.ascontiguousarray(q * (d / np.abs(d)))


def random_matching(n: int, rng: np.random.Generator) -> List[Tuple[int, int]]:
    """Random perfect matching of 0..n-1 (one qubit left over when n is odd):
    a uniform shuffle s, pairs (s[2k], s[2k+1]) with the first as control."""
    s = rng.permutation(n)
    return [(int(s[2 * k]), int(s[2 * k + 1])) for k in range(n // 2)]


def biased_pairs(n: int, rng: np.random.Generator) -> List[Tuple[int, int]]:
    """floor(n/4) disjoint qubit pairs biased toward high qubits: 2*floor(n/4)
    distinct qubits drawn without replacement with weight (q+1)^2, paired in
    draw order."""
    k = n // 4
    if k == 0:
        return []
    w = (np.arange(n, dtype=np.float64) + 1.0) ** 2
    drawn = rng.choice(n, size=2 * k, replace=False, p=w / w.sum())
    return [(int(drawn[2 * i]), int(drawn[2 * i + 1])) for i in range(k)]


# ---------------------------------------------------------------------------
# Workload constructions
# ---------------------------------------------------------------------------

def haar_cnot_circuit(n: int, layers: int, seed: int) -> Circuit:
    """n qubits, `layers` layers: a Haar-random 2x2 on every qubit (q = 0..n-1),
    then CNOTs on a random perfect matching.  Used at n=12, 20 layers."""
    rng = np.random.default_rng(seed)
    c: Circuit = []
    for _ in range(layers):
        for q in range(n):
            c.append(Gate("U1", (q,), matrix=haar_2x2(rng)))
        for a, b in random_matching(n, rng):
            c.append(Gate("CNOT", (a, b)))
    return c


def rzrx_cz_circuit(n: int, layers: int, seed: int) -> Circuit:
    """n qubits, `layers` layers: for q = 0..n-1 RZ(theta_q) then RX(phi_q) with
    angles U(0, 2 pi), then floor(n/4) CZ on pairs biased toward high qubits.
    Used at n=30 (40 layers), n=32/33 (30 layers)."""
    rng = np.random.default_rng(seed)
    c: Circuit = []
    for _ in range(layers):
        for q in range(n):
            c.append(Gate("RZ", (q,), param=_uniform_angle(rng)))
            c.append(Gate("RX", (q,), param=_uniform_angle(rng)))
        for a, b in biased_pairs(n, rng):
            c.append(Gate("CZ", (a, b)))
    return c


def mixed_batch_circuit(n: int, depth: int, rng: np.random.Generator) -> Circuit:
    """One circuit of the batched workload: per layer a Haar 2x2 on every qubit,
    then on a random matching each pair gets CNOT or CZ with probability 1/2."""
    c: Circuit = []
    for _ in range(depth):
        for q in range(n):
            c.append(Gate("U1", (q,), matrix=haar_2x2(rng)))
        for a, b in random_matching(n, rng):
            c.append(Gate("CNOT" if rng.uniform() < 0.5 else "CZ", (a, b)))
    return c


def batched_workload(count: int, seed: int, nmin: int = 10, nmax: int = 20,
                     dmin: int = 10, dmax: int = 60) -> List[Tuple[int, Circuit]]:
    """`count` circuits with n ~ U{nmin..nmax} and depth ~ U{dmin..dmax}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        d = int(rng.integers(dmin, dmax + 1))
        out.append((n, mixed_batch_circuit(n, d, rng)))
    return out


@dataclass
class Request:
    arrival_s: float
    n: int
    dtype: str          # "c64" or "c128"
    circuit: Circuit


def serving_workload(count: int, rate_hz: float, seed: int, nmin: int = 12, nmax: int = 28,
                     dmin: int = 20, dmax: int = 100) -> List[Request]:
    """Poisson arrivals at `rate_hz`; n = floor(exp(U(ln nmin, ln(nmax+1)))),
    depth ~ U{dmin..dmax}, dtype c64 / c128 with probability 1/2 each; gates as
    in `mixed_batch_circuit`."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n = int(math.floor(math.exp(rng.uniform(math.log(nmin), math.log(nmax + 1)))))
        n = min(max(n, nmin), nmax)
        d = int(rng.integers(dmin, dmax + 1))
        dt = "c64" if rng.uniform() < 0.5 else "c128"
        out.append(Request(t, n, dt, mixed_batch_circuit(n, d, rng)))
    return out


def paper_random_circuit(n: int, p: float, seed: int, ngates: Optional[int] = None) -> Circuit:
    """The random circuits of the numerical-results section: `ngates` (default
    30 n) gates, each a CNOT with probability p (uniform ordered pair of distinct
    qubits), otherwise H or Y with equal probability on a uniform qubit."""
    rng = np.random.default_rng(seed)
    if ngates is None:
        ngates = 30 * n
    c: Circuit = []
    for _ in range(ngates):
        if rng.uniform() < p:
            a = int(rng.integers(0, n))
            b = int(rng.integers(0, n - 1))
            if b >= a:
                b += 1
            c.append(Gate("CNOT", (a, b)))
        else:
            kind = "H" if rng.uniform() < 0.5 else "Y"
            c.append(Gate(kind, (int(rng.integers(0, n)),)))
    return c


def qft_like_circuit(n: int) -> Circuit:
    """QFT-shaped circuit with each controlled-Rz replaced by a CNOT
    (Appendix C): for j = n-1 down to 0, H on j, then CNOT(control k, target j)
    for k = j-1 down to 0.  No final qubit reversal."""
    c: Circuit = []
    for j in range(n - 1, -1, -1):
        c.append(Gate("H", (j,)))
        for k in range(j - 1, -1, -1):
            c.append(Gate("CNOT", (k, j)))
    return c


def qft_circuit(n: int) -> Circuit:
    """Textbook QFT with controlled phases and the final qubit reversal (SWAPs)."""
    c: Circuit = []
    for j in range(n - 1, -1, -1):
        c.append(Gate("H", (j,)))
        for k in range(j - 1, -1, -1):
            c.append(Gate("CP", (k, j), param=math.pi / (1 << (j - k))))
    for j in range(n // 2):
        c.append(Gate("SWAP", (j, n - 1 - j)))
    return c


def single_qubit_run_circuit(n: int, layers: int, seed: int) -> Circuit:
    """Long runs of single-qubit gates on each qubit, for gate-fusion tests: per layer and
    qubit one of a Haar 2x2, RZ + RX, S + T + P (diagonal only), H + H (identity product),
    X + RZ + X (diagonal product), RY + Y; every third layer one CNOT, CZ or SWAP on two of
    the upper half of the qubits interrupts their runs."""
    rng = np.random.default_rng(seed)
    c: Circuit = []
    for layer in range(layers):
        for q in range(n):
            k = int(rng.integers(0, 6))
            if k == 0:
                c.append(Gate("U1", (q,), matrix=haar_2x2(rng)))
            elif k == 1:
                c += [Gate("RZ", (q,), param=_uniform_angle(rng)), Gate("RX", (q,), param=_uniform_angle(rng))]
            elif k == 2:
                c += [Gate("S", (q,)), Gate("T", (q,)), Gate("P", (q,), param=_uniform_angle(rng))]
            elif k == 3:
                c += [Gate("H", (q,)), Gate("H", (q,))]
            elif k == 4:
                c += [Gate("X", (q,)), Gate("RZ", (q,), param=_uniform_angle(rng)), Gate("X", (q,))]
            else:
                c += [Gate("RY", (q,), param=_uniform_angle(rng)), Gate("Y", (q,))]
        if layer % 3 == 2 and n >= 4:
            a, b = rng.choice(np.arange(n // 2, n), 2, replace=False)
            c.append(Gate(str(rng.choice(["CNOT", "CZ", "SWAP"])), (int(a), int(b))))
    return c


def random_mixed_circuit(n: int, ngates: int, seed: int, kinds: Sequence[str] = None,
                         kmax: int = 3) -> Circuit:
    """Random circuit drawing every gate kind (for parity tests)."""
    rng = np.random.default_rng(seed)
    if kinds is None:
        kinds = [k for k in KINDS if k != "RELABEL"]
    c: Circuit = []
    for _ in range(ngates):
        kind = kinds[int(rng.integers(0, len(kinds)))]
        if kind in ("CNOT", "CZ", "CP", "CU", "SWAP", "U2") and n < 2:
            kind = "H"
        if kind == "U1":
            c.append(Gate("U1", (int(rng.integers(0, n)),), matrix=haar_2x2(rng)))
        elif kind in KINDS_1Q_NAMED:
            c.append(Gate(kind, (int(rng.integers(0, n)),)))
        elif kind in KINDS_1Q_PARAM:
            c.append(Gate(kind, (int(rng.integers(0, n)),), param=_uniform_angle(rng)))
        elif kind in ("CNOT", "CZ", "SWAP"):
            a, b = rng.choice(n, size=2, replace=False)
            c.append(Gate(kind, (int(a), int(b))))
        elif kind == "CP":
            a, b = rng.choice(n, size=2, replace=False)
            c.append(Gate("CP", (int(a), int(b)), param=_uniform_angle(rng)))
        elif kind == "CU":
            a, b = rng.choice(n, size=2, replace=False)
            c.append(Gate("CU", (int(a), int(b)), matrix=haar_2x2(rng)))
        elif kind == "U2":
            a, b = rng.choice(n, size=2, replace=False)
            c.append(Gate("U2", (int(a), int(b)), matrix=haar_unitary(4, rng)))
        elif kind == "UK":
            k = int(rng.integers(1, min(kmax, n) + 1))
            qs = rng.choice(n, size=k, replace=False)
            c.append(Gate("UK", tuple(int(x) for x in qs), matrix=haar_unitary(1 << k, rng)))
    return c


def random_permutation(n: int, rng: np.random.Generator) -> List[int]:
    return [int(x) for x in rng.permutation(n)]

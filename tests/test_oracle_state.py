"""Pins of the FP64 state-vector oracle against facts that do not come from it.

* gate definitions vs. matrix exponentials / algebraic identities (scipy, numpy);
* every gate routine vs. a dense 2^n x 2^n matrix built entry by entry from the
  embedding definition <i|M|j> = U[r(i), r(j)] when i, j agree off the gate's
  qubits (textbook linear algebra), for n <= 7;
* closed forms: X|0>=|1>, GHZ, QFT of basis states, norm preservation, mirror
  circuits C C^dagger |0> = |0>.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import gates as og
from oracle import sv
from workloads import circuits as wc

PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)


# ---------------------------------------------------------------------------
# gate definitions
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("theta", [0.0, 0.3, 1.7, math.pi, 5.9])
def test_rotations_are_matrix_exponentials(theta):
    for kind, P in (("RX", PX), ("RY", PY), ("RZ", PZ)):
        ref = scipy.linalg.expm(-0.5j * theta * P)
        np.testing.assert_allclose(og.one_qubit_matrix(kind, theta), ref, atol=1e-15, rtol=0)
    np.testing.assert_allclose(og.one_qubit_matrix("P", theta), np.diag([1, np.exp(1j * theta)]), atol=1e-15)


def test_fixed_gate_identities():
    H = og.one_qubit_matrix("H")
    np.testing.assert_allclose(H, (PX + PZ) / math.sqrt(2), atol=1e-16)
    np.testing.assert_allclose(og.one_qubit_matrix("X"), PX)
    np.testing.assert_allclose(og.one_qubit_matrix("Y"), PY)
    np.testing.assert_allclose(og.one_qubit_matrix("Z"), PZ)
    S = og.one_qubit_matrix("S")
    T = og.one_qubit_matrix("T")
    np.testing.assert_allclose(S @ S, PZ, atol=1e-16)
    np.testing.assert_allclose(T @ T, S, atol=1e-15)


def test_two_qubit_truth_tables():
    # index r = b(q0) + 2 b(q1); CNOT(q0 = control, q1 = target)
    cnot = og.gate_full_matrix(wc.Gate("CNOT", (0, 1)))
    # |c=1,t=0> (r=1) -> |c=1,t=1> (r=3)
    e = np.eye(4)
    np.testing.assert_allclose(cnot @ e[1], e[3])
    np.testing.assert_allclose(cnot @ e[3], e[1])
    np.testing.assert_allclose(cnot @ e[0], e[0])
    np.testing.assert_allclose(cnot @ e[2], e[2])
    cz = og.gate_full_matrix(wc.Gate("CZ", (0, 1)))
    np.testing.assert_allclose(np.diag(cz), [1, 1, 1, -1])
    sw = og.gate_full_matrix(wc.Gate("SWAP", (0, 1)))
    np.testing.assert_allclose(sw @ e[1], e[2])
    np.testing.assert_allclose(sw @ e[2], e[1])


def test_haar_generator_is_unitary_and_spread():
    rng = np.random.default_rng(5)
    us = [wc.haar_2x2(rng) for _ in range(4000)]
    for u in us[:50]:
        np.testing.assert_allclose(u @ u.conj().T, np.eye(2), atol=1e-14)
    # Haar measure: |U00|^2 ~ U(0,1) -> mean 1/2, variance 1/12
    a = np.array([abs(u[0, 0]) ** 2 for u in us])
    assert abs(a.mean() - 0.5) < 0.02 and abs(a.var() - 1 / 12) < 0.01


# ---------------------------------------------------------------------------
# dense embedding built entry by entry
# ---------------------------------------------------------------------------
def dense_embedding(n, U, qubits):
    """<i|M|j> = U[r(i), r(j)] if i and j agree on all other bits, else 0,
    with r(x) = sum_t bit(x, qubits[t]) 2^t."""
    N = 1 << n
    mask = 0
    for q in qubits:
        mask |= 1 << q
    idx = np.arange(N)
    r = np.zeros(N, dtype=np.int64)
    for t, q in enumerate(qubits):
        r |= ((idx >> q) & 1) << t
    same = (idx[:, None] & ~mask) == (idx[None, :] & ~mask)
    M = np.where(same, np.asarray(U)[r[:, None], r[None, :]], 0)
    return M


def dense_gate_matrix(n, g):
    return dense_embedding(n, og.gate_full_matrix(g), g.qubits)


def test_dense_embedding_small_loops():
    """The vectorised embedding agrees with explicit python loops (n = 3)."""
    rng = np.random.default_rng(0)
    U = wc.haar_unitary(4, rng)
    n, qs = 3, (2, 0)
    M = dense_embedding(n, U, qs)
    for i in range(8):
        for j in range(8):
            if (i & ~0b101) == (j & ~0b101):
                ri = ((i >> 2) & 1) | (((i >> 0) & 1) << 1)
                rj = ((j >> 2) & 1) | (((j >> 0) & 1) << 1)
                assert M[i, j] == U[ri, rj]
            else:
                assert M[i, j] == 0


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("seed", [1, 2])
def test_oracle_matches_dense_products(n, seed):
    circ = wc.random_mixed_circuit(n, 40, seed=seed + 100 * n, kmax=min(3, n))
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    for g in circ:
        psi = dense_gate_matrix(n, g) @ psi
    got = sv.simulate(n, circ)
    np.testing.assert_allclose(got, psi, atol=1e-13, rtol=0)


@pytest.mark.parametrize("kind", ["U1", "H", "X", "Y", "Z", "S", "T", "RZ", "RX", "RY", "P",
                                  "CNOT", "CZ", "CP", "CU", "SWAP", "U2", "UK"])
def test_each_gate_kind_on_random_state(kind):
    n = 6
    rng = np.random.default_rng(sum(map(ord, kind)))
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    circ = wc.random_mixed_circuit(n, 12, seed=7, kinds=[kind], kmax=4)
    st = sv.OracleState(n, psi)
    ref = psi.copy()
    for g in circ:
        st.apply_gate(g)
        ref = dense_gate_matrix(n, g) @ ref
    np.testing.assert_allclose(st.psi, ref, atol=1e-14, rtol=0)


# ---------------------------------------------------------------------------
# closed forms and invariants
# ---------------------------------------------------------------------------
def test_basis_flips():
    n = 4
    for q in range(n):
        psi = sv.simulate(n, [wc.Gate("X", (q,))])
        e = np.zeros(1 << n)
        e[1 << q] = 1
        np.testing.assert_array_equal(psi, e)


@pytest.mark.parametrize("n", [2, 5, 10])
def test_ghz(n):
    circ = [wc.Gate("H", (0,))] + [wc.Gate("CNOT", (0, k)) for k in range(1, n)]
    psi = sv.simulate(n, circ)
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, ref, atol=1e-15, rtol=0)


@pytest.mark.parametrize("n", [3, 6, 9])
def test_qft_of_basis_states(n):
    """QFT |x> = 2^{-n/2} sum_y exp(2 pi i x y / 2^n) |y>."""
    N = 1 << n
    for x in (0, 1, 5 % N, N - 1):
        prep = [wc.Gate("X", (q,)) for q in range(n) if (x >> q) & 1]
        psi = sv.simulate(n, prep + wc.qft_circuit(n))
        y = np.arange(N)
        ref = np.exp(2j * np.pi * x * y / N) / math.sqrt(N)
        np.testing.assert_allclose(psi, ref, atol=1e-13, rtol=0)


def test_norm_preserved_and_mirror():
    n = 12
    circ = wc.haar_cnot_circuit(n, 20, seed=3)
    st = sv.OracleState(n).run(circ)
    assert abs(st.norm2() - 1.0) < 1e-13
    # mirror: apply C^dagger gate by gate in reverse order
    inv = []
    for g in reversed(circ):
        if g.kind == "U1":
            inv.append(wc.Gate("U1", g.qubits, matrix=g.matrix.conj().T))
        else:
            inv.append(g)   # CNOT is self-inverse
    st.run(inv)
    e0 = np.zeros(1 << n)
    e0[0] = 1
    np.testing.assert_allclose(st.psi, e0, atol=1e-13, rtol=0)


def test_probabilities_and_inner():
    n = 8
    psi = sv.simulate(n, wc.random_mixed_circuit(n, 30, seed=11))
    st = sv.OracleState(n, psi)
    np.testing.assert_allclose(st.probabilities(), np.abs(psi) ** 2, atol=1e-16)
    assert abs(sv.inner(psi, psi, n) - 1.0) < 1e-13
    phi = sv.simulate(n, wc.random_mixed_circuit(n, 30, seed=12))
    np.testing.assert_allclose(sv.inner(psi, phi, n), np.vdot(psi, phi), atol=1e-14)

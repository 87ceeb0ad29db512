"""Pins of the oracle's PermuteQubits against brute force of the storage-index
definition j(i, sigma) = sum_q i_q 2^{sigma(q)} (Sec. 2)."""
import itertools

import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc


def brute_store(psi_logical, n, sigma):
    """v[j(i, sigma)] = alpha_i written with an explicit double loop over bits."""
    v = np.zeros_like(psi_logical)
    for i in range(1 << n):
        j = 0
        for q in range(n):
            if (i >> q) & 1:
                j += 2 ** sigma[q]
        v[j] = psi_logical[i]
    return v


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_permute_all_sigma_pairs_small(n):
    rng = np.random.default_rng(n)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    perms = list(itertools.permutations(range(n)))
    for s0 in perms:
        v0 = brute_store(psi, n, s0)
        np.testing.assert_array_equal(sv.to_logical(v0, n, s0), psi)
        for s1 in perms[:: max(1, len(perms) // 6)]:
            v1 = sv.permute_storage(v0, n, s0, s1)
            np.testing.assert_array_equal(v1, brute_store(psi, n, s1))


def test_permute_all_sigma_n6():
    n = 6
    rng = np.random.default_rng(6)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    ident = list(range(n))
    for s in itertools.permutations(range(n)):
        got = sv.permute_storage(psi, n, ident, s)
        np.testing.assert_array_equal(got, brute_store(psi, n, s))


@pytest.mark.parametrize("n", [10, 16])
def test_permute_inverse_is_identity_bitwise(n):
    rng = np.random.default_rng(n)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    s0 = wc.random_permutation(n, rng)
    s1 = wc.random_permutation(n, rng)
    v0 = sv.permute_storage(psi, n, list(range(n)), s0)
    v1 = sv.permute_storage(v0, n, s0, s1)
    back = sv.permute_storage(v1, n, s1, s0)
    assert back.tobytes() == v0.tobytes()
    assert sv.to_logical(v1, n, s1).tobytes() == psi.tobytes()


def test_gates_in_storage_order_match_logical():
    """A circuit run in storage order (gate on q acts on bit sigma(q)) with
    permutations interleaved gives the logical-order result."""
    n = 7
    rng = np.random.default_rng(3)
    circ = wc.random_mixed_circuit(n, 60, seed=9)
    prog = []
    for k, g in enumerate(circ):
        if k % 10 == 5:
            prog.append(("permute", wc.random_permutation(n, rng)))
        prog.append(("gate", g))
    got = sv.run_storage_program(n, prog)
    ref = sv.simulate(n, circ)
    np.testing.assert_allclose(got, ref, atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_logical_index_against_brute_force(n):
    """sv.logical_index (the storage -> logical map the full-size GPU permutation tests use)
    agrees with the brute-force j(i, sigma) loop for every sigma at these sizes."""
    ident = np.arange(1 << n, dtype=np.float64).astype(np.complex128)
    j = np.arange(1 << n, dtype=np.uint64)
    for s in itertools.permutations(range(n)):
        stored = brute_store(ident, n, s)          # stored[j(i, s)] = i
        np.testing.assert_array_equal(sv.logical_index(j, s), stored.real.astype(np.uint64))


def test_logical_index_high_bits():
    """Positions past 2^32 (a 36-qubit index space) map through every bit."""
    n = 36
    rng = np.random.default_rng(36)
    s = wc.random_permutation(n, rng)
    i = rng.integers(0, 1 << n, 1000, dtype=np.uint64)
    j = np.zeros_like(i)
    for q in range(n):
        j |= ((i >> np.uint64(q)) & np.uint64(1)) << np.uint64(s[q])
    np.testing.assert_array_equal(sv.logical_index(j, s), i)

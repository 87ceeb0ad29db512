"""Pins of the oracle's compiler-side algorithms (Sec. 3, Sec. 4, Appendix A/C).

* the commutation-pruned DAG: every linear extension simulates to the same
  state (checked on the FP64 state-vector oracle, itself pinned by dense
  products);
* Algorithm 1: the emitted program is a linear extension, it simulates to the
  original state in storage order, it terminates, and on the paper's random
  circuits it reproduces the printed communication statistics (~20% -> ~3.5%,
  Sec. 4, Fig. 3) and the Appendix C bound of 2(n-m) permutations;
* Algorithm 2: the stated invariants by brute force over all (sigma, sigma');
* the 8.5x model arithmetic printed in Sec. 4 (49.5%, 60%).
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import compiler_ref as cr
from oracle import sv
from workloads import circuits as wc

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def random_topo_order(preds, rng):
    G = len(preds)
    npred = [len(p) for p in preds]
    succ = [[] for _ in range(G)]
    for j, ps in enumerate(preds):
        for i in ps:
            succ[i].append(j)
    ready = [v for v in range(G) if npred[v] == 0]
    out = []
    while ready:
        k = int(rng.integers(0, len(ready)))
        v = ready.pop(k)
        out.append(v)
        for s in succ[v]:
            npred[s] -= 1
            if npred[s] == 0:
                ready.append(s)
    assert len(out) == G
    return out


@pytest.mark.parametrize("seed", range(6))
def test_dag_linear_extensions_are_equivalent(seed):
    n = 5
    kinds = ["RZ", "RX", "H", "CNOT", "CZ", "CP", "X", "Z", "S", "SWAP", "U1", "CU"]
    circ = wc.random_mixed_circuit(n, 50, seed=seed, kinds=kinds)
    preds = cr.build_dag(circ)
    ref = sv.simulate(n, circ)
    rng = np.random.default_rng(seed)
    for _ in range(5):
        order = random_topo_order(preds, rng)
        got = sv.simulate(n, [circ[v] for v in order])
        np.testing.assert_allclose(got, ref, atol=1e-13, rtol=0)


def test_dag_drops_commuting_edges():
    c = [wc.Gate("RZ", (0,), param=0.1), wc.Gate("CZ", (0, 1)), wc.Gate("CNOT", (0, 2)),
         wc.Gate("RX", (2,), param=0.2), wc.Gate("CNOT", (1, 2)), wc.Gate("H", (2,))]
    preds = cr.build_dag(c)
    # Z-type actions on q0/q1 commute, X-type actions on q2 commute: no edges
    assert preds[:5] == [[], [], [], [], []]
    # H on q2 commutes with nothing there
    assert preds[5] == [2, 3, 4]


def _check_program_valid(circ, prog, n, m):
    preds = cr.build_dag(circ)
    pos = {}
    sigma = list(range(n))
    for k, ins in enumerate(prog):
        if ins[0] == "gate":
            v, comm = ins[1], ins[2]
            assert v not in pos
            pos[v] = k
            for p in preds[v]:
                assert p in pos, "dependency violated"
            assert comm == (not cr.is_local(circ[v], sigma, m))
        else:
            new = ins[1]
            diff = [q for q in range(n) if new[q] != sigma[q]]
            assert len(diff) == 2, "one transposition per PermuteQubits"
            a, b = diff
            assert (sigma[a] < m) != (sigma[b] < m), "local <-> global exchange"
            sigma = list(new)
    assert len(pos) == len(circ)


@pytest.mark.parametrize("scoring", ["closure", "frontier"])
@pytest.mark.parametrize("seed", range(4))
def test_alg1_program_simulates_to_original(scoring, seed):
    n, m = 9, 6
    circ = wc.random_mixed_circuit(n, 80, seed=seed, kinds=["H", "Y", "CNOT", "RZ", "RX", "CZ", "U1", "CU", "U2"])
    prog, st = cr.alg1(n, m, circ, scoring=scoring)
    _check_program_valid(circ, prog, n, m)
    storage_prog = [("gate", circ[i[1]]) if i[0] == "gate" else i for i in prog]
    got = sv.run_storage_program(n, storage_prog)
    np.testing.assert_allclose(got, sv.simulate(n, circ), atol=1e-13, rtol=0)


def test_alg1_on_paper_random_circuits_small():
    n, m = 12, 9
    for p in (0.0, 0.3, 1.0):
        for seed in range(3):
            circ = wc.paper_random_circuit(n, p, seed)
            prog, st = cr.alg1(n, m, circ)
            _check_program_valid(circ, prog, n, m)
            storage_prog = [("gate", circ[i[1]]) if i[0] == "gate" else i for i in prog]
            got = sv.run_storage_program(n, storage_prog)
            np.testing.assert_allclose(got, sv.simulate(n, circ), atol=1e-12, rtol=0)
            assert st["comm_fraction"] <= cr.original_comm_fraction(n, m, circ)


@pytest.mark.parametrize("n", [35, 50])
def test_fig3_communication_fractions(n):
    """1/5 of the qubits global, p = 0.3, 30 n gates, 20 circuits:
    ~20% of the gates communicate before the pass and ~3.5% after (Sec. 4)."""
    m = n - n // 5
    orig, opt = [], []
    for seed in range(20):
        circ = wc.paper_random_circuit(n, 0.3, seed)
        orig.append(cr.original_comm_fraction(n, m, circ))
        _, st = cr.alg1(n, m, circ, scoring="closure")
        opt.append(st["comm_fraction"])
    g0 = GOLDEN["comm_fraction_original_1to5_p03"]["value"]
    g1 = GOLDEN["comm_fraction_optimized_1to5_p03"]["value"]
    assert abs(np.mean(orig) - g0) < 0.01
    assert abs(np.mean(opt) - g1) < 0.01


def test_literal_scoring_does_not_terminate():
    """Taken literally (count every remaining vertex, threshold 0) the search
    can permute forever without unblocking a frontier gate."""
    circ = wc.paper_random_circuit(35, 1.0, 0)
    with pytest.raises(RuntimeError):
        cr.alg1(35, 28, circ, scoring="literal", max_steps=3000)


@pytest.mark.parametrize("n", [5, 10, 20, 30])
def test_appendix_c_qft_like_bound(n):
    m = n - max(1, n // 5)
    circ = wc.qft_like_circuit(n)
    prog, st = cr.alg1(n, m, circ)
    assert st["n_permutes"] <= 2 * (n - m)
    assert st["n_comm_gates"] == 0


def test_model_arithmetic():
    assert abs(cr.model_reduction(0.2, 0.035) - GOLDEN["model_reduction_at_3p5"]["value"]) < 0.001
    assert abs(cr.model_reduction(0.2, 0.0) - GOLDEN["model_reduction_no_comm"]["value"]) < 1e-12
    # the printed expression itself
    assert abs((1 - (0.965 + 0.035 * 8.5) / (0.8 + 0.2 * 8.5)) - 0.495) < 1e-12


def _inv(s):
    r = [0] * len(s)
    for q, p in enumerate(s):
        r[p] = q
    return r


def _check_alg2(n, m, s, t):
    s1, s2 = cr.alg2(n, m, s, t)
    assert sorted(s1) == list(range(n)) and sorted(s2) == list(range(n))
    inv, inv1, inv2 = _inv(s), _inv(s1), _inv(s2)
    # step 1: global positions untouched, local set unchanged
    assert all(inv1[p] == inv[p] for p in range(m, n))
    # step 2: local positions untouched
    assert all(inv2[p] == inv1[p] for p in range(m))
    # qubits local (global) in both sigma and sigma' are in place after step 1 (2)
    for q in range(n):
        if s[q] < m and t[q] < m:
            assert s1[q] == t[q]
        if s[q] >= m and t[q] >= m:
            assert s2[q] == t[q]
    # step 3: only local <-> global transpositions
    for q in range(n):
        if s2[q] != t[q]:
            p_from, p_to = s2[q], t[q]
            assert (p_from < m) != (p_to < m)
            partner = inv2[p_to]
            assert t[partner] == p_from


@pytest.mark.parametrize("n", [3, 4, 5])
def test_alg2_all_pairs(n):
    perms = list(itertools.permutations(range(n)))
    for m in range(1, n):
        for s in perms:
            for t in perms:
                _check_alg2(n, m, list(s), list(t))


def test_alg2_random_large():
    rng = np.random.default_rng(0)
    for _ in range(500):
        n = int(rng.integers(6, 40))
        m = int(rng.integers(1, n))
        _check_alg2(n, m, wc.random_permutation(n, rng), wc.random_permutation(n, rng))


def test_alg2_composition_on_states():
    """sigma -> sigma1 -> sigma2 -> sigma' applied to a stored vector gives the
    same bytes as the direct permutation."""
    n, m = 8, 5
    rng = np.random.default_rng(1)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    for _ in range(10):
        s = wc.random_permutation(n, rng)
        t = wc.random_permutation(n, rng)
        v = sv.permute_storage(psi, n, list(range(n)), s)
        s1, s2 = cr.alg2(n, m, s, t)
        a = sv.permute_storage(v, n, s, s1)
        a = sv.permute_storage(a, n, s1, s2)
        a = sv.permute_storage(a, n, s2, t)
        assert a.tobytes() == sv.permute_storage(v, n, s, t).tobytes()

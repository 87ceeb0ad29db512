"""GPU parity: the CUDA path against the FP64 oracle on the same seeded inputs.

Tolerances (stated requirements of the hot path):
  complex128 (double-float or native FP64 arithmetic): fidelity loss 1-|<gpu|oracle>|^2
  <= 1e-10 and max |amplitude difference| <= 1e-12;
  complex64: fidelity loss <= 1e-5 (and max difference <= 1e-5, derived from FP32 rounding
  ~6e-8 per operation over a few hundred gates on unit-norm states);
  permutations: bit-exact.
"""

import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")

TOL = {"c128": (1e-10, 1e-12), "c64": (1e-5, 1e-5)}


def check(got, ref, dtype):
    fid_tol, amp_tol = TOL[dtype]
    got = np.asarray(got, dtype=np.complex128)
    err = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    fid = sv.fidelity_loss(got, ref)
    assert err <= amp_tol, f"max amplitude error {err:.3e} > {amp_tol}"
    assert fid <= fid_tol, f"fidelity loss {fid:.3e} > {fid_tol}"
    return err, fid


MODES = [("c128", "df"), ("c128", "f64"), ("c64", "auto")]


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("kind", ["U1", "H", "X", "Y", "Z", "S", "T", "RZ", "RX", "RY", "P", "CNOT", "CZ", "CP",
                                  "CU", "SWAP", "U2", "UK"])
def test_pergate_each_kind(dtype, arith, kind):
    n = 11
    circ = wc.random_mixed_circuit(n, 24, seed=sum(map(ord, kind)), kinds=[kind], kmax=5)
    # start from a spread state so that every amplitude is exercised
    prep = [wc.Gate("H", (q,)) for q in range(n)] + [wc.Gate("RZ", (q,), param=0.37 * (q + 1)) for q in range(n)]
    st = qs.State(n, dtype, arith=arith)
    st.run(prep + circ, mode="pergate")
    check(st.amplitudes(), sv.simulate(n, prep + circ), dtype)


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13])
def test_pergate_apply_calls(dtype, arith, n):
    rng = np.random.default_rng(n)
    st = qs.State(n, dtype, arith=arith)
    ref = sv.OracleState(n)
    for k in range(30):
        q = int(rng.integers(0, n))
        U = wc.haar_2x2(rng)
        st.apply_1q(U, q)
        ref.apply_1q(U, q)
        if n >= 2:
            a, b = (int(x) for x in rng.choice(n, 2, replace=False))
            U2 = wc.haar_unitary(4, rng)
            st.apply_2q(U2, a, b)
            ref.apply_dense(U2, [a, b])
            st.apply_controlled(U, b, a)
            ref.apply_ctrl(U, b, a)
        if n >= 3 and k % 5 == 0:
            qq = [int(x) for x in rng.choice(n, 3, replace=False)]
            U3 = wc.haar_unitary(8, rng)
            st.apply_dense(U3, qq)
            ref.apply_dense(U3, qq)
    check(st.amplitudes(), ref.psi, dtype)


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n,L,c", [(6, 4, 1), (9, 6, 2), (12, 8, 3), (14, 10, 3), (16, 12, 3), (16, 13, 4)])
def test_tile_mode_random_circuits(dtype, arith, n, L, c):
    circ = wc.random_mixed_circuit(n, 150, seed=n * 31 + L, kmax=min(4, L - c))
    st = qs.State(n, dtype, arith=arith)
    plan = qs.compile(n, circ, mode="tile", dtype=dtype, arith=arith, tile_bits=L, low_bits=c)
    st.execute(plan)
    check(st.amplitudes(), sv.simulate(n, circ), dtype)


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n,m", [(10, 6), (13, 9), (16, 12)])
def test_paper_mode(dtype, arith, n, m):
    circ = wc.paper_random_circuit(n, 0.3, seed=n) + wc.rzrx_cz_circuit(n, 3, seed=n)
    st = qs.State(n, dtype, arith=arith)
    plan = qs.compile(n, circ, mode="paper", dtype=dtype, arith=arith, tile_bits=m)
    assert plan.stats()["n_permutes"] > 0
    st.execute(plan)
    assert st.permutation() == plan.final_permutation()
    check(st.amplitudes(), sv.simulate(n, circ), dtype)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_config1_12q_haar_cnot(dtype, arith):
    """12 qubits, 20 layers of Haar 2x2 on every qubit + CNOT perfect matching."""
    n = 12
    for seed in range(3):
        circ = wc.haar_cnot_circuit(n, 20, seed)
        ref = sv.simulate(n, circ)
        for mode in ("pergate", "tile", "paper"):
            st = qs.State(n, dtype, arith=arith)
            kw = {"tile_bits": 8} if mode == "paper" else {}
            st.run(circ, mode=mode, **kw)
            check(st.amplitudes(), ref, dtype)


@pytest.mark.parametrize("dtype,arith", [("c128", "df"), ("c64", "auto")])
@pytest.mark.parametrize("n", [20, 22])
def test_rzrx_cz_construction_medium(dtype, arith, n):
    """The 30-qubit workload's construction at a size the oracle finishes in seconds,
    several tiles per pass and a ragged last pass."""
    circ = wc.rzrx_cz_circuit(n, 40, seed=1)
    ref = sv.simulate(n, circ)
    st = qs.State(n, dtype, arith=arith)
    st.run(circ, mode="tile")
    check(st.amplitudes(), ref, dtype)
    if dtype == "c128":
        st2 = qs.State(n, dtype, arith=arith)
        st2.run(circ[:300], mode="pergate")
        check(st2.amplitudes(), sv.simulate(n, circ[:300]), dtype)


@pytest.mark.parametrize("store", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 10, 15, 20])
def test_permute_bit_exact(store, n):
    rng = np.random.default_rng(100 + n)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    dt = np.complex128 if store == "c128" else np.complex64
    psi = psi.astype(dt)
    st = qs.State(n, store)
    st.set_amplitudes(psi)          # stored under the identity
    sigma = list(range(n))
    cur = psi.astype(np.complex128)
    for _ in range(4):
        new = wc.random_permutation(n, rng)
        st.permute(new)
        cur = sv.permute_storage(cur, n, sigma, new)
        sigma = new
        got = st.amplitudes(order=qs.QS_ORDER_STORAGE)
        assert got.tobytes() == cur.astype(dt).tobytes()
        # logical read-out unchanged by any permutation
        assert st.amplitudes(order=qs.QS_ORDER_LOGICAL).tobytes() == psi.tobytes()
    st.permute(list(range(n)))
    assert st.amplitudes(order=qs.QS_ORDER_STORAGE).tobytes() == psi.tobytes()


def test_permute_rejects_non_permutation():
    st = qs.State(4, "c128")
    with pytest.raises(qs.QSError):
        st.permute([0, 1, 1, 2])
    with pytest.raises(qs.QSError):
        st.permute([0, 1, 2, 4])


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_gates_after_permute(dtype):
    n = 12
    rng = np.random.default_rng(3)
    circ = wc.random_mixed_circuit(n, 80, seed=4, kmax=3)
    st = qs.State(n, dtype)
    st.run(circ[:40], mode="pergate")
    st.permute(wc.random_permutation(n, rng))
    st.run(circ[40:60], mode="tile")
    st.permute(wc.random_permutation(n, rng))
    st.run(circ[60:], mode="paper", tile_bits=7)
    check(st.amplitudes(), sv.simulate(n, circ), dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_readouts(dtype):
    n = 14
    circ = wc.random_mixed_circuit(n, 60, seed=8)
    ref = sv.simulate(n, circ)
    st = qs.State(n, dtype)
    st.run(circ, mode="tile")
    st.permute(wc.random_permutation(n, np.random.default_rng(1)))
    p = st.probabilities()
    tol = 1e-12 if dtype == "c128" else 1e-6
    np.testing.assert_allclose(p, np.abs(ref) ** 2, atol=tol, rtol=0)
    ps = st.probabilities(order=qs.QS_ORDER_STORAGE)
    np.testing.assert_allclose(np.sort(ps), np.sort(p), atol=0, rtol=0)
    assert abs(st.norm() - 1.0) < (1e-12 if dtype == "c128" else 1e-5)
    a = st.amplitudes(first=100, count=37)
    np.testing.assert_allclose(a, ref[100:137], atol=10 * tol, rtol=0)


def test_df_conversion_round_trip():
    """double -> (hi, lo) floats -> double inside a tile pass loses at most 2^-46 relative."""
    n = 16
    rng = np.random.default_rng(9)
    mags = 10.0 ** rng.uniform(-30, 0, 1 << n)
    psi = mags * np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << n))
    psi[:7] = [0, 1, -1, 1j, 2 ** -60, 1e-37, 0.5]
    st = qs.State(n, "c128", arith="df")
    st.set_amplitudes(psi)
    st.run([wc.Gate("X", (0,)), wc.Gate("X", (0,))], mode="tile", tile_bits=10)
    got = st.amplitudes(order=qs.QS_ORDER_STORAGE)
    # per real component: |err| <= 2^-46 |x| + 2^-120 (the low word flushes below the float range)
    for a, b in ((got.real, psi.real), (got.imag, psi.imag)):
        assert np.all(np.abs(a - b) <= 2.0 ** -46 * np.abs(b) + 2.0 ** -120)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_appendix_b_export_runs_as_permutations(dtype):
    """The exported SWAP + Emulated-SWAP list run per gate on the GPU: SWAP moves data,
    RELABEL changes sigma, and the logical state is the original circuit's."""
    n, m = 11, 8
    circ = wc.paper_random_circuit(n, 0.3, seed=4)
    plan = qs.compile(n, circ, mode="paper", tile_bits=m)
    ir = plan.export_swaps(circ)
    st = qs.State(n, dtype)
    st.run(ir, mode="pergate")
    assert st.permutation() == plan.final_permutation()
    check(st.amplitudes(), sv.simulate(n, circ), dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_tangent_rx_matches_full_form(dtype):
    """The tangent-form RX (default) and the full form (QS_FLAG_FULL_RX) agree to rounding
    and both meet the tolerance against the oracle, on circuits with RX at every angle
    range (|tan| above and below 1)."""
    n = 16
    circ = wc.rzrx_cz_circuit(n, 12, seed=11)
    ref = sv.simulate(n, circ)
    out = {}
    for full in (False, True):
        st = qs.State(n, dtype)
        st.execute(qs.compile(n, circ, mode="tile", dtype=dtype, full_rx=full))
        out[full] = st.amplitudes().astype(np.complex128)
    if dtype == "c128":
        for v in out.values():
            assert np.max(np.abs(v - ref)) <= 1e-12 and sv.fidelity_loss(v, ref) <= 1e-10
        assert np.max(np.abs(out[True] - out[False])) <= 1e-13
    else:
        for v in out.values():
            assert sv.fidelity_loss(v, ref) <= 1e-5


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_tile_mode_every_register_width(dtype, arith, K):
    """Every register-stage width the kernels instantiate (complex128 up to 4, complex64 up to
    5), on mixed circuits with 1- to 4-qubit gates, controls and diagonals, plus the
    RZ/RX/CZ construction (tangent-form RX runs, phase tables)."""
    if dtype == "c128" and K > 4:
        pytest.skip("complex128 holds at most 4 register bits")
    n = 15
    circ = wc.random_mixed_circuit(n, 200, seed=100 + K, kmax=3) + wc.rzrx_cz_circuit(n, 6, seed=K)
    st = qs.State(n, dtype, arith=arith)
    st.execute(qs.compile(n, circ, mode="tile", dtype=dtype, arith=arith, tile_bits=11, reg_bits=K))
    check(st.amplitudes(), sv.simulate(n, circ), dtype)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_controlled_diagonals_in_phase_tables(dtype, arith):
    """Controlled diagonal gates (controlled RZ-type 2x2) between rotations: inside a register
    stage they become phase-table factors whose value at index 0 is 1 (control clear) while
    other entries take d0 or d1, the case the table's multiply mask must cover."""
    n = 14
    rng = np.random.default_rng(5)
    circ = []
    for layer in range(8):
        for q in range(n):
            circ.append(wc.Gate("RX", (q,), param=float(rng.uniform(0, 2 * np.pi))))
        for _ in range(n):
            c, t = (int(x) for x in rng.choice(n, 2, replace=False))
            a, b = rng.uniform(0, 2 * np.pi, 2)
            circ.append(wc.Gate("CU", (c, t), matrix=np.diag([np.exp(1j * a), np.exp(1j * b)])))
    st = qs.State(n, dtype, arith=arith)
    st.execute(qs.compile(n, circ, mode="tile", dtype=dtype, arith=arith))
    check(st.amplitudes(), sv.simulate(n, circ), dtype)

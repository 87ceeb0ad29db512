"""GPU parity at the benchmark's full sizes, against the oracle and the closed forms.

* PermuteQubits (Sec. 2, Appendix A) on the 30-qubit complex128 state (16 GiB, byte offsets
  past 2^32) and a 31-qubit complex64 state: every amplitude holds its own index, so the
  value found at storage position j after the permutation must be the logical index
  i = j^-1(j, sigma') (oracle.sv.logical_index), bit for bit, on seeded windows and on the
  first and last elements; permuting back restores the original bytes.
* The paper's Algorithm 1 (one local<->global transposition per PermuteQubits, m = 12 local
  qubits) on the first 4 layers of the 30-qubit benchmark circuit, and the tile passes on
  its first 8 layers (several passes, ragged ones included), both against the full FP64
  oracle state (2^30 amplitudes).
* Appendix C's QFT-like circuit at 22 qubits in tile, Algorithm 1 and per-gate modes.
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
    err = float(np.max(np.abs(got - ref)))
    fid = sv.fidelity_loss(got, ref)
    assert err <= amp_tol, f"max amplitude error {err:.3e} > {amp_tol}"
    assert fid <= fid_tol, f"fidelity loss {fid:.3e} > {fid_tol}"


def index_encoded(n, dtype):
    """Amplitude j = (j, -j) for complex128; (j mod 2^24, j >> 24) for complex64, so that every
    value is exact and distinct."""
    j = np.arange(1 << n, dtype=np.uint64)
    if dtype == "c128":
        out = np.empty(1 << n, dtype=np.complex128)
        f = out.view(np.float64).reshape(-1, 2)
        f[:, 0] = j
        f[:, 1] = -f[:, 0]
    else:
        out = np.empty(1 << n, dtype=np.complex64)
        f = out.view(np.float32).reshape(-1, 2)
        f[:, 0] = (j & np.uint64(0xFFFFFF)).astype(np.float32)
        f[:, 1] = (j >> np.uint64(24)).astype(np.float32)
    return out


def encoded_values(idx, dtype):
    idx = np.asarray(idx, dtype=np.uint64)
    if dtype == "c128":
        out = np.empty(idx.size, dtype=np.complex128)
        f = out.view(np.float64).reshape(-1, 2)
        f[:, 0] = idx
        f[:, 1] = -f[:, 0]
    else:
        out = np.empty(idx.size, dtype=np.complex64)
        f = out.view(np.float32).reshape(-1, 2)
        f[:, 0] = (idx & np.uint64(0xFFFFFF)).astype(np.float32)
        f[:, 1] = (idx >> np.uint64(24)).astype(np.float32)
    return out


def windows(n, count=48, width=1 << 13, seed=7):
    rng = np.random.default_rng(seed)
    starts = [int(s) for s in rng.integers(0, (1 << n) - width, count)]
    return [(0, width), ((1 << n) - width, width)] + [(s, width) for s in starts]


@pytest.mark.parametrize("n,dtype", [(30, "c128"), (31, "c64")])
def test_permute_full_size_bit_exact(n, dtype):
    rng = np.random.default_rng(1000 + n)
    st = qs.State(n, dtype)
    st.set_amplitudes(index_encoded(n, dtype))   # stored under the identity
    ident = list(range(n))
    swap_top = [n - 1] + list(range(1, n - 1)) + [0]                      # one local<->global pair
    high_only = list(range(12)) + [12 + int(x) for x in rng.permutation(n - 12)]   # every rest bit moves
    cases = [wc.random_permutation(n, rng), swap_top, high_only, wc.random_permutation(n, rng)]
    win = windows(n)
    for sigma in cases:
        st.permute(ident)
        st.permute(sigma)
        assert st.permutation() == list(sigma)
        for s, w in win:
            got = st.amplitudes(s, w, order=qs.QS_ORDER_STORAGE)
            want = encoded_values(sv.logical_index(np.arange(s, s + w, dtype=np.uint64), sigma), dtype)
            assert got.tobytes() == want.tobytes(), (sigma, s)
        # the logical-order read-out does not depend on sigma
        got = st.amplitudes(12345, 4096)
        assert got.tobytes() == encoded_values(np.arange(12345, 12345 + 4096), dtype).tobytes()
    st.permute(ident)
    for s, w in win:
        got = st.amplitudes(s, w, order=qs.QS_ORDER_STORAGE)
        assert got.tobytes() == encoded_values(np.arange(s, s + w), dtype).tobytes()
    st.close()


@pytest.fixture(scope="module")
def oracle_30q():
    """FP64 oracle states of the 30-qubit benchmark construction (seed 0) after 4 and after
    8 of its 40 layers (the 4-layer circuit is a prefix of the 8-layer one)."""
    n = 30
    c8 = wc.rzrx_cz_circuit(n, 8, seed=0)
    c4 = wc.rzrx_cz_circuit(n, 4, seed=0)
    assert [(g.kind, g.qubits, g.param) for g in c8[:len(c4)]] == [(g.kind, g.qubits, g.param) for g in c4]
    o = sv.OracleState(n)
    o.run(c4)
    after4 = o.psi.copy()
    o.run(c8[len(c4):])
    return {"n": n, "c4": c4, "c8": c8, "after4": after4, "after8": o.psi}


def test_paper_mode_30q_against_oracle(oracle_30q):
    """Algorithm 1 with m = 12: tile passes over storage bits [0, 12) between single
    local<->global transpositions (K3), on the full 2^30-amplitude state."""
    n, circ = oracle_30q["n"], oracle_30q["c4"]
    st = qs.State(n, "c128")
    plan = qs.compile(n, circ, mode="paper", dtype="c128", tile_bits=12)
    stats = plan.stats()
    assert stats["n_permutes"] >= 10
    st.execute(plan)
    assert st.permutation() == plan.final_permutation()
    got = st.amplitudes()
    st.close()
    check(got, oracle_30q["after4"], "c128")


def test_tile_mode_30q_8_layers_against_oracle(oracle_30q):
    n, circ = oracle_30q["n"], oracle_30q["c8"]
    st = qs.State(n, "c128")
    plan = qs.compile(n, circ, mode="tile", dtype="c128")
    assert plan.stats()["n_passes"] >= 5
    st.execute(plan)
    got = st.amplitudes()
    st.close()
    check(got, oracle_30q["after8"], "c128")


@pytest.mark.parametrize("dtype,arith", [("c128", "df"), ("c128", "f64"), ("c64", "auto")])
@pytest.mark.parametrize("mode", ["tile", "paper", "pergate"])
def test_qft_like_22q(dtype, arith, mode):
    """Appendix C's QFT-like circuit (controlled phase rotations replaced by CNOT) on a
    spread input state, against the oracle; Algorithm 1 needs at most 2(n - m) permutations
    on it."""
    n, m = 22, 12
    prep = [wc.Gate("H", (q,)) for q in range(n)] + [wc.Gate("RZ", (q,), param=0.11 * (q + 1)) for q in range(n)]
    circ = prep + wc.qft_like_circuit(n)
    ref = sv.simulate(n, circ)
    kw = {"tile_bits": m} if mode == "paper" else {}
    plan = qs.compile(n, circ, mode=mode, dtype=dtype, arith=arith, **kw)
    if mode == "paper":
        bare = qs.compile(n, wc.qft_like_circuit(n), mode="paper", dtype=dtype, arith=arith, tile_bits=m)
        assert bare.stats()["n_permutes"] <= 2 * (n - m)
    st = qs.State(n, dtype, arith=arith)
    st.execute(plan)
    check(st.amplitudes(), ref, dtype)
    st.close()

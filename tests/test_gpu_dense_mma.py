"""GPU: the tensor-core dense k-qubit kernel (complex64, TF32 operands with a three-term
split) against the FP64 oracle and against the CUDA-core kernel, for every k, qubit
orders, states of one to many tiles per CTA, and the permutation it inserts when the
qubits are not on the lowest storage bits."""
import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def check_c64(got, ref):
    got = got.astype(np.complex128)
    assert sv.fidelity_loss(got, ref) <= 1e-5
    # per amplitude: each TF32 split factor keeps ~2^-22 relative, FP32 sums over 128 terms
    # of a 6-qubit block (random signs, |W| ~ 1/8) and the complex64 input rounding add up
    # to ~1e-6 of the largest amplitude; the bound leaves a factor 4
    assert np.max(np.abs(got - ref)) <= 4e-6 * np.max(np.abs(ref))


def run_dense(n, k, qubits, path, seed, psi0=None):
    U = wc.haar_unitary(1 << k, np.random.default_rng(100 + seed))
    psi0 = rand_state(n, seed) if psi0 is None else psi0
    st = qs.State(n, "c64")
    st.set_amplitudes(psi0)
    st.set_dense_path(path)
    st.set_profiling(True)
    st.apply_dense(U, qubits)
    got = st.amplitudes()
    names = {k_["name"] for k_ in st.kernel_stats()}
    ref = sv.OracleState(n, psi0)
    ref.apply_dense(U, qubits)
    return got, ref.psi, names, st


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_tensor_low_qubits_every_k(k):
    rng = np.random.default_rng(k)
    qubits = [int(q) for q in rng.permutation(k)]   # storage bits 0..k-1 in a random order
    for n in (12, 17, 22):   # 1 tile; 32 tiles; 1024 tiles (several per CTA, ring wraps)
        got, ref, names, _ = run_dense(n, k, qubits, "tensor", seed=n + k)
        assert "dense_mma_c64" in names
        check_c64(got, ref)


def test_tensor_matches_cuda_cores():
    n, k = 20, 6
    qubits = [5, 0, 3, 1, 4, 2]
    a, ref, names_t, _ = run_dense(n, k, qubits, "tensor", seed=3)
    b, _, names_c, _ = run_dense(n, k, qubits, "cuda_cores", seed=3)
    assert "dense_mma_c64" in names_t and "dense_mma_c64" not in names_c
    check_c64(a, ref)
    check_c64(b, ref)
    assert np.max(np.abs(a.astype(np.complex128) - b)) <= 2e-6 * np.max(np.abs(ref))


def test_tensor_permutes_high_qubits_first():
    n, k = 18, 4
    qubits = [17, 2, 9, 12]
    got, ref, names, st = run_dense(n, k, qubits, "tensor", seed=5)
    assert "permute" in names and "dense_mma_c64" in names
    perm = st.permutation()
    assert [perm[q] for q in qubits] == [0, 1, 2, 3]
    check_c64(got, ref)          # amplitudes() reads logical order under the new sigma
    # a following ordinary gate still addresses logical qubits
    st.apply_1q(np.array([[0, 1], [1, 0]]), 17)
    o = sv.OracleState(n, ref)
    o.apply_1q(np.array([[0, 1], [1, 0]]), 17)
    check_c64(st.amplitudes(), o.psi)


def test_auto_path_choice():
    n = 16
    _, _, names, _ = run_dense(n, 6, list(range(6)), "auto", seed=1)
    assert "dense_mma_c64" in names
    _, _, names, _ = run_dense(n, 3, [0, 1, 2], "auto", seed=1)
    assert "dense_mma_c64" not in names
    _, _, names, _ = run_dense(n, 5, [0, 1, 2, 3, 15], "auto", seed=1)   # not low, k < 6: no permute
    assert "dense_mma_c64" not in names and "permute" not in names
    got, ref, names, _ = run_dense(n, 6, [15, 1, 2, 3, 4, 9], "auto", seed=2)   # not low, k = 6: permute first
    assert "dense_mma_c64" in names and "permute" in names
    check_c64(got, ref)
    _, _, names, _ = run_dense(n, 6, list(range(6)), "cuda_cores", seed=1)
    assert "dense_mma_c64" not in names


def test_tensor_rejections():
    st = qs.State(12, "c128")
    st.set_dense_path("tensor")
    with pytest.raises(qs.QSError):
        st.apply_dense(np.eye(4), [0, 1])
    st = qs.State(11, "c64")
    st.set_dense_path("tensor")
    with pytest.raises(qs.QSError):
        st.apply_dense(np.eye(4), [0, 1])
    st = qs.State(12, "c64")
    with pytest.raises(qs.QSError):
        st.apply_dense(np.eye(4), [0, 0])


def test_tensor_circuit_of_blocks():
    """Twelve 6-qubit Haar blocks on rotating qubit sets (each permuted to the bottom first):
    the error stays at complex64 level over a sequence."""
    n = 20
    rng = np.random.default_rng(9)
    st = qs.State(n, "c64")
    st.set_dense_path("tensor")
    ref = sv.OracleState(n)
    for i in range(12):
        qubits = [int(q) for q in rng.choice(n, 6, replace=False)]
        U = wc.haar_unitary(64, rng)
        st.apply_dense(U, qubits)
        ref.apply_dense(U, qubits)
    got = st.amplitudes().astype(np.complex128)
    assert sv.fidelity_loss(got, ref.psi) <= 1e-5
    assert abs(st.norm() - 1.0) <= 1e-5

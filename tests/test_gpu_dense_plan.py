"""GPU: dense tensor-core blocks that the compiler puts into complex64 plans.

When the cost model predicts that the gates ready on storage bits 0..5 alone cost more as
tile-pass arithmetic than one dense 64 x 64 block on the tensor cores, the compiler fuses them
into such a block (Sec. 1's gate fusion, chosen from measured kernel costs as Sec. 3
suggests).  The results must still match the FP64 oracle at the complex64 tolerance
(fidelity loss and max amplitude error <= 1e-5).
"""
import ctypes

import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")
from paper_2010_09746_gb300 import _lib  # noqa: E402


def cheap_dense_model():
    m = qs.default_cost_model("c64")
    for i, v in enumerate((0.0, 1e-12, 0.0)):
        m.dense[i] = v
    m.tile[2] = 1e-6   # tile-pass arithmetic made dear
    return m


def check(got, ref, tol=1e-5):
    got = np.asarray(got, dtype=np.complex128)
    err = float(np.max(np.abs(got - ref)))
    fid = sv.fidelity_loss(got, ref)
    assert err <= tol and fid <= tol, (err, fid)


@pytest.mark.parametrize("n", [12, 16, 20])
def test_compiled_dense_blocks_match_oracle(n):
    circ = wc.rzrx_cz_circuit(n, 10, seed=n) + wc.haar_cnot_circuit(n, 4, seed=n) + \
        wc.random_mixed_circuit(n, 80, seed=n, kmax=3)
    plan = qs.compile(n, circ, mode="tile", dtype="c64", cost=cheap_dense_model())
    assert plan.stats()["n_dense"] > 0
    trace_kinds = {k for k, _ in plan.trace()}
    assert 5 in trace_kinds
    st = qs.State(n, "c64")
    st.execute(plan)
    check(st.amplitudes(), sv.simulate(n, circ))
    st.close()


def test_dense_blocks_after_a_permutation_start():
    """A plan compiled for a non-identity start permutation fuses the gates on whichever
    logical qubits sit on storage bits 0..5."""
    n = 14
    rng = np.random.default_rng(4)
    sigma0 = wc.random_permutation(n, rng)
    circ = wc.rzrx_cz_circuit(n, 8, seed=4)
    plan = qs.compile(n, circ, sigma0=sigma0, mode="tile", dtype="c64", cost=cheap_dense_model())
    assert plan.stats()["n_dense"] > 0
    st = qs.State(n, "c64")
    st.permute(sigma0)
    st.execute(plan)
    check(st.amplitudes(), sv.simulate(n, circ))
    st.close()


@pytest.mark.parametrize("model", ["default", "cheap_dense"])
def test_30q_c64_against_c128(model):
    """The 30-qubit circuit as complex64 -- with whatever dense blocks the default model picks
    (none once gate fusion has shrunk the tile work), and with a model that makes dense blocks
    cheap so that several run at full size -- against the oracle-validated complex128 tile
    path on the whole state (FP64 inner product)."""
    n = 30
    circ = wc.rzrx_cz_circuit(n, 40, seed=0)
    p64 = qs.compile(n, circ, mode="tile", dtype="c64", cost=cheap_dense_model() if model == "cheap_dense" else None)
    if model == "cheap_dense":
        assert p64.stats()["n_dense"] >= 1
    s64 = qs.State(n, "c64")
    s64.execute(p64)
    s128 = qs.State(n, "c128")
    s128.execute(qs.compile(n, circ, mode="tile", dtype="c128"))
    assert 1.0 - s64.fidelity(s128) <= 1e-5
    assert abs(s64.norm() - 1.0) <= 1e-5
    s64.close()
    s128.close()


def test_batches_never_take_dense_blocks():
    work = [(14, wc.rzrx_cz_circuit(14, 12, seed=s)) for s in range(3)]
    b = qs.Batch(work, dtype="c64", graph=False)
    b.run()
    norms = b.norms()
    assert np.all(np.abs(norms - 1.0) <= 1e-5)
    for i, (n, c) in enumerate(work):
        check(b.amplitudes(i), sv.simulate(n, c))

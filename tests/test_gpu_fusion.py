"""GPU parity of gate fusion (tile mode's default): plans whose single-qubit runs were
replaced by diag . RX . diag products against the FP64 oracle, and against the same plans
compiled without fusion, in every arithmetic mode; tolerances as in test_gpu_parity."""

import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")

TOL = {"c128": (1e-10, 1e-12), "c64": (1e-5, 1e-5)}
MODES = [("c128", "df"), ("c128", "f64"), ("c64", "auto")]


def check(got, ref, dtype):
    fid_tol, amp_tol = TOL[dtype]
    got = np.asarray(got, dtype=np.complex128)
    err = float(np.max(np.abs(got - ref)))
    fid = sv.fidelity_loss(got, ref)
    assert err <= amp_tol and fid <= fid_tol, (err, fid)


def run(n, circ, dtype, arith, **opts):
    st = qs.State(n, dtype, arith=arith)
    st.execute(qs.compile(n, circ, mode="tile", dtype=dtype, arith=arith, **opts))
    out = st.amplitudes()
    st.close()
    return out


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n", [9, 14, 20])
def test_fused_runs_match_oracle_and_unfused(dtype, arith, n):
    circ = wc.single_qubit_run_circuit(n, 10, seed=n) + wc.rzrx_cz_circuit(n, 12, seed=n)
    ref = sv.simulate(n, circ)
    fused = run(n, circ, dtype, arith)
    check(fused, ref, dtype)
    unfused = run(n, circ, dtype, arith, fuse=False)
    check(unfused, ref, dtype)
    assert float(np.max(np.abs(fused - unfused))) <= 2 * TOL[dtype][1]


def test_fusion_on_the_30_qubit_construction_at_20_qubits():
    """The benchmark construction (40 layers, CZ biased toward high qubits: long RZ/RX runs on
    the low qubits) at 20 qubits, complex128, fused against the oracle."""
    n = 20
    circ = wc.rzrx_cz_circuit(n, 40, seed=0)
    plan = qs.compile(n, circ, mode="tile")
    assert plan.stats()["alu_instr"] < 0.7 * qs.compile(n, circ, mode="tile", fuse=False).stats()["alu_instr"]
    st = qs.State(n, "c128")
    st.execute(plan)
    check(st.amplitudes(), sv.simulate(n, circ), "c128")
    st.close()

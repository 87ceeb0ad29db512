"""GPU parity at the workloads' full sizes.

* 30 qubits, complex128, the bench construction at depth 2: the whole 2^30-amplitude state
  against the FP64 oracle (16 GiB on each side).
* 30 qubits, complex128, the bench circuit itself (40 layers, 2680 gates) in the bench's
  launch configuration: norm, and the mirror circuit C^dagger C |0> = |0> (properties that
  hold at any size; the oracle would need minutes here).
* precision study: 32 qubits complex128 vs complex64 on 2^20 sampled amplitudes (64
  seeded windows), norms, and 33 qubits complex64 (64 GiB) mirror fidelity.
"""
import math

import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")


def inverse(circ):
    out = []
    for g in reversed(circ):
        if g.kind in ("RZ", "RX"):
            out.append(wc.Gate(g.kind, g.qubits, param=-g.param))
        elif g.kind == "U1":
            out.append(wc.Gate("U1", g.qubits, matrix=np.conj(g.matrix).T))
        elif g.kind in ("CZ", "CNOT", "H", "X", "Y", "Z", "SWAP"):
            out.append(g)
        else:
            raise ValueError(g.kind)
    return out


def windows(n, count=64, width=1 << 14, seed=0):
    rng = np.random.default_rng(seed)
    starts = rng.integers(0, (1 << n) - width, count)
    return [(int(s) & ~(width - 1), width) for s in starts]


def test_30q_full_state_shallow():
    n = 30
    circ = wc.rzrx_cz_circuit(n, 2, seed=0)
    st = qs.State(n, "c128")
    st.run(circ, mode="tile")
    got = st.amplitudes()
    st.close()
    ref = sv.simulate(n, circ)
    err = float(np.max(np.abs(got - ref)))
    fid = sv.fidelity_loss(got, ref)
    assert err <= 1e-12 and fid <= 1e-10, (err, fid)


def test_30q_bench_circuit_properties():
    n = 30
    circ = wc.rzrx_cz_circuit(n, 40, seed=0)
    st = qs.State(n, "c128")
    plan = qs.compile(n, circ, mode="tile", dtype="c128")
    st.execute(plan)
    assert abs(st.norm() - 1.0) <= 1e-12
    st.run(inverse(circ), mode="tile")
    a0 = st.amplitudes(0, 1)[0]
    assert abs(a0 - 1.0) <= 1e-12
    for s, w in windows(n, 16):
        if s == 0:
            continue
        assert np.max(np.abs(st.amplitudes(s, w))) <= 1e-12


def test_precision_32q_c64_vs_c128():
    n = 32
    circ = wc.rzrx_cz_circuit(n, 30, seed=0)
    assert len(circ) == 2160
    win = windows(n)
    st = qs.State(n, "c128")
    st.run(circ, mode="tile")
    ref_norm = st.norm()
    ref = np.concatenate([st.amplitudes(s, w) for s, w in win])
    st.close()
    assert abs(ref_norm - 1.0) <= 1e-12
    st = qs.State(n, "c64")
    st.run(circ, mode="tile")
    norm64 = st.norm()
    got = np.concatenate([st.amplitudes(s, w) for s, w in win]).astype(np.complex128)
    st.close()
    assert abs(norm64 - 1.0) <= 1e-5
    # fidelity of the sampled sub-vectors (normalised overlap)
    ov = abs(np.vdot(ref, got)) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real)
    assert 1.0 - ov <= 1e-5
    assert np.max(np.abs(got - ref)) <= 1e-5 * math.sqrt(2 ** -n) * 64


def test_33q_c64_mirror():
    n = 33
    circ = wc.rzrx_cz_circuit(n, 30, seed=0)
    assert len(circ) == 2220
    st = qs.State(n, "c64")
    st.run(circ, mode="tile")
    assert abs(st.norm() - 1.0) <= 1e-5
    st.run(inverse(circ), mode="tile")
    a0 = complex(st.amplitudes(0, 1)[0])
    assert 1.0 - abs(a0) ** 2 <= 1e-5

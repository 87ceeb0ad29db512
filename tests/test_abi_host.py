"""CPU tests of the C ABI: the library loads, exports every symbol include/qs.h declares,
validates its arguments, and its host compiler (no GPU needed to compile) emits the
schedules the oracle's Algorithm 1 emits and valid tile-pass schedules."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2010_09746_gb300 as qs
from paper_2010_09746_gb300 import _lib
from oracle import compiler_ref as cr
from oracle import sv
from workloads import circuits as wc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "qs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    syms = declared_symbols()
    assert len(syms) >= 30
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) == set(_lib.SIGNATURES), "binding and header disagree"


def test_struct_layout():
    assert ctypes.sizeof(_lib.qs_op) == 48
    assert ctypes.sizeof(_lib.qs_compile_opts) == 48
    assert ctypes.sizeof(_lib.qs_plan_stats) == 96
    assert ctypes.sizeof(_lib.qs_cost_model) == 96


def test_marshal_matches_field_by_field():
    """The binding's column-wise marshalling gives the qs_op records and matrix doubles that
    writing each struct field in turn gives: kind, qubits, param, the first double of the
    gate's matrix (-1 without one), and each matrix as row-major (re, im) pairs."""
    rng = np.random.default_rng(4)
    circs = [wc.random_mixed_circuit(12, 400, seed=4, kmax=6), wc.qft_like_circuit(9),
             wc.rzrx_cz_circuit(7, 3, seed=4), [], [wc.Gate("UK", (3, 0, 5), matrix=wc.haar_unitary(8, rng))],
             wc.mixed_batch_circuit(14, 20, rng)]
    for circ in circs:
        ops, n, mats = qs.marshal(circ)
        assert n == len(circ)
        want_mats = []
        off = 0
        for i, g in enumerate(circ):
            o = ops[i]
            assert o.kind == _lib.OP_CODES[g.kind] and o.nq == len(g.qubits)
            assert list(o.q)[:o.nq] == list(g.qubits) and all(v == 0 for v in list(o.q)[o.nq:])
            assert o.param == float(g.param or 0.0)
            if g.matrix is None:
                assert o.mat == -1
            else:
                assert o.mat == off
                flat = [x for z in np.asarray(g.matrix, dtype=complex).ravel() for x in (z.real, z.imag)]
                want_mats += flat
                off += len(flat)
        if want_mats:
            assert np.array_equal(mats, np.array(want_mats))
    with pytest.raises(ValueError):
        qs.marshal([type("G", (), {"kind": "UK", "qubits": tuple(range(7)), "param": 0.0, "matrix": None})()])


def test_version():
    assert b"sm_103a" in _lib.load().qs_version()


def _compile_status(n, circ, **kw):
    try:
        qs.compile(n, circ, **kw)
        return _lib.QS_OK
    except qs.QSError as e:
        return e.status


def test_compile_rejects_bad_input():
    g = wc.Gate("H", (0,))
    assert _compile_status(3, [g]) == _lib.QS_OK
    assert _compile_status(3, [wc.Gate("H", (3,))]) == _lib.QS_EINVAL
    assert _compile_status(3, [wc.Gate("CNOT", (1, 1))]) == _lib.QS_EINVAL
    assert _compile_status(0, [g]) == _lib.QS_EINVAL
    assert _compile_status(3, [g], sigma0=[0, 0, 1]) == _lib.QS_EINVAL
    # matrix offset beyond the buffer
    ops, nops, mats = qs.marshal([wc.Gate("U1", (0,), matrix=np.eye(2))])
    ops[0].mat = 100
    h = ctypes.c_void_p()
    o = qs._opts()
    st = _lib.load().qs_compile(2, ops, nops, mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mats.size,
                                None, ctypes.byref(o), ctypes.byref(h))
    assert st == _lib.QS_EINVAL
    assert b"offset" in _lib.load().qs_last_error()


def test_state_calls_validate_null():
    L = _lib.load()
    assert L.qs_destroy(None) == _lib.QS_OK
    assert L.qs_sync(None) == _lib.QS_EINVAL
    assert L.qs_norm(None, None) == _lib.QS_EINVAL
    h = ctypes.c_void_p()
    assert L.qs_create(0, 1, ctypes.byref(h)) == _lib.QS_EINVAL
    assert L.qs_create(37, 1, ctypes.byref(h)) == _lib.QS_EINVAL


def test_server_rejects_bad_options():
    """Options are checked before any device is touched."""
    L = _lib.load()
    h = ctypes.c_void_p()
    for field, value in (("slots", -1), ("slots", 1000), ("compile_threads", -2), ("order", 2), ("readout", -1),
                         ("tile_bits", 15), ("mem_budget", -5), ("reserved", 1), ("batch_max", -1)):
        o = _lib.qs_server_opts()
        setattr(o, field, value)
        assert L.qs_server_create(ctypes.byref(o), ctypes.byref(h)) == _lib.QS_EINVAL, field
        assert not h.value
    assert L.qs_server_create(None, None) == _lib.QS_EINVAL
    assert L.qs_server_destroy(None) == _lib.QS_OK
    cnt = ctypes.c_int()
    assert L.qs_server_poll(None, None, 0, ctypes.byref(cnt), 0) == _lib.QS_EINVAL


def test_server_struct_layout():
    assert ctypes.sizeof(_lib.qs_server_opts) == 48
    assert ctypes.sizeof(_lib.qs_server_result) == 64 + 128
    assert ctypes.sizeof(_lib.qs_server_stats) == 7 * 8 + 3 * 8


def oracle_trace(n, m, circ, scoring="closure"):
    prog, st = cr.alg1(n, m, circ, scoring=scoring)
    out = []
    sigma = list(range(n))
    for ins in prog:
        if ins[0] == "gate":
            out.append((1 if ins[2] else 0, ins[1]))
        else:
            new = ins[1]
            a, b = [q for q in range(n) if new[q] != sigma[q]]
            l, g = (a, b) if sigma[a] < m else (b, a)
            out.append((2, 64 * l + g))
            sigma = list(new)
    return out, st


@pytest.mark.parametrize("scoring", [0, 1])
@pytest.mark.parametrize("n,m,p,seed", [(12, 9, 0.3, 0), (12, 9, 1.0, 1), (12, 9, 0.0, 2), (20, 16, 0.3, 3),
                                        (35, 28, 0.3, 4), (35, 28, 1.0, 5), (50, 40, 0.3, 6)])
def test_paper_mode_schedule_matches_oracle_alg1(n, m, p, seed, scoring):
    """Integer work, bit-exact: the library's Algorithm 1 emits exactly the oracle's
    instruction list (gates, non-local gates, transpositions)."""
    if n > 36:
        pytest.skip("library limit n <= 36")
    circ = wc.paper_random_circuit(n, p, seed)
    want, st = oracle_trace(n, m, circ, scoring="closure" if scoring == 0 else "frontier")
    plan = qs.compile(n, circ, mode="paper", tile_bits=m, scoring=scoring)
    got = plan.trace()
    assert got == want
    s = plan.stats()
    assert s["n_permutes"] == st["n_permutes"]
    assert s["n_comm_gates"] == st["n_comm_gates"]


def test_paper_mode_fig3_statistic_through_library():
    n, m = 35, 28
    fr = []
    for seed in range(20):
        circ = wc.paper_random_circuit(n, 0.3, seed)
        s = qs.compile(n, circ, mode="paper", tile_bits=m).stats()
        fr.append((s["n_permutes"] + s["n_comm_gates"]) / s["n_gates"])
    assert abs(np.mean(fr) - 0.035) < 0.01


def tile_schedule(plan):
    passes = []
    for k, v in plan.trace():
        if k == 3:
            passes.append([v, []])
        elif k == 4:
            passes[-1][0] |= v << 31
        else:
            assert k == 0
            passes[-1][1].append(v)
    return passes


@pytest.mark.parametrize("n,L,c,seed", [(10, 6, 2, 0), (14, 8, 3, 1), (16, 9, 3, 2), (30, 12, 3, 3)])
def test_tile_mode_schedule_is_valid(n, L, c, seed):
    circ = wc.rzrx_cz_circuit(n, 6, seed) + wc.random_mixed_circuit(n, 60, seed, kmax=3)
    plan = qs.compile(n, circ, mode="tile", tile_bits=L, low_bits=c, fuse=False)
    passes = tile_schedule(plan)
    preds = cr.build_dag(circ)
    seen = set()
    for mask, ids in passes:
        assert bin(mask).count("1") == L
        assert mask & ((1 << c) - 1) == (1 << c) - 1
        for v in ids:
            for p in preds[v]:
                assert p in seen
            seen.add(v)
            g = circ[v]
            need = [q for q, k in zip(g.qubits, cr.qubit_classes(g)) if k != cr.CLS_Z]
            if g.kind in ("U2", "UK") and len(g.qubits) >= 2:
                need = list(g.qubits)
            for q in need:
                assert (mask >> q) & 1, "non-diagonal qubit outside the tile"
    assert seen == set(range(len(circ)))
    assert plan.stats()["n_passes"] == len(passes)


def test_fusion_keeps_every_gate_in_the_trace_and_cuts_the_work():
    """With gate fusion (default) the tile-mode trace still names every input gate once, the
    stats count the input gates, the counted arithmetic of the rzrx construction (long RZ/RX
    runs on the qubits the biased CZs leave alone) drops by more than a third, and the other
    modes do not fuse."""
    n = 16
    circ = wc.rzrx_cz_circuit(n, 20, seed=7) + wc.single_qubit_run_circuit(n, 6, seed=7)
    plan = qs.compile(n, circ, mode="tile")
    ids = sorted(v for k, v in plan.trace() if k == 0)
    assert ids == list(range(len(circ)))
    a = plan.stats()
    b = qs.compile(n, circ, mode="tile", fuse=False).stats()
    assert a["n_gates"] == b["n_gates"] == len(circ)
    assert a["n_fused"] > 0 and b["n_fused"] == 0
    assert a["alu_instr"] < 0.66 * b["alu_instr"]
    for dt in ("c128", "c64"):
        for mode in ("paper", "pergate"):
            x = qs.compile(n, circ, mode=mode, dtype=dt, tile_bits=10 if mode == "paper" else 0).stats()
            y = qs.compile(n, circ, mode=mode, dtype=dt, tile_bits=10 if mode == "paper" else 0, fuse=False).stats()
            assert x["alu_instr"] == y["alu_instr"] and x["hbm_bytes"] == y["hbm_bytes"]


def test_tile_mode_order_simulates_to_original():
    n = 9
    circ = wc.random_mixed_circuit(n, 120, seed=5, kmax=3)
    plan = qs.compile(n, circ, mode="tile", tile_bits=6, low_bits=2, fuse=False)
    order = [v for _, ids in tile_schedule(plan) for v in ids]
    np.testing.assert_allclose(sv.simulate(n, [circ[v] for v in order]), sv.simulate(n, circ), atol=1e-13)


def test_tile_mode_pass_count_beats_per_gate():
    n = 30
    circ = wc.rzrx_cz_circuit(n, 40, seed=0)
    st = qs.compile(n, circ, mode="tile").stats()
    assert st["n_gates"] == 2680
    assert st["n_passes"] < 300
    pg = qs.compile(n, circ, mode="pergate").stats()
    assert st["hbm_bytes"] < pg["hbm_bytes"] / 5


def test_appendix_b_export_is_the_circuit_on_hardware():
    """SWAP + Emulated-SWAP export (Appendix B): with RELABEL read as a hardware SWAP every
    pair cancels, so the exported list simulates to the original circuit."""
    n, m = 10, 7
    circ = wc.paper_random_circuit(n, 0.3, seed=3)
    plan = qs.compile(n, circ, mode="paper", tile_bits=m)
    ir = plan.export_swaps(circ)
    assert sum(1 for g in ir if g.kind == "RELABEL") == plan.stats()["n_permutes"] > 0
    hw = [wc.Gate(g.kind, g.qubits, g.param, g.matrix) for g in ir]
    np.testing.assert_allclose(sv.simulate(n, hw), sv.simulate(n, circ), atol=1e-12)


def test_relabel_only_in_pergate_mode():
    c = [wc.Gate("H", (0,)), wc.Gate("RELABEL", (0, 1))]
    assert _compile_status(3, c, mode="pergate") == _lib.QS_OK
    assert _compile_status(3, c, mode="tile") == _lib.QS_EINVAL
    p = qs.compile(3, c, mode="pergate")
    assert p.final_permutation() == [1, 0, 2]


def test_renorm_every_schedule():
    """Periodic renormalisation adds one norm + scaling (3 state sweeps) after every R kernels."""
    n = 12
    circ = wc.rzrx_cz_circuit(n, 6, seed=3)
    base = qs.compile(n, circ, mode="pergate", dtype="c64").stats()
    S = (1 << n) * 8
    for R in (1, 5, 7):
        s = qs.compile(n, circ, mode="pergate", dtype="c64", renorm_every=R).stats()
        k = base["n_pergate"] // R
        assert s["hbm_bytes"] == pytest.approx(base["hbm_bytes"] + 3 * S * k)
        assert s["n_pergate"] == base["n_pergate"]
    with pytest.raises(qs.QSError):
        qs.compile(n, circ, mode="tile", dtype="c64", renorm_every=-1)


def test_tangent_rx_lowers_the_count():
    """Uncontrolled register-stage RX after a pass's first one use the tangent form (24
    double-float / 2 FP32 instructions per amplitude instead of 32 / 4); QS_FLAG_FULL_RX
    keeps the full form; unknown flags are rejected."""
    n = 20
    circ = wc.rzrx_cz_circuit(n, 10, seed=2)
    for dt in ("c128", "c64"):
        a = qs.compile(n, circ, mode="tile", dtype=dt).stats()
        b = qs.compile(n, circ, mode="tile", dtype=dt, full_rx=True).stats()
        assert a["alu_instr"] < b["alu_instr"]
        assert a["hbm_bytes"] == b["hbm_bytes"] and a["n_passes"] == b["n_passes"]
    o = qs._opts()
    o.flags = 8   # no such flag
    h = ctypes.c_void_p()
    ops, nops, mats = qs.marshal(circ[:3])
    assert _lib.load().qs_compile(n, ops, nops, mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mats.size,
                                  None, ctypes.byref(o), ctypes.byref(h)) == _lib.QS_EINVAL


def test_batch_rejects_periodic_renorm():
    n = 6
    circ = wc.rzrx_cz_circuit(n, 2, seed=0)
    ops, nops, mats = qs.marshal(circ)
    o = qs._opts(dtype="c64", renorm_every=2)
    n_arr = np.array([n], dtype=np.int32)
    offs = np.array([0, nops], dtype=np.int64)
    h = ctypes.c_void_p()
    st = _lib.load().qs_batch_create(1, n_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ops,
                                     offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mats.size,
                                     ctypes.byref(o), ctypes.byref(h))
    assert st == _lib.QS_EINVAL

"""Compiled plans executed on the host, against the FP64 oracle (no GPU).

`plan_emulator_host.cpp` compiles a circuit with the library's own host compiler (the
same make_hgate / compile_circuit the C ABI calls). It then runs every step in
complex<double> with the kernels' op semantics: tile passes with their register stages,
phase tables, merged tangent-form RX and, for complex128 double-float plans, the S-dagger
phase frame; per-gate steps; permutations; renormalisations. Any scheduling, lowering,
table, folding or frame mistake gives an O(1) error. The emulation's own rounding is
~1e-15, so the bound is 1e-10. The GPU parity tests run the same compiled plans on the
kernels.
"""
import ctypes
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

qs = pytest.importorskip("paper_2010_09746_gb300")
from paper_2010_09746_gb300 import _lib  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2010_09746_gb300", "csrc")
TOL = 1e-10


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("emu")
    exe = str(d / "plan_emulator_host")
    srcs = [os.path.join(HERE, "plan_emulator_host.cpp")] + \
        [os.path.join(CSRC, f) for f in ("gates.cpp", "compiler.cpp", "stages.cpp")]
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-o", exe] + srcs, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]

    def run(n, circ, cost=None, threads=0, **opts):
        ops, nops, mats = qs.marshal(circ)
        o = qs._opts(**opts)
        inp, out = str(d / "in.bin"), str(d / "out.bin")
        with open(inp, "wb") as f:
            f.write(struct.pack("<iiq", n, nops, mats.size if nops else 0))
            f.write(bytes(o))
            f.write(struct.pack("<i", 1 if cost is not None else 0))
            f.write(bytes(cost if cost is not None else _lib.qs_cost_model()))
            f.write(bytes(ops)[: nops * 48])
            if nops:
                f.write(np.ascontiguousarray(mats, dtype=np.float64).tobytes())
        extra = ["--threads", str(threads)] if threads else []
        r = subprocess.run([exe, inp, out] + extra, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-3000:]
        run.threads_consistent = (int(r.stderr.split("threads_consistent")[1].split()[0])
                                  if threads else None)
        run.max_register_abs = float(r.stderr.split("max_register_abs")[1].split()[0])
        run.min_register_scale = float(r.stderr.split("min_register_scale")[1].split()[0])
        run.steps = r.stderr.split("steps", 1)[1].splitlines()[0].split()
        with open(out, "rb") as f:
            n2, nsteps = struct.unpack("<ii", f.read(8))
            sigma = np.frombuffer(f.read(4 * n2), dtype=np.int32)
            psi = np.frombuffer(f.read(), dtype=np.complex128)
        assert n2 == n and psi.size == 1 << n
        # logical index i sits at storage index sum_q bit_q(i) << sigma[q]
        idx = np.zeros(1 << n, dtype=np.int64)
        ar = np.arange(1 << n, dtype=np.int64)
        for q in range(n):
            idx |= ((ar >> q) & 1) << int(sigma[q])
        return psi[idx], nsteps

    run.exe = exe
    run.tmp = d
    return run


def check(got, circ, n):
    ref = sv.simulate(n, circ)
    err = float(np.max(np.abs(got - ref)))
    assert err <= TOL, f"max amplitude error {err:.3e}"


MODES = [("c128", "df"), ("c128", "f64"), ("c64", "auto")]


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n,L,c", [(6, 4, 1), (9, 6, 2), (12, 8, 3), (12, 10, 3), (13, 12, 3)])
def test_tile_mode_random_circuits(emulator, dtype, arith, n, L, c):
    circ = wc.random_mixed_circuit(n, 150, seed=n * 31 + L, kmax=min(4, L - c))
    got, _ = emulator(n, circ, mode="tile", dtype=dtype, arith=arith, tile_bits=L, low_bits=c)
    check(got, circ, n)


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n,L,c", [(6, 4, 1), (9, 6, 2), (12, 8, 3)])
def test_fused_single_qubit_runs(emulator, dtype, arith, n, L, c):
    """Gate fusion (the default in tile mode): runs of general, diagonal-only, identity- and
    X-conjugated products, interrupted by CNOT / CZ / SWAP, match the oracle and the unfused
    plan; the fused plan also holds the rzrx construction and random circuits."""
    circ = wc.single_qubit_run_circuit(n, 9, seed=n + 17 * L) + wc.rzrx_cz_circuit(n, 4, seed=n) + \
        wc.random_mixed_circuit(n, 40, seed=n, kmax=min(3, L - c))
    got, _ = emulator(n, circ, mode="tile", dtype=dtype, arith=arith, tile_bits=L, low_bits=c)
    check(got, circ, n)
    unfused, _ = emulator(n, circ, mode="tile", dtype=dtype, arith=arith, tile_bits=L, low_bits=c, fuse=False)
    assert float(np.max(np.abs(got - unfused))) <= 1e-12


def test_euler_split_of_2x2_unitaries(emulator):
    """The split diag . RX . diag that fused runs and general gates take inside tile passes
    (the library's own function): for Haar-random 2x2 unitaries and exact special cases (X, Y,
    H, S, diagonal, an RX, a matrix with a tiny off-diagonal) the factors have the forms the
    lowering needs -- d1 = diag(1, .), rx = c I - i s X with c, s >= 0, d2 diagonal -- and
    their product, taken with numpy, reproduces the matrix to 1e-14."""
    rng = np.random.default_rng(11)
    h = 1 / np.sqrt(2)
    mats = [wc.haar_2x2(rng) for _ in range(300)]
    eps = 1e-9
    mats += [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[h, h], [h, -h]]),
             np.diag([1, 1j]), np.diag([np.exp(0.3j), np.exp(-1.1j)]),
             np.array([[np.cos(0.2), -1j * np.sin(0.2)], [-1j * np.sin(0.2), np.cos(0.2)]]),
             np.array([[np.sqrt(1 - eps ** 2), eps], [-eps, np.sqrt(1 - eps ** 2)]]) * np.exp(0.7j)]
    mats = [np.asarray(m, dtype=np.complex128) for m in mats]
    inp, out = str(emulator.tmp / "euler_in.bin"), str(emulator.tmp / "euler_out.bin")
    with open(inp, "wb") as f:
        f.write(struct.pack("<i", len(mats)))
        for m in mats:
            f.write(np.ascontiguousarray(m.reshape(-1)).view(np.float64).tobytes())
    r = subprocess.run([emulator.exe, "--euler", inp, out], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    raw = open(out, "rb").read()
    rec = 4 + 3 * 64
    assert len(raw) == rec * len(mats)
    for k, m in enumerate(mats):
        ok = struct.unpack("<i", raw[rec * k: rec * k + 4])[0]
        fac = np.frombuffer(raw[rec * k + 4: rec * (k + 1)], dtype=np.complex128).reshape(3, 2, 2)
        d1, rx, d2 = fac
        assert ok == 1, k
        assert d1[0, 0] == 1 and d1[0, 1] == 0 and d1[1, 0] == 0, k
        assert rx[0, 0] == rx[1, 1] and rx[0, 0].imag == 0 and rx[0, 0].real >= 0, k
        assert rx[0, 1] == rx[1, 0] and rx[0, 1].real == 0 and rx[0, 1].imag <= 0, k
        assert d2[0, 1] == 0 and d2[1, 0] == 0, k
        assert np.max(np.abs(d2 @ rx @ d1 - m)) <= 1e-14, (k, np.max(np.abs(d2 @ rx @ d1 - m)))


def storage_forms_consistent(steps):
    """The state's storage form along a plan: binary64 at its start and end and into every
    per-gate kernel, renormalisation and dense block; a pass reads the form the step before
    left (a permutation moves elements unchanged)."""
    form = "b"
    for t in steps:
        if t[0] == "P":
            if t[1] != form:
                return False
            form = t[2]
        elif t in ("G", "R", "D"):
            if form != "b":
                return False
    return form == "b"


@pytest.mark.parametrize("mode,dtype,arith,kw", [
    ("tile", "c128", "df", {"tile_bits": 8}), ("tile", "c128", "df", {"tile_bits": 8, "renorm_every": 2}),
    ("paper", "c128", "df", {"tile_bits": 8}), ("paper", "c128", "df", {"tile_bits": 6}),
    ("tile", "c128", "f64", {"tile_bits": 8}), ("tile", "c64", "auto", {"tile_bits": 8})])
def test_double_float_storage_between_passes(emulator, mode, dtype, arith, kw):
    """Consecutive double-float tile passes keep the state in double-float form (no binary64
    split / join between them); everything else sees binary64, and the results still match
    the oracle (the emulator computes in complex<double>, so the check here is the rule)."""
    n = 12
    circ = wc.rzrx_cz_circuit(n, 12, seed=5) + wc.random_mixed_circuit(n, 60, seed=5, kmax=2)
    got, _ = emulator(n, circ, mode=mode, dtype=dtype, arith=arith, **kw)
    check(got, circ, n)
    steps = emulator.steps
    assert storage_forms_consistent(steps), steps
    uses_df = any("d" in t[1:3] for t in steps if t[0] == "P")
    if dtype == "c128" and arith == "df" and "renorm_every" not in kw:
        assert sum(t[0] == "P" for t in steps) >= 2 and uses_df, steps
    if arith != "df":
        assert not uses_df, steps


@pytest.mark.parametrize("dtype,arith", MODES)
def test_compiles_on_many_threads_at_once(emulator, dtype, arith):
    """Batch builds and the server compile on many host threads at once, and the compiler
    keeps its working arrays per thread: eight threads compiling the same circuits three
    times each produce the serial plan byte for byte (stages, register ops, pool entries)."""
    rng = np.random.default_rng(13)
    for n, circ in ((12, wc.rzrx_cz_circuit(12, 10, seed=13)), (14, wc.mixed_batch_circuit(14, 30, rng)),
                    (11, wc.qft_like_circuit(11))):
        emulator(n, circ, dtype=dtype, arith=arith, threads=8)
        assert emulator.threads_consistent == 1


def out_of_place(steps):
    """Steps that write the state into the second buffer: a permutation kernel, or a tile
    pass whose store carries a permutation."""
    return [t for t in steps if t == "X" or (t[0] == "P" and t.endswith("s"))]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_tile_plans_run_in_place(emulator, dtype):
    """The serving memory admission counts one state vector per request because tile-mode
    plans (what the server compiles) never write the state out of place: no permutation
    kernel, no permutation fused into a pass's store, whatever the circuit.  Algorithm 1's
    plans on the same circuits do both, so the check can see them."""
    n = 12
    circs = [wc.rzrx_cz_circuit(n, 10, seed=3), wc.qft_like_circuit(n), wc.haar_cnot_circuit(n, 8, 4),
             wc.random_mixed_circuit(n, 200, seed=3, kmax=3), wc.single_qubit_run_circuit(n, 6, seed=3)]
    seen_paper = []
    for circ in circs:
        for kw in ({}, {"tile_bits": 8}, {"tile_bits": 8, "renorm_every": 2}):
            emulator(n, circ, mode="tile", dtype=dtype, **kw)
            assert not out_of_place(emulator.steps), (kw, emulator.steps)
        emulator(n, circ, mode="paper", dtype=dtype, tile_bits=8)
        seen_paper += out_of_place(emulator.steps)
    assert any(t == "X" for t in seen_paper) and any(t != "X" for t in seen_paper), seen_paper


@pytest.mark.parametrize("dtype,arith", MODES)
def test_tangent_growth_stays_bounded_in_long_passes(emulator, dtype, arith):
    """A pass of hundreds of tangent-form RX (a deep Haar + CNOT circuit on a tile-sized state,
    every Haar 2x2 fused into diag . RX . diag) keeps its register magnitudes within 2^25 of
    the unit-norm state, and no register op scales by less than 2^-25: the dropped cos / sin
    factors are absorbed in segments (one product of all of them would be ~2^-200, zero in
    FP32)."""
    n = 10
    circ = wc.haar_cnot_circuit(n, 120, seed=9)
    got, _ = emulator(n, circ, mode="tile", dtype=dtype, arith=arith, tile_bits=10)
    check(got, circ, n)
    assert emulator.max_register_abs < 2.0 ** 25, emulator.max_register_abs
    assert emulator.min_register_scale > 2.0 ** -25, emulator.min_register_scale


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_tile_mode_every_register_width(emulator, dtype, arith, K):
    if dtype == "c128" and K > 4:
        pytest.skip("complex128 holds at most 4 register bits")
    n = 12
    circ = wc.random_mixed_circuit(n, 160, seed=100 + K, kmax=3) + wc.rzrx_cz_circuit(n, 6, seed=K)
    got, _ = emulator(n, circ, mode="tile", dtype=dtype, arith=arith, tile_bits=10, reg_bits=K)
    check(got, circ, n)


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("full_rx", [False, True])
def test_rzrx_cz_construction(emulator, dtype, arith, full_rx):
    """The 30-qubit workload's construction: tangent-form RX runs (both forms), phase tables
    with masks, the pass-level factor folded into the first table, CZ sign flips."""
    n = 14
    circ = wc.rzrx_cz_circuit(n, 24, seed=3)
    got, nsteps = emulator(n, circ, mode="tile", dtype=dtype, arith=arith, tile_bits=10, full_rx=full_rx)
    assert nsteps > 1
    check(got, circ, n)


@pytest.mark.parametrize("dtype,arith", MODES)
@pytest.mark.parametrize("n,m", [(10, 6), (12, 8)])
def test_paper_mode(emulator, dtype, arith, n, m):
    circ = wc.paper_random_circuit(n, 0.3, seed=n) + wc.rzrx_cz_circuit(n, 3, seed=n)
    got, _ = emulator(n, circ, mode="paper", dtype=dtype, arith=arith, tile_bits=m)
    check(got, circ, n)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_pergate_mode(emulator, dtype, arith):
    n = 9
    circ = wc.random_mixed_circuit(n, 120, seed=9, kmax=4)
    got, _ = emulator(n, circ, mode="pergate", dtype=dtype, arith=arith)
    check(got, circ, n)


@pytest.mark.parametrize("dtype,arith", MODES)
def test_controlled_diagonals_in_phase_tables(emulator, dtype, arith):
    n = 12
    rng = np.random.default_rng(5)
    circ = []
    for layer in range(6):
        for q in range(n):
            circ.append(wc.Gate("RX", (q,), param=float(rng.uniform(0, 2 * np.pi))))
        for _ in range(n):
            cq, t = (int(x) for x in rng.choice(n, 2, replace=False))
            a, b = rng.uniform(0, 2 * np.pi, 2)
            circ.append(wc.Gate("CU", (cq, t), matrix=np.diag([np.exp(1j * a), np.exp(1j * b)])))
    got, _ = emulator(n, circ, mode="tile", dtype=dtype, arith=arith, tile_bits=10)
    check(got, circ, n)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_default_options(emulator, dtype):
    """Default tile / low / register bits, as qs_compile fills them in."""
    n = 14
    circ = wc.rzrx_cz_circuit(n, 10, seed=21) + wc.random_mixed_circuit(n, 60, seed=21, kmax=3)
    got, _ = emulator(n, circ, dtype=dtype)
    check(got, circ, n)


@pytest.mark.parametrize("mode", ["tile", "paper", "pergate"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_appendix_c_and_config1_circuits(emulator, mode, dtype):
    """The QFT-like circuit of Appendix C (controlled phases, Hadamards) and 12-qubit
    Haar + CNOT layers, in every mode."""
    kw = {"tile_bits": 8} if mode == "paper" else {}
    for n, circ in ((11, wc.qft_like_circuit(11)), (11, wc.qft_circuit(11)), (12, wc.haar_cnot_circuit(12, 8, 2))):
        got, _ = emulator(n, circ, mode=mode, dtype=dtype, **kw)
        check(got, circ, n)


def test_periodic_renormalisation(emulator):
    n = 10
    circ = wc.rzrx_cz_circuit(n, 8, seed=4)
    got, _ = emulator(n, circ, mode="tile", dtype="c64", tile_bits=8, renorm_every=2)
    check(got, circ, n)


def test_emulator_sees_a_planted_mistake(emulator):
    """The check has teeth: the same plan against a circuit with one angle changed fails."""
    n = 10
    circ = wc.rzrx_cz_circuit(n, 6, seed=8)
    got, _ = emulator(n, circ, mode="tile", dtype="c128", tile_bits=8)
    wrong = list(circ)
    g = wrong[17]
    wrong[17] = wc.Gate(g.kind, tuple(g.qubits), param=float(g.param) + 1e-3)
    ref_wrong = sv.simulate(n, wrong)
    assert float(np.max(np.abs(got - ref_wrong))) > 1e-6


def cheap_dense_model():
    """A cost model under which dense tensor-core blocks are cheap and tile-pass arithmetic
    dear, so that the compiler picks dense blocks even on small states."""
    m = _lib.qs_cost_model()
    for i, v in enumerate((0.005, 1e-10, 1e-6)):
        m.tile[i] = v
    for i, v in enumerate((0.0, 1e-12, 0.0)):
        m.dense[i] = v
    for i, v in enumerate((0.005, 1e-10, 0.0)):
        m.gate[i] = v
        m.permute[i] = v
    return m


@pytest.mark.parametrize("n", [12, 14])
def test_dense_blocks_fused_by_the_compiler(emulator, n):
    """Where the cost model prefers them, gates on storage bits 0..5 leave the tile passes
    for dense 64 x 64 blocks; the fused blocks reproduce the circuit exactly (in FP64 here;
    on the GPU the tensor cores add complex64-level rounding)."""
    circ = wc.rzrx_cz_circuit(n, 8, seed=n) + wc.haar_cnot_circuit(n, 3, seed=n) + \
        wc.random_mixed_circuit(n, 60, seed=n, kmax=3)
    ops, nops, mats = qs.marshal(circ)
    o = qs._opts(mode="tile", dtype="c64")
    model = cheap_dense_model()
    o.cost = ctypes.pointer(model)
    h = ctypes.c_void_p()
    _lib.check(_lib.load().qs_compile(n, ops, nops, mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mats.size,
                                      None, ctypes.byref(o), ctypes.byref(h)))
    st = _lib.qs_plan_stats()
    _lib.check(_lib.load().qs_plan_get_stats(h, ctypes.byref(st)))
    _lib.load().qs_plan_destroy(h)
    assert st.n_dense > 0 and st.predicted_ms > 0
    got, _ = emulator(n, circ, cost=model, mode="tile", dtype="c64")
    check(got, circ, n)


def test_no_dense_flag_and_default_model(emulator):
    """QS_FLAG_NO_DENSE keeps every gate in tile passes; the default model picks no dense
    block on a small state (the launch would cost more than the arithmetic it saves), and
    complex128 plans never get one."""
    n = 14
    circ = wc.rzrx_cz_circuit(n, 8, seed=3)
    for dtype, kw, want in (("c64", {}, 0), ("c64", {"flags": _lib.QS_FLAG_NO_DENSE}, 0), ("c128", {}, 0)):
        model = cheap_dense_model() if kw or dtype == "c128" else None
        ops, nops, mats = qs.marshal(circ)
        o = qs._opts(mode="tile", dtype=dtype)
        o.flags |= kw.get("flags", 0)
        if model is not None:
            o.cost = ctypes.pointer(model)
        h = ctypes.c_void_p()
        _lib.check(_lib.load().qs_compile(n, ops, nops, mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          mats.size, None, ctypes.byref(o), ctypes.byref(h)))
        st = _lib.qs_plan_stats()
        _lib.check(_lib.load().qs_plan_get_stats(h, ctypes.byref(st)))
        _lib.load().qs_plan_destroy(h)
        assert st.n_dense == want, (dtype, kw)


def test_random_configurations(emulator):
    """Seeded random circuits and compile options together: 3-12 qubits; every gate kind, or
    a few kinds, or diagonal-heavy, X-heavy, single-qubit runs, the benchmark construction
    plus Appendix C's circuit; tile, Algorithm 1 and per-gate modes; random tile, low and
    register bits, renormalisation, full-form RX, fusion off.  Every plan matches the oracle;
    the only refusal allowed is a gate wider than the tile the options leave room for."""
    kinds_all = [k for k in wc.KINDS if k != "RELABEL"]
    diag = ["Z", "S", "T", "RZ", "P", "CZ", "CP", "U1"]
    xs = ["X", "RX", "CNOT", "H", "U1", "RY"]
    refused = 0
    for seed in range(150):
        rng = np.random.default_rng(1000 + seed)
        n = int(rng.integers(3, 13))
        dtype, arith = MODES[int(rng.integers(0, 3))]
        mode = ["tile", "tile", "tile", "paper", "pergate"][int(rng.integers(0, 5))]
        which = int(rng.integers(0, 6))
        kmax = int(rng.integers(1, 4))
        ng = int(rng.integers(1, 300))
        if which == 0:
            circ = wc.random_mixed_circuit(n, ng, seed=seed, kmax=kmax)
        elif which == 1:
            kinds = [str(k) for k in rng.choice(kinds_all, size=int(rng.integers(1, 5)), replace=False)]
            circ = wc.random_mixed_circuit(n, ng, seed=seed, kinds=kinds, kmax=kmax)
        elif which == 2:
            circ = wc.random_mixed_circuit(n, ng, seed=seed, kinds=diag, kmax=kmax)
        elif which == 3:
            circ = wc.random_mixed_circuit(n, ng, seed=seed, kinds=xs, kmax=kmax)
        elif which == 4:
            circ = wc.single_qubit_run_circuit(n, int(rng.integers(1, 8)), seed=seed)
        else:
            circ = wc.rzrx_cz_circuit(n, int(rng.integers(1, 10)), seed=seed) + wc.qft_like_circuit(n)
        kw = {}
        if mode != "pergate":
            if rng.random() < 0.7:
                kw["tile_bits"] = int(rng.integers(min(n, 3), n + 1))
                if rng.random() < 0.5:
                    kw["low_bits"] = int(rng.integers(0, max(1, kw["tile_bits"] - 2)))
            if rng.random() < 0.3:
                kw["reg_bits"] = int(rng.integers(1, 6))
        if rng.random() < 0.2:
            kw["renorm_every"] = int(rng.integers(1, 4))
        if rng.random() < 0.2:
            kw["full_rx"] = True
        if rng.random() < 0.2:
            kw["fuse"] = False
        what = f"seed {seed}: n={n} {dtype}/{arith} {mode} circuit {which} {kw}"
        try:
            got, _ = emulator(n, circ, mode=mode, dtype=dtype, arith=arith, **kw)
        except AssertionError as e:
            assert "needs more qubits than a tile holds" in str(e) and "tile_bits" in kw, (what, str(e)[-500:])
            refused += 1
            continue
        ref = sv.simulate(n, circ)
        err = float(np.max(np.abs(got - ref)))
        assert err <= TOL, (what, err)
    assert refused < 40, refused

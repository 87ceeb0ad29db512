"""GPU: the autotuner picks compile options among timed candidates and caches them; the
options it returns give the same amplitudes as any other tile width (within tolerance)."""
import os

import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")
pytest.importorskip("torch")
from paper_2010_09746_gb300 import tuning  # noqa: E402


def test_autotune_and_cache(tmp_path):
    n = 16
    circ = wc.rzrx_cz_circuit(n, 8, seed=2)
    cache = os.path.join(tmp_path, "tune.json")
    r = tuning.autotune(n, circ, dtype="c128", tile_bits=(10, 12), reg_bits=(3, 4), low_bits=(3, 4), measure_top=2,
                        cache_path=cache)
    assert r["tile_bits"] in (10, 12) and r["reg_bits"] in (3, 4) and r["low_bits"] in (3, 4)
    assert len(r["candidates"]) == 2 and len(r["ranked"]) == 8
    r2 = tuning.autotune(n, circ, dtype="c128", cache_path=cache)
    assert r2.get("cached") and r2["tile_bits"] == r["tile_bits"]
    st = qs.State(n, "c128")
    st.execute(qs.compile(n, circ, mode="tile", dtype="c128", tile_bits=r["tile_bits"], reg_bits=r["reg_bits"],
                          low_bits=r["low_bits"]))
    assert np.abs(st.amplitudes() - sv.simulate(n, circ)).max() <= 1e-12


def test_cost_model_fit_on_measured_plans():
    import torch
    m = tuning.CostModel()
    st = qs.State(18, "c64")
    plans = []
    for layers in (2, 4, 8):
        for mode in ("tile", "pergate"):
            p = qs.compile(18, wc.rzrx_cz_circuit(18, layers, seed=layers), mode=mode, dtype="c64")
            st.set_profiling(True)
            st.reset_kernel_stats()
            tuning.time_plan(p, st)
            m.add_kernel_stats(st.kernel_stats())
            st.set_profiling(False)
            plans.append(p)
    coef = m.fit()
    assert "tile_pass_c64" in coef and "gate_c64" in coef
    assert all(x >= 0 for c in coef.values() for x in c)
    for p in plans:
        assert m.predict_plan(p, "c64") > 0


def test_autotune_batch():
    work = [(10 + (i % 4), wc.rzrx_cz_circuit(10 + (i % 4), 4, seed=i)) for i in range(24)]
    r = tuning.autotune_batch(work, dtype="c64", tile_bits=(8, 10), reps=2)
    assert r["tile_bits"] in (8, 10) and len(r["candidates"]) == 2
    b = qs.Batch(work, dtype="c64", tile_bits=r["tile_bits"])
    b.run()
    b.sync()
    for i in (0, 5, 23):
        n, c = work[i]
        ref = sv.simulate(n, c)
        got = b.amplitudes(i).astype(np.complex128)
        assert sv.fidelity_loss(got, ref) <= 1e-5

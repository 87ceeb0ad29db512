"""CPU: the cost model's least-squares fit recovers known per-launch / per-byte / per-
instruction costs, and circuit keys for the autotuner cache are stable and distinct."""
import numpy as np

from paper_2010_09746_gb300 import tuning
from workloads import circuits as wc


def test_cost_model_recovers_coefficients():
    rng = np.random.default_rng(0)
    m = tuning.CostModel()
    true = (0.004, 1.5e-10, 2.5e-11)      # ms per launch, per byte, per instruction
    for _ in range(40):
        l, b, a = rng.integers(1, 100), rng.uniform(1e9, 1e12), rng.uniform(1e10, 1e14)
        m.add("tile_pass_c128_df", l, b, a, true[0] * l + true[1] * b + true[2] * a)
    c = m.fit()["tile_pass_c128_df"]
    np.testing.assert_allclose(c, true, rtol=1e-6)
    assert max(abs(r) for r in m.residuals("tile_pass_c128_df")) < 1e-6


def test_plan_class_features():
    import paper_2010_09746_gb300 as qs
    n = 14
    circ = wc.rzrx_cz_circuit(n, 6, seed=1)
    S = (1 << n) * 8
    p = qs.compile(n, circ, mode="tile", dtype="c64")
    f = tuning.plan_class_features(p, "c64")
    st = p.stats()
    assert set(f) == {"tile_pass_c64"}
    assert f["tile_pass_c64"] == (st["n_passes"], 2 * S * st["n_passes"], st["alu_instr"])
    p = qs.compile(n, circ, mode="pergate", dtype="c64")
    f = tuning.plan_class_features(p, "c64")
    assert set(f) == {"gate_c64"} and f["gate_c64"][1] == p.stats()["hbm_bytes"]
    p = qs.compile(n, circ, mode="paper", dtype="c64", tile_bits=8)
    f = tuning.plan_class_features(p, "c64")
    st = p.stats()
    assert sum(v[1] for v in f.values()) == st["hbm_bytes"]
    m = tuning.CostModel(coef={k: [0.01, 1e-10, 1e-12] for k in ("tile_pass_c64", "permute", "gate_c64")})
    assert m.predict_plan(p, "c64") > 0


def test_circuit_key():
    a = wc.rzrx_cz_circuit(10, 3, seed=1)
    b = wc.rzrx_cz_circuit(10, 3, seed=2)
    assert tuning.circuit_key(10, "c128", a) == tuning.circuit_key(10, "c128", list(a))
    assert tuning.circuit_key(10, "c128", a) != tuning.circuit_key(10, "c128", b)
    assert tuning.circuit_key(10, "c128", a) != tuning.circuit_key(10, "c64", a)

"""Cost model fitted to measured kernel times, and an autotuner for tile width / register bits.

The paper estimates a circuit's simulation time by summing benchmarked per-operation times
(Sec. 4) and notes that a compiler pass could draw on those benchmarks in full (Sec. 3).  Here every plan reports, per execution, its kernel launches, its
algorithmic HBM bytes and the arithmetic instructions its formulas need (qs_plan_stats);
the cost model is the least-squares fit

    t = c_launch * launches + c_byte * bytes + c_alu * alu_instructions

over launches timed with CUDA events (qs_set_profiling).  `autotune` compiles the
candidate tile widths / register bits on the host, ranks them with the model, times the
best few on the GPU and keeps the fastest; results are cached in a JSON file keyed by
device, qubit count, dtype and a hash of the circuit.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

from . import Plan, State, compile as qs_compile


def plan_features(plan: Plan) -> Tuple[float, float, float]:
    s = plan.stats()
    launches = s["n_passes"] + s["n_pergate"] + s["n_permute_kernels"]
    return float(launches), float(s["hbm_bytes"]), float(s["alu_instr"])


def plan_class_features(plan: Plan, dtype: str) -> Dict[str, Tuple[float, float, float]]:
    """(launches, bytes, alu) of a plan per kernel class: tile passes and permutations read
    and write the state once each; the per-gate kernels take the remaining bytes; the
    arithmetic is charged to the tile passes when there are any, else to the gates."""
    s = plan.stats()
    S = float((1 << plan.n) * (16 if dtype == "c128" else 8))
    pol = {"c64": "c64", "c128": "c128_df"}[dtype]
    out = {}
    b_pass, b_perm = 2 * S * s["n_passes"], 2 * S * s["n_permute_kernels"]
    b_dense = 2 * S * s.get("n_dense", 0)
    if s["n_passes"]:
        out[f"tile_pass_{pol}"] = (float(s["n_passes"]), b_pass, float(s["alu_instr"]))
    if s["n_permute_kernels"]:
        out["permute"] = (float(s["n_permute_kernels"]), b_perm, 0.0)
    if s.get("n_dense", 0):
        out["dense_mma_c64"] = (float(s["n_dense"]), b_dense, 0.0)
    if s["n_pergate"]:
        out[f"gate_{pol}"] = (float(s["n_pergate"]), max(0.0, s["hbm_bytes"] - b_pass - b_perm - b_dense),
                              0.0 if s["n_passes"] else float(s["alu_instr"]))
    return out


@dataclass
class CostModel:
    """Per kernel class (the names qs_get_kernel_stats reports, e.g. tile_pass_c64):
    t[ms] = c_launch * launches + c_byte * bytes + c_alu * alu, fitted by least squares to
    measured totals of that class (minimum-norm solution where the samples do not separate
    the terms, negative coefficients clipped to zero)."""
    coef: Dict[str, List[float]] = field(default_factory=dict)
    samples: Dict[str, List[Tuple[float, float, float, float]]] = field(default_factory=dict)

    def add(self, cls: str, launches: float, bytes_: float, alu: float, ms: float):
        self.samples.setdefault(cls, []).append((launches, bytes_, alu, ms))

    def add_kernel_stats(self, kstats: Iterable[dict]):
        for k in kstats:
            if k["launches"] > 0:
                self.add(k["name"], float(k["launches"]), float(k["bytes"]), float(k["alu"]), float(k["total_ms"]))

    def fit(self) -> Dict[str, List[float]]:
        for cls, rows in self.samples.items():
            a = np.array([[r[0], r[1] * 1e-9, r[2] * 1e-12] for r in rows])
            y = np.array([r[3] for r in rows])
            c, *_ = np.linalg.lstsq(a, y, rcond=None)
            c = np.maximum(c, 0.0)   # a negative cost per unit has no meaning
            self.coef[cls] = [float(c[0]), float(c[1]) * 1e-9, float(c[2]) * 1e-12]
        return self.coef

    def predict(self, cls: str, launches: float, bytes_: float, alu: float) -> float:
        c = self.coef[cls]
        return c[0] * launches + c[1] * bytes_ + c[2] * alu

    def predict_plan(self, plan: Plan, dtype: str) -> Optional[float]:
        """Sum over the plan's kernel classes; None if a class has no fit."""
        total = 0.0
        for cls, f in plan_class_features(plan, dtype).items():
            if cls not in self.coef:
                return None
            total += self.predict(cls, *f)
        return total

    def residuals(self, cls: str) -> List[float]:
        return [r[3] - self.predict(cls, r[0], r[1], r[2]) for r in self.samples.get(cls, [])]

    def to_json(self) -> dict:
        return {"coef_ms_per_launch_byte_alu": self.coef}

    def native(self, dtype: str, arith: str = "auto"):
        """The fitted coefficients as the compiler's qs_cost_model for plans of this dtype
        (classes without samples keep the library's defaults), so that qs_compile's choices
        and its predicted_ms follow the measured kernel times."""
        from . import default_cost_model
        m = default_cost_model(dtype, arith)
        pol = {"c64": "c64", "c128": "c128_f64" if arith == "f64" else "c128_df"}[dtype]
        for field_, cls in (("tile", f"tile_pass_{pol}"), ("gate", f"gate_{pol}"), ("permute", "permute"),
                            ("dense", "dense_mma_c64")):
            if cls in self.coef:
                arr = getattr(m, field_)
                for i in range(3):
                    arr[i] = self.coef[cls][i]
        return m


def circuit_key(n: int, dtype: str, circuit: Sequence) -> str:
    h = hashlib.sha1()
    h.update(f"{n}:{dtype}".encode())
    for g in circuit:
        h.update(f"{g.kind}{tuple(g.qubits)}{float(getattr(g, 'param', 0.0) or 0.0):.17g}".encode())
        m = getattr(g, "matrix", None)
        if m is not None:
            h.update(np.ascontiguousarray(m, dtype=np.complex128).tobytes())
    return h.hexdigest()


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:  # noqa: BLE001
        return "unknown"


def time_plan(plan: Plan, state: State, reps: int = 2) -> float:
    """Milliseconds per execution (reset + plan) with CUDA events on the state's stream."""
    import torch
    stream = torch.cuda.current_stream()
    state.set_stream(stream)
    state.reset()
    state.execute(plan)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        state.reset()
        state.execute(plan)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(n: int, circuit: Sequence, dtype: str = "c128", model: Optional[CostModel] = None,
             tile_bits: Sequence[int] = (11, 12, 13), reg_bits: Sequence[int] = (3, 4, 5), measure_top: int = 2,
             cache_path: Optional[str] = None, state: Optional[State] = None,
             low_bits: Sequence[int] = (0,)) -> dict:
    """Pick tile width L, register bits K and segment bits c (low_bits; 0 = the dtype's
    default) for `circuit`: rank every candidate with the cost model (or by predicted bytes
    + instructions when no model is given), time the best `measure_top` on the GPU, return
    the fastest as compile options."""
    circuit = list(circuit)
    key = circuit_key(n, dtype, circuit)
    dev = _device_name()
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    ck = f"{dev}|{key}"
    if ck in cache:
        return dict(cache[ck], cached=True)
    kmax = 4 if dtype == "c128" else 5
    cands = []
    for L in tile_bits:
        for K in reg_bits:
            for c in low_bits:
                if K > kmax or L > n or L - K < 0 or c > L:
                    continue
                p = qs_compile(n, circuit, mode="tile", dtype=dtype, tile_bits=L, reg_bits=K, low_bits=c)
                launches, b, a = plan_features(p)
                pred = model.predict_plan(p, dtype) if model is not None else None
                if pred is None:   # rough: the HBM time plus the arithmetic at half the FP32 issue rate
                    pred = b / 6.8e12 * 1e3 + a / 20e12 * 1e3
                cands.append((pred, L, K, c, p))
    cands.sort(key=lambda t: t[0])
    own = state is None
    st = state or State(n, dtype)
    measured = []
    for pred, L, K, c, p in cands[:max(1, measure_top)]:
        ms = time_plan(p, st)
        measured.append({"tile_bits": L, "reg_bits": K, "low_bits": c, "predicted_ms": pred, "measured_ms": ms})
    if own:
        st.close()
    best = min(measured, key=lambda r: r["measured_ms"])
    out = {"tile_bits": best["tile_bits"], "reg_bits": best["reg_bits"], "low_bits": best["low_bits"],
           "measured_ms": best["measured_ms"], "candidates": measured,
           "ranked": [(round(c[0], 3), c[1], c[2], c[3]) for c in cands]}
    if cache_path:
        cache[ck] = {k: out[k] for k in ("tile_bits", "reg_bits", "low_bits", "measured_ms")}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return out


def autotune_batch(work, dtype: str = "c64", tile_bits: Sequence[int] = (11, 12, 13), reps: int = 3) -> dict:
    """Tile width for a batch of small circuits (fusion width of every circuit's passes):
    build the batch at each candidate width, time `reps` graph-replayed runs, keep the
    fastest."""
    import torch
    from . import Batch
    stream = torch.cuda.Stream()
    res = []
    arrays = Batch.marshal(work)   # once for every candidate
    for L in tile_bits:
        b = Batch(dtype=dtype, stream=stream, tile_bits=L, marshalled=arrays)
        for _ in range(2):
            b.run()
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            b.run()
        e1.record(stream)
        b.sync()
        res.append({"tile_bits": L, "ms": e0.elapsed_time(e1) / reps, "waves": b.stats()["n_waves"]})
        del b
    best = min(res, key=lambda r: r["ms"])
    return {"tile_bits": best["tile_bits"], "ms": best["ms"], "candidates": res}

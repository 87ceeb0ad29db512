#!/usr/bin/env python3
"""Benchmark: 30-qubit random-circuit simulation on one GB300 (replicas on N GPUs).

Workload (default): 30 qubits, complex128 (16 GiB state), 40 layers of RZ(U(0,2pi)) and
RX(U(0,2pi)) on every qubit followed by floor(n/4) CZ on pairs biased toward high qubits
(seed 0; 2680 gates).  One step = state preparation |0..0> + the compiled circuit (tile
passes, and permutations / per-gate kernels where the mode uses them) + the FP64 norm
read-out.  The plan is compiled before the timed region; `e2e` compiles from host buffers
every step and copies inputs / results between host and device inside its timed region.

`value` = circuit gates / device-timed step time (CUDA events on the library's stream),
whole job (sum over replicas).  The state (16 GiB) is far larger than L2 (129 MB), so no
flush is needed between steps.  `modes` reports the same circuit without the reordering
pass (one kernel per gate, measured on the first 4 layers) and with the paper's
Algorithm 1 (m = 12 local qubits, one transposition per PermuteQubits).

`--impl reference` times the FP64 CPU oracle (test infrastructure) on this host's cores on
a bounded sample of the same workload (the first gates of the same circuit on the same
30-qubit state), the only other place this file runs oracle code.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import circuits as wc  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
FP32_LANES = 128        # FP32 FMA-pipe lanes per SM (4 partitions x 32)
FP64_PER_CLK = 1.7      # DFMA per clock per SM on GB300, measured with a register-resident probe


def device_info(dev, clk):
    """SM count from the device properties; SM clock: the maximum nvidia-smi reported during
    the timed region, else the measured one."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    peaks, _ = load_peaks()
    mhz = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    return {"sms": int(props.multi_processor_count), "sm_max_mhz": float(mhz), "name": props.name}


# FP64 floating-point operations per amplitude that each gate needs as the method writes it
# (complex 2x2 on an amplitude pair: 2 complex multiplies + 1 add = 14 per amplitude; a
# diagonal phase: 1 complex multiply = 6; sign flips and swaps: 0; a control halves the
# amplitudes touched; a general 4x4: 4 multiplies + 3 adds = 30 per amplitude).
METHOD_FLOPS = {"U1": 14, "H": 14, "RX": 14, "RY": 14, "Y": 0, "X": 0, "Z": 0, "RZ": 6, "P": 6 / 2, "S": 6 / 2,
                "T": 6 / 2, "CZ": 0, "CNOT": 0, "CP": 6 / 4, "CU": 14 / 2, "SWAP": 0, "U2": 30}


def method_flops(circ, n):
    return sum(METHOD_FLOPS[g.kind] for g in circ) * float(1 << n)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


def workload(args):
    if args.workload == "rzrx30":
        circ = wc.rzrx_cz_circuit(args.n, args.layers, seed=args.seed)
        name = f"rzrx_cz_{args.n}q_{args.layers}layers_{args.dtype}"
        return args.n, circ, name
    if args.workload == "haar12":
        circ = wc.haar_cnot_circuit(12, 20, seed=args.seed)
        return 12, circ, f"haar_cnot_12q_20layers_{args.dtype}"
    raise SystemExit(f"unknown workload {args.workload}")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:  # noqa: BLE001
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def reduce_max(value, pg):
    """Max over ranks (the slowest replica sets the whole job's time)."""
    if pg is None:
        return float(value)
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, max_ms):
    """Whole-job throughput: every rank processed `units_per_rank`; time = slowest rank."""
    return world * units_per_rank / (max_ms / 1e3)


KERNEL_SOURCES = ("paper_2010_09746_gb300/csrc/kernels_tile.cu", "paper_2010_09746_gb300/csrc/arith.cuh")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(kernel_name, n):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary
    (profiles/<kernel>.md, measured on a smaller state and scaled by the amplitudes one
    launch processes), or None when the kernel source changed since the capture."""
    import re
    path = os.path.join(ROOT, "profiles", f"{kernel_name}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_source_sha1:\s*([0-9a-f]{40})", text)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)\s+at\s+n\s*=\s*(\d+)", text)
    if not m_hash or not m_b or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_b.group(1)) * 2.0 ** (n - int(m_b.group(2)))


def roofline(kstats, steps, step_ms, peaks, peaks_kind, policy, dev, circ_flops):
    """Roofline of the dominant kernel (the most device time per step).

    bound / frac: the HBM fraction -- algorithmic bytes per launch (2 S for a tile pass: the
    state read and written once) over the launch's CUDA-event time, against the measured copy
    bandwidth.  `method_alu`: the FP64 flops the circuit's gates need (METHOD_FLOPS; all of the
    circuit's arithmetic runs in this kernel, split evenly over its launches) per second,
    against the native FP64 pipe.  `fma_pipe`: a diagnostic, not the method's work -- the
    lane operations the arithmetic's own formulas issue (for complex128 that is the
    double-float emulation), against the FP32 FMA lanes at the maximum clock."""
    if not kstats:
        return None
    dom = max(kstats, key=lambda k: k["total_ms"])
    per_launch_ms = dom["total_ms"] / dom["launches"]
    launches_per_step = dom["launches"] / steps
    bytes_pl = dom["bytes"] / dom["launches"]
    alu_pl = dom["alu"] / dom["launches"]
    hbm = bytes_pl / (per_launch_ms * 1e-3) / 1e9
    clk = dev["sm_max_mhz"] * 1e6
    out = {"kernel": dom["name"], "launches_per_step": launches_per_step,
           "ms_per_launch": round(per_launch_ms, 4), "share_of_step": round(dom["total_ms"] / steps / step_ms, 4),
           "bound": "hbm", "achieved": round(hbm, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": round(hbm / peaks["hbm_gbs"], 4), "peak_source": f"{peaks_kind} hbm_gbs (copy)",
           "traffic": None, "algorithmic_bytes": bytes_pl}
    if circ_flops and dom["name"].startswith("tile_pass"):
        fl = circ_flops / launches_per_step
        fp64_peak = dev["sms"] * FP64_PER_CLK * 2 * clk / 1e12
        ach = fl / (per_launch_ms * 1e-3) / 1e12
        out["method_alu"] = {"fp64_flops_per_launch": fl, "achieved_tflops": round(ach, 3),
                             "fp64_pipe_peak_tflops": round(fp64_peak, 3), "frac_of_fp64_pipe": round(ach / fp64_peak, 3),
                             "peak_source": f"{dev['sms']} SMs x {FP64_PER_CLK} DFMA/clk (measured) x 2 x "
                                            f"{dev['sm_max_mhz']:.0f} MHz"}
    lanes = FP64_PER_CLK if policy == "f64" else FP32_LANES
    peak_alu = dev["sms"] * lanes * clk / 1e12
    alu = alu_pl / (per_launch_ms * 1e-3) / 1e12
    out["fma_pipe"] = {"lane_ops_per_launch": alu_pl, "achieved": round(alu, 3), "peak": round(peak_alu, 2),
                       "unit": "T DFMA/s" if policy == "f64" else "T FP32 lane-ops/s", "frac": round(alu / peak_alu, 4),
                       "what": "instructions the arithmetic's formulas issue (double-float emulation for complex128): "
                               "FMA-pipe occupancy, not the method's work",
                       "peak_source": f"{dev['sms']} SMs x {lanes}/clk x {dev['sm_max_mhz']:.0f} MHz"}
    return out


def measure(qs, st, plan, steps, warmup, torch, stream, profile=False):
    """Time `steps` steps (state preparation + plan + FP64 norm); `plan` may be a list,
    step i then runs plan i mod len."""
    plans = plan if isinstance(plan, (list, tuple)) else [plan]
    it = [0]

    def step():
        st.reset()
        st.execute(plans[it[0] % len(plans)])
        it[0] += 1
        return st.norm()

    for _ in range(warmup):
        step()
    it[0] = 0
    torch.cuda.synchronize()
    if profile:
        st.set_profiling(True)
        st.reset_kernel_stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    norms = [step() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ks = st.kernel_stats() if profile else []
    if profile:
        st.set_profiling(False)
    return e0.elapsed_time(e1) / steps, norms, ks


def per_gate_bound(qs, n, circ, args, peaks, gates_per_s):
    """What a simulator that moves the state through HBM once per gate could reach at best:
    the per-gate plan's algorithmic bytes (2 S per gate, less for controlled and diagonal
    two-qubit gates) at the measured copy bandwidth; `ratio` = this path's gates/s over it."""
    p = qs.compile(n, circ, mode="pergate", dtype=args.dtype, arith=args.arith)
    b = p.stats()["hbm_bytes"]
    ideal = len(circ) / (b / (peaks["hbm_gbs"] * 1e9))
    return {"bytes_per_circuit": b, "ideal_gates_per_s": round(ideal, 2), "ratio": round(gates_per_s / ideal, 3)}


def fit_cost_model(qs, torch, st, stream, args, runs):
    """Per kernel class, least squares t = c_launch*launches + c_byte*bytes + c_alu*instructions
    over the CUDA-event totals of the training runs (one sample per class and run).  The
    fitted model then goes into the compiler (qs_compile_opts.cost), which predicts each
    plan's time (predicted_ms); the check is out of sample: circuits the fit never saw (another
    seed of the same construction, 28 qubits, Appendix C's QFT-like circuit under the tile
    passes and under Algorithm 1), each measured once after a warm-up."""
    from paper_2010_09746_gb300 import tuning
    m = tuning.CostModel()
    for _, (_, _, ks, steps) in runs.items():
        m.add_kernel_stats([dict(k, launches=k["launches"] / steps, total_ms=k["total_ms"] / steps,
                                 bytes=k["bytes"] / steps, alu=k["alu"] / steps) for k in ks])
    coef = m.fit()
    native = m.native(args.dtype, args.arith)
    init_norm = sum(m.predict(c, 1, (1 << args.n) * (16 if args.dtype == "c128" else 8), 0)
                    for c in ("init", "norm") if c in coef)

    def predicted(n, circ, **kw):
        p = qs.compile(n, circ, dtype=args.dtype, arith=args.arith, cost=native, **kw)
        return p, p.stats()["predicted_ms"]

    train = {}
    for name, (p, ms, _, _) in runs.items():
        _, pr = predicted(p.n, runs_circuits[name], **runs_opts[name])
        train[name] = {"predicted_ms": round(pr + init_norm, 3), "measured_ms": round(ms, 3)}
    held = {}
    cases = [("rzrx_30q_seed1_tile", args.n, wc.rzrx_cz_circuit(args.n, args.layers, seed=args.seed + 1), {"mode": "tile"}),
             ("qft_like_30q_tile", args.n, wc.qft_like_circuit(args.n), {"mode": "tile"}),
             ("qft_like_30q_alg1_m12", args.n, wc.qft_like_circuit(args.n), {"mode": "paper", "tile_bits": 12})]
    for name, n, circ, kw in cases:
        p, pr = predicted(n, circ, **kw)
        ms, _, _ = measure(qs, st, p, 1, 1, torch, stream)
        held[name] = {"predicted_ms": round(pr + init_norm, 3), "measured_ms": round(ms, 3),
                      "rel_err": round((pr + init_norm - ms) / ms, 4)}
    n2 = args.n - 2
    st2 = qs.State(n2, args.dtype, arith=args.arith, stream=stream)
    p, pr = predicted(n2, wc.rzrx_cz_circuit(n2, args.layers, seed=args.seed), mode="tile")
    ms, _, _ = measure(qs, st2, p, 1, 1, torch, stream)
    st2.close()
    init_norm2 = init_norm / 4.0   # the state is a quarter of the size
    held[f"rzrx_{n2}q_tile"] = {"predicted_ms": round(pr + init_norm2, 3), "measured_ms": round(ms, 3),
                                "rel_err": round((pr + init_norm2 - ms) / ms, 4)}
    return {"coef_ms_per_launch_byte_instr": {k: [float(f"{x:.4g}") for x in v] for k, v in coef.items()},
            "train": train, "held_out": held,
            "held_out_max_abs_rel_err": max(abs(v["rel_err"]) for v in held.values())}


runs_circuits = {}
runs_opts = {}


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    import paper_2010_09746_gb300 as qs

    qs.use_torch_allocator(local)
    n, circ, name = workload(args)
    G = len(circ)
    # the timed steps cycle over the circuits of seeds seed .. seed + seeds - 1 (same
    # construction, same gate count); everything else uses the first
    circs = [circ] + [workload(argparse.Namespace(**dict(vars(args), seed=args.seed + k)))[1]
                      for k in range(1, max(1, args.seeds))]
    assert all(len(c) == G for c in circs)
    stream = torch.cuda.Stream(device=local)
    policy = {"c64": "f32", "c128": ("f64" if args.arith == "f64" else "df")}[args.dtype]
    st = qs.State(n, args.dtype, arith=args.arith, stream=stream)
    plans = [qs.compile(n, c, mode=args.mode, dtype=args.dtype, arith=args.arith, tile_bits=args.tile_bits,
                        low_bits=args.low_bits, reg_bits=args.reg_bits) for c in circs]
    plan = plans[0]
    pstats = plan.stats()

    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms, norms, kstats = measure(qs, st, plans, args.steps, args.warmup, torch, stream, profile=True)
    clk = clocks.stop()
    ms = reduce_max(ms, pg)
    value = job_rate(G, world, ms)

    peaks, peaks_kind = load_peaks()
    dev = device_info(local, clk)
    roof = roofline(kstats, args.steps, ms, peaks, peaks_kind, policy, dev,
                    method_flops(circ, n) if args.workload == "rzrx30" else None)
    if roof:
        roof["traffic"] = profiled_traffic(roof["kernel"], n)
    launches = int(round(sum(k["launches"] for k in kstats)))
    total_bytes = pstats["hbm_bytes"] + (1 << n) * (16 if args.dtype == "c128" else 8) * 2  # + init, norm
    out = {
        "metric": "30q random-circuit gates/s & % HBM roofline",
        "value": round(value, 2), "unit": "gates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"df": "f32x2", "f32": "f32", "f64": "f64"}[policy], "data": "synthetic (seeded random circuit)",
        "config": {"workload": name, "seeds": list(range(args.seed, args.seed + len(circs))),
                   "passes_per_seed": [p.stats()["n_passes"] for p in plans],
                   "n_qubits": n, "gates": G, "mode": args.mode, "state_dtype": args.dtype,
                   "arith": {"df": "double-float (pairs of f32) on packed f32x2 lanes, f64 storage", "f32": "f32", "f64": "f64"}[policy],
                   "tile_bits": args.tile_bits or None, "low_bits": args.low_bits or None,
                   "reg_bits": args.reg_bits or None,
                   "passes": pstats["n_passes"], "fused_gates": pstats["n_fused"],
                   "fusion": "runs of single-qubit gates on one qubit applied as diag.RX.diag" if pstats["n_fused"] else None,
                   "permutes": pstats["n_permutes"],
                   "permute_kernels": pstats["n_permute_kernels"], "pergate": pstats["n_pergate"],
                   "parallelism": f"replicas{world}",
                   "l2": "state 16 GiB >> 129 MB L2, no flush needed" if n >= 27 else "state small vs L2"},
        "hbm_frac_step": round(total_bytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
        "per_gate_hbm_bound": per_gate_bound(qs, n, circ, args, peaks, value / world),
        "norm_max_dev": max(abs(x - 1.0) for x in norms),
        "compile_ms": round(pstats["compile_ms"], 2),
        "roofline": roof, "gpu_launches": launches, "kernels": kstats, "clocks": clk,
    }

    def section(key, fn):
        """A side measurement: its failure is recorded in the line instead of losing it."""
        try:
            out[key] = fn()
        except Exception as e:  # noqa: BLE001
            import traceback
            traceback.print_exc()
            out[key] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.synchronize()

    # ---- e2e: host circuit -> compile -> execute -> read back, every step
    if not args.no_e2e:
        ops, nops, mats = qs.marshal(circ)
        h2d = nops * 48 + mats.nbytes
        readout = 1 << min(n, 16)
        d2h = readout * (16 if args.dtype == "c128" else 8) + 8
        torch.cuda.synchronize()
        e2e_steps = max(1, args.steps if args.e2e_steps <= 0 else min(args.steps, args.e2e_steps))
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            st.reset()
            st.run(circs[k % len(circs)], mode=args.mode, tile_bits=args.tile_bits, low_bits=args.low_bits,
                   reg_bits=args.reg_bits)
            st.amplitudes(0, readout)
            st.norm()
        torch.cuda.synchronize()
        t_e2e = reduce_max((time.perf_counter() - t0) / e2e_steps * 1e3, pg)
        out["e2e"] = {"value": round(job_rate(G, world, t_e2e), 2), "unit": "gates/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "ms_per_step": round(t_e2e, 3), "steps": e2e_steps,
                      "what": "per step, host wall clock: the circuit's ops and matrices from host memory through "
                              "qs_run (compile + execute), then the first %d amplitudes and the FP64 norm copied back "
                              "to the host (not the whole %d-byte state)" % (readout, (1 << n) * (16 if args.dtype == "c128" else 8))}

    # ---- the same circuit without the reordering pass, and with the paper's Algorithm 1
    if args.modes and args.mode == "tile":
        modes = {"tile": {"gates_per_s": out["value"] / world, "passes": pstats["n_passes"]}}
        per_layer = 2 * n + n // 4 if args.workload == "rzrx30" else len(circ) // 20
        sub = circ[: 4 * per_layer]   # first 4 layers
        p_pg = qs.compile(n, sub, mode="pergate", dtype=args.dtype, arith=args.arith)
        ms_pg, _, ks_pg = measure(qs, st, p_pg, 1, 1, torch, stream, profile=True)
        modes["pergate"] = {"gates_per_s": round(len(sub) / (ms_pg / 1e3), 2), "sample": f"first {len(sub)} gates",
                            "kernels": p_pg.stats()["n_pergate"]}
        p_uf = qs.compile(n, circ, mode="tile", dtype=args.dtype, arith=args.arith, tile_bits=args.tile_bits,
                          low_bits=args.low_bits, reg_bits=args.reg_bits, fuse=False)
        ms_uf, _, _ = measure(qs, st, p_uf, 1, 1, torch, stream, profile=False)
        modes["tile_unfused"] = {"gates_per_s": round(G / (ms_uf / 1e3), 2), "passes": p_uf.stats()["n_passes"],
                                 "alu_instr_per_amp": round(p_uf.stats()["alu_instr"] / (1 << n), 1),
                                 "fused_alu_instr_per_amp": round(pstats["alu_instr"] / (1 << n), 1)}
        p_pa = qs.compile(n, circ, mode="paper", dtype=args.dtype, arith=args.arith, tile_bits=12)
        ms_pa, _, ks_pa = measure(qs, st, p_pa, 1, 1, torch, stream, profile=True)
        s_pa = p_pa.stats()
        modes["paper_alg1_m12"] = {"gates_per_s": round(G / (ms_pa / 1e3), 2), "passes": s_pa["n_passes"],
                                   "permutes": s_pa["n_permutes"], "permute_kernels": s_pa["n_permute_kernels"],
                                   "nonlocal_gates": s_pa["n_comm_gates"]}
        out["modes"] = modes
        runs_circuits.update({"tile": circ, "pergate": sub, "paper_alg1_m12": circ})
        runs_opts.update({"tile": dict(mode=args.mode, tile_bits=args.tile_bits, low_bits=args.low_bits,
                                       reg_bits=args.reg_bits),
                          "pergate": {"mode": "pergate"}, "paper_alg1_m12": {"mode": "paper", "tile_bits": 12}})
        if args.workload == "rzrx30":
            section("cost_model", lambda: fit_cost_model(qs, torch, st, stream, args, {
                "tile": (plan, ms, kstats, args.steps), "pergate": (p_pg, ms_pg, ks_pg, 1),
                "paper_alg1_m12": (p_pa, ms_pa, ks_pa, 1)}))
    if args.modes and args.workload == "rzrx30":
        section("permute", lambda: measure_permute(qs, torch, st, stream, n, (1 << n) * (16 if args.dtype == "c128" else 8)))
    if args.small and args.workload == "rzrx30":
        section("haar_cnot_12q", lambda: measure_small(qs, torch, args))
    if args.qft and args.workload == "rzrx30":
        section("qft_like", lambda: measure_qft_like(qs, torch, st, stream, args))
    if args.batched:
        section("batched", lambda: measure_batched(qs, torch, args))
    if args.dense and args.workload == "rzrx30":
        section("dense_k", lambda: measure_dense(qs, torch, args))
    if args.precision and args.workload == "rzrx30":
        st.close()
        torch.cuda.empty_cache()
        section("precision", lambda: measure_precision(qs, torch, args))
    if args.serve_requests:
        section("serving", lambda: measure_serving(args))
    if args.cpu_baseline and rank == 0 and world == 1:
        section("cpu_baseline", lambda: cpu_baseline(args, n, circ))
    if pg:
        pg.destroy_process_group()
    return out, rank


def measure_small(qs, torch, args):
    """12 qubits (64 KiB state, cache-resident: launch-bound), 20 layers of Haar 2x2 on every
    qubit + CNOT on a random perfect matching, seeds 0..19; gates/s per mode, with the
    step's launches replayed from a captured CUDA graph and without."""
    n, dt = 12, args.dtype
    circs = [wc.haar_cnot_circuit(n, 20, seed=s) for s in range(20)]
    G = sum(len(c) for c in circs)
    stream = torch.cuda.Stream()
    res = {"circuits": len(circs), "gates": G}
    for mode in ("tile", "paper", "pergate"):
        kw = {"tile_bits": 8} if mode == "paper" else {}
        plans = [qs.compile(n, c, mode=mode, dtype=dt, arith=args.arith, **kw) for c in circs]
        st = qs.State(n, dt, arith=args.arith, stream=stream)

        def run_all():
            for p in plans:
                st.reset()
                st.execute(p)

        run_all()   # uploads the plans
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            run_all()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        entry = {"gates_per_s": round(G / (ms / 1e3), 1), "launches_per_circuit": plans[0].stats()["n_passes"]
                 + plans[0].stats()["n_pergate"] + plans[0].stats()["n_permute_kernels"] + 1}
        if mode != "paper":   # permutations swap buffers on the host: not replayable as one graph
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
                run_all()
            with torch.cuda.stream(stream):   # replay launches on the current stream
                g.replay()
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(reps):
                    g.replay()
                e1.record(stream)
            torch.cuda.synchronize()
            msg = e0.elapsed_time(e1) / reps
            entry["graph_gates_per_s"] = round(G / (msg / 1e3), 1)
        res[mode] = entry
        st.close()
    return res


def measure_permute(qs, torch, st, stream, n, S):
    """PermuteQubits (K3) on the benchmark's own state: one local<->global transposition
    (qubits 0 and n-1) and a random permutation of all n qubits (seed 0); CUDA events, best
    of 3 after a warm-up; algorithmic bytes 2*S per permutation."""
    peaks, _ = load_peaks()
    rng = np.random.default_rng(0)
    res = {}
    cases = {"swap_0_top": [n - 1] + list(range(1, n - 1)) + [0], "random_all": [int(x) for x in rng.permutation(n)]}
    for name, perm in cases.items():
        ident = list(range(n))
        st.permute(ident)
        st.permute(perm)
        st.permute(ident)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st.permute(perm)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
            st.permute(ident)
        gbs = 2 * S / (best * 1e-3) / 1e9
        res[name] = {"ms": round(best, 3), "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / peaks["hbm_gbs"], 4)}
    return res


def measure_dense(qs, torch, args):
    """Dense k-qubit blocks (Haar 2^k x 2^k, seed k) on a 30-qubit complex64 state: the
    CUDA-core kernel against the tensor-core kernel, qubits on storage bits 0..k-1, and at
    k = 6 also on high qubits (the tensor path then permutes first).  Per application: CUDA
    events on the state's stream, best of 3 after a warm-up; HBM fraction of the measured
    copy bandwidth; tensor TF32 FLOP/s (three split products) against the measured bf16
    peak x 1.1/2.25 (the nominal tf32 : bf16 ratio)."""
    n = 30
    peaks, _ = load_peaks()
    tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25
    stream = torch.cuda.Stream()
    st = qs.State(n, "c64", stream=stream)
    S = (1 << n) * 8
    res = {"n_qubits": n, "state": "complex64", "tf32_peak_tflops": round(tf32_peak, 1)}

    def timed_apply(U, qubits, reps=3):
        st.apply_dense(U, qubits)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st.apply_dense(U, qubits)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    for k in (4, 5, 6):
        U = wc.haar_unitary(1 << k, np.random.default_rng(k))
        row = {}
        for path in ("cuda_cores", "tensor"):
            st.reset()
            st.set_dense_path(path)
            ms = timed_apply(U, list(range(k)))
            gbs = 2 * S / (ms * 1e-3) / 1e9
            row[path] = {"ms": round(ms, 3), "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / peaks["hbm_gbs"], 4)}
            if path == "tensor":
                tf = 3 * 2 * 128 * 128 * (1 << (n - 6)) / (ms * 1e-3) / 1e12
                row[path]["tf32_tflops"] = round(tf, 1)
                row[path]["tensor_frac"] = round(tf / tf32_peak, 4)
        row["tensor_speedup"] = round(row["cuda_cores"]["ms"] / row["tensor"]["ms"], 2)
        res[f"k{k}_low"] = row
    U = wc.haar_unitary(64, np.random.default_rng(6))
    high = [24, 25, 26, 27, 28, 29]
    row = {}
    for path in ("cuda_cores", "tensor"):
        st.reset()
        st.set_dense_path(path)
        # the tensor path permutes these qubits to the bottom on the first call only, so time
        # alternating qubit sets to include a permutation in every application
        alt = [high, [18, 19, 20, 21, 22, 23]]
        st.apply_dense(U, alt[0])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(4):
            st.apply_dense(U, alt[(i + 1) % 2])
        e1.record(stream)
        torch.cuda.synchronize()
        row[path] = {"ms": round(e0.elapsed_time(e1) / 4, 3)}
    row["tensor_speedup"] = round(row["cuda_cores"]["ms"] / row["tensor"]["ms"], 2)
    res["k6_high_with_permute"] = row
    # the compiler's own choice: the 30-qubit circuit as complex64, with the dense blocks the
    # default cost model picks (gates ready on storage bits 0..5 fused into one tensor-core
    # launch when that is predicted cheaper than their tile-pass arithmetic) and without
    circ = wc.rzrx_cz_circuit(n, 40, seed=0)
    plans = {}
    for key, dense in (("with_dense_blocks", True), ("tile_passes_only", False)):
        p = qs.compile(n, circ, mode="tile", dtype="c64", dense=dense)
        ms, _, ks = measure(qs, st, p, 3, 2, torch, stream, profile=True)
        s_ = p.stats()
        plans[key] = {"gates_per_s": round(len(circ) / (ms / 1e3), 1), "ms": round(ms, 2),
                      "passes": s_["n_passes"], "dense_blocks": s_["n_dense"],
                      "predicted_ms": round(s_["predicted_ms"], 2),
                      "dense_ms_per_launch": next((round(k["total_ms"] / k["launches"], 3) for k in ks
                                                   if k["name"] == "dense_mma_c64"), None)}
    plans["speedup"] = round(plans["tile_passes_only"]["ms"] / plans["with_dense_blocks"]["ms"], 3)
    res["rzrx_30q_c64_compiled"] = plans
    st.close()
    torch.cuda.empty_cache()
    return res


def measure_precision(qs, torch, args):
    """The precision study: 32 qubits, the same construction at depth 30 (2160 gates), run
    as complex128 (double-float arithmetic, 64 GiB) and as complex64 (32 GiB, with and without
    renormalisation after every 4 passes); the full-state fidelity 1 - |<psi64|psi128>|^2 /
    (norms) and both norms, every reduction in FP64 on the device; then 33 qubits complex64
    (64 GiB), norm only."""
    stream = torch.cuda.Stream()
    n = 32
    circ = wc.rzrx_cz_circuit(n, 30, seed=0)
    res = {"circuit": f"rzrx_cz_{n}q_30layers", "gates": len(circ)}

    def timed_run(st, plan):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        st.reset()
        e0.record(stream)
        st.execute(plan)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    s128 = qs.State(n, "c128", stream=stream)
    ms128 = timed_run(s128, qs.compile(n, circ, mode="tile", dtype="c128"))
    res["c128"] = {"ms": round(ms128, 1), "gates_per_s": round(len(circ) / ms128 * 1e3, 1),
                   "norm_dev": abs(s128.norm() - 1.0)}
    s64 = qs.State(n, "c64", stream=stream)
    for R in (0, 4):
        ms64 = timed_run(s64, qs.compile(n, circ, mode="tile", dtype="c64", renorm_every=R))
        key = "c64" if R == 0 else f"c64_renorm_every_{R}"
        res[key] = {"ms": round(ms64, 1), "gates_per_s": round(len(circ) / ms64 * 1e3, 1),
                    "norm_dev": abs(s64.norm() - 1.0), "fidelity_loss_vs_c128": 1.0 - s64.fidelity(s128)}
    s64.close()
    s128.close()
    torch.cuda.empty_cache()
    n = 33
    circ = wc.rzrx_cz_circuit(n, 30, seed=0)
    s = qs.State(n, "c64", stream=stream)
    ms = timed_run(s, qs.compile(n, circ, mode="tile", dtype="c64"))
    res["c64_33q"] = {"gates": len(circ), "ms": round(ms, 1), "gates_per_s": round(len(circ) / ms * 1e3, 1),
                      "norm_dev": abs(s.norm() - 1.0)}
    s.close()
    torch.cuda.empty_cache()
    return res


def measure_qft_like(qs, torch, st, stream, args):
    """Appendix C's QFT-like circuit (controlled-Rz replaced by CNOT) on the same state:
    the tile passes vs Algorithm 1 at m = 12 (whose permutation count the appendix bounds
    by 2(n - m)) vs one kernel per gate."""
    n = args.n
    circ = wc.qft_like_circuit(n)
    res = {"gates": len(circ)}
    for mode, kw in (("tile", {}), ("paper_alg1_m12", {"mode": "paper", "tile_bits": 12}), ("pergate", {"mode": "pergate"})):
        opts = dict(mode="tile", dtype=args.dtype, arith=args.arith)
        opts.update(kw)
        plan = qs.compile(n, circ, **opts)
        ms, _, _ = measure(qs, st, plan, 1, 1, torch, stream)
        ps = plan.stats()
        res[mode] = {"gates_per_s": round(len(circ) / (ms / 1e3), 2), "ms": round(ms, 2), "passes": ps["n_passes"],
                     "permutes": ps["n_permutes"], "permute_kernels": ps["n_permute_kernels"],
                     "pergate_kernels": ps["n_pergate"]}
    res["paper_alg1_m12"]["permute_bound_2(n-m)"] = 2 * (n - 12)
    return res


def measure_batched(qs, torch, args):
    """The batched workload: `--batched` circuits (n ~ U{10..20}, depth ~ U{10..60}, Haar 2x2 on
    every qubit + CNOT/CZ on a random matching per layer, seed 0), complex64, one persistent
    launch per wave of tile passes replayed from a CUDA graph, at the tile width (fusion
    width) the autotuner picks by timing each candidate.  Beside it: the first 256 circuits
    run one plan launch sequence per circuit (qs_execute on separate states)."""
    from paper_2010_09746_gb300 import tuning
    work = wc.batched_workload(args.batched, seed=0)
    tune = tuning.autotune_batch(work, dtype="c64", tile_bits=tuple(args.batch_tile_bits), reps=2)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    arrays = qs.Batch.marshal(work)   # Python gate objects -> the C arrays (a C caller starts here)
    marshal_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = qs.Batch(dtype="c64", stream=stream, tile_bits=tune["tile_bits"], marshalled=arrays)
    build_s = time.perf_counter() - t0
    for _ in range(3):
        b.run()
    b.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        b.run()
    e1.record(stream)
    b.sync()
    ms = e0.elapsed_time(e1) / reps
    st = b.stats()
    norms = b.norms()
    gates = st["n_gates"]
    res = {"circuits": len(work), "gates": gates, "ms_per_run": round(ms, 3),
           "circuits_per_s": round(len(work) / (ms / 1e3), 1), "gates_per_s": round(gates / (ms / 1e3), 1),
           "waves": st["n_waves"], "passes": st["n_passes"], "state_gib": round(st["state_bytes"] / 2 ** 30, 2),
           "marshal_s": round(marshal_s, 3),
           "build_s": round(build_s, 3),
           "build_what": "qs_batch_create: every circuit compiled on the host cores (threads), concatenated "
                         "and uploaded",
           "circuits_per_s_with_build": round(len(work) / (build_s + ms / 1e3), 1),
           "norm_max_dev": float(np.max(np.abs(norms - 1.0))),
           "autotuned_tile_bits": tune["tile_bits"],
           "autotune": [{k: (round(v, 3) if isinstance(v, float) else v) for k, v in c.items()}
                        for c in tune["candidates"]]}
    # one launch sequence per circuit, on the first 256 circuits
    sub = work[:256]
    states = [qs.State(n, "c64", stream=stream) for n, _ in sub]
    plans = [qs.compile(n, c, mode="tile", dtype="c64") for n, c in sub]
    for s_, p_ in zip(states, plans):
        s_.reset()
        s_.execute(p_)
    torch.cuda.synchronize()
    e0.record(stream)
    for s_, p_ in zip(states, plans):
        s_.reset()
        s_.execute(p_)
    e1.record(stream)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    sub_gates = sum(len(c) for _, c in sub)
    res["solo_first256"] = {"circuits_per_s": round(len(sub) / (ms1 / 1e3), 1),
                            "gates_per_s": round(sub_gates / (ms1 / 1e3), 1), "ms": round(ms1, 3)}
    return res


def measure_serving(args):
    """The serving workload through the library's native server (qs_server_*): random circuits
    (n = floor(exp(U(ln 12, ln 29))), depth U{20..100}, Haar 2x2 + CNOT/CZ layers, complex64 or
    complex128 with probability 1/2), Poisson arrivals.  First all requests at once (the
    saturation throughput), then Poisson arrivals at fixed fractions of that throughput;
    latency = arrival -> result (FP64 norm and first amplitudes) in host memory."""
    import paper_2010_09746_gb300 as qs
    from paper_2010_09746_gb300 import serve
    budget = int(args.serve_mem_gib * (1 << 30))

    def one(reqs, realtime, order):
        srv = serve.Server(slots=args.serve_slots, mem_budget=budget, order=order)
        t0 = time.perf_counter()
        res = srv.run(reqs, realtime=realtime)
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return dict(serve.latency_summary(res, wall), peak_in_flight=st["peak_in_flight"],
                    batched_requests=st["batched_requests"], batches=st["batches"],
                    peak_mem_gib=round(st["peak_mem_bytes"] / 2 ** 30, 2)), wall

    reqs = wc.serving_workload(args.serve_requests, rate_hz=1.0, seed=0)
    # the device work in the mix, as the compiler's cost model predicts each request alone
    work_s = sum(qs.compile(r.n, r.circuit, mode="tile", dtype=r.dtype).stats()["predicted_ms"] for r in reqs) / 1e3
    sat_entry, wall = one(reqs, False, args.serve_order)
    sat = len(reqs) / wall
    sat_entry["predicted_device_s"] = round(work_s, 3)
    sat_entry["predicted_device_s_over_wall"] = round(work_s / wall, 3)
    out = {"requests_per_load": len(reqs), "slots": args.serve_slots, "mem_budget_gib": args.serve_mem_gib,
           "order": args.serve_order, "server": "native (qs_server_*: compile threads + admission thread)",
           "saturation": sat_entry}
    for frac in args.serve_loads:
        rate = frac * sat
        reqs = wc.serving_workload(args.serve_requests, rate_hz=rate, seed=0)   # same circuits, Poisson times
        entry, _ = one(reqs, True, args.serve_order)
        out[f"load_{frac:g}"] = dict(entry, offered_rate_hz=round(rate, 3))
    # the other admission order at 0.9 of saturation, same requests
    other = "sjf" if args.serve_order == "fifo" else "fifo"
    alt = {}
    alt["load_0.9"], _ = one(wc.serving_workload(args.serve_requests, rate_hz=0.9 * sat, seed=0), True, other)
    out[f"order_{other}"] = alt
    return out


def cpu_baseline(args, n, circ, budget_s=None):
    """The FP64 oracle, as it stands, on this host's cores: a bounded sample of the same
    workload (the first gates of the same circuit on an n-qubit state)."""
    from oracle import sv
    budget_s = budget_s or args.cpu_budget_s
    st = sv.OracleState(n)
    t0 = time.perf_counter()
    k = 0
    while k < len(circ) and time.perf_counter() - t0 < budget_s:
        st.apply_gate(circ[k])
        k += 1
    dt = time.perf_counter() - t0
    return {"value": round(k / dt, 4), "unit": "gates/s", "cores": sv.num_threads(), "kind": "oracle",
            "sample": f"first {k} of {len(circ)} gates of the same circuit on the {n}-qubit FP64 state "
                      f"(init excluded), {dt:.1f} s"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None, rank
    n, circ, name = workload(args)
    from oracle import sv
    sv.lib()
    per_step = max(1.0, args.cpu_budget_s / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(args, n, circ, budget_s=per_step)
    runs = [cpu_baseline(args, n, circ, budget_s=per_step) for _ in range(args.steps)]
    v = statistics.median(r["value"] for r in runs)
    out = {
        "impl": "reference", "metric": "30q random-circuit gates/s & % HBM roofline", "value": v,
        "unit": "gates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 / v, 3) if v else None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random circuit)",
        "config": {"workload": name, "n_qubits": n, "gates": len(circ), "mode": "oracle (per gate, FP64, CPU)",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": v, "unit": "gates/s", "cores": sv.num_threads(), "kind": "oracle",
                         "sample": runs[0]["sample"]},
        "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return out, rank


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rzrx30", choices=["rzrx30", "haar12"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--layers", type=int, default=40)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--seeds", type=int, default=5, help="timed steps cycle over this many circuit seeds")
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--arith", default="auto", choices=["auto", "df", "f64"])
    ap.add_argument("--mode", default="tile", choices=["tile", "paper", "pergate"])
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--low-bits", type=int, default=0)
    ap.add_argument("--reg-bits", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0, help="end-to-end steps (0 = the same as --steps)")
    ap.add_argument("--modes", type=int, default=1, help="also time per-gate and Algorithm 1 modes")
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--qft", type=int, default=1, help="also time Appendix C's QFT-like circuit")
    ap.add_argument("--dense", type=int, default=1,
                    help="also time dense k-qubit blocks on CUDA cores vs tensor cores (30q complex64)")
    ap.add_argument("--precision", type=int, default=1,
                    help="also run the 32q complex128/complex64 and 33q complex64 precision study")
    ap.add_argument("--small", type=int, default=1, help="also time the 12-qubit Haar + CNOT circuits")
    ap.add_argument("--batched", type=int, default=4096, help="circuits in the batched measurement (0 = skip)")
    ap.add_argument("--batch-tile-bits", type=int, nargs="+", default=[10, 12, 13],
                    help="tile widths the batched measurement's autotuner times")
    ap.add_argument("--serve-requests", type=int, default=500, help="requests per serving load point (0 = skip)")
    ap.add_argument("--serve-order", default="fifo", choices=["fifo", "sjf"],
                    help="admission order: first come, or least estimated work first (1 s maximum wait)")
    ap.add_argument("--serve-loads", type=float, nargs="*", default=[0.5, 0.9, 1.1],
                    help="Poisson arrival rates as fractions of the measured saturation throughput")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-mem-gib", type=float, default=96.0)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    args = ap.parse_args(argv)
    if args.impl == "reference":
        out, rank = run_reference(args)
    else:
        out, rank = run_ours(args)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()

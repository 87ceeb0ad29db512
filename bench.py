#!/usr/bin/env python3
"""Benchmark: 30-qubit random-circuit simulation on one GB300 (replicas on N GPUs).

Workload (default): 30 qubits, complex128 (16 GiB state), 40 layers of RZ(U(0,2pi)) and
RX(U(0,2pi)) on every qubit followed by floor(n/4) CZ on pairs biased toward high qubits
(seed 0; 2680 gates).  One step = state preparation |0..0> + the compiled circuit (tile
passes, and permutations / per-gate kernels where the mode uses them) + the FP64 norm
read-out.  The plan is compiled before the timed region; `e2e` re-compiles from host
buffers every step and copies inputs / results over PCIe/C2C inside its timed region.

`value` = circuit gates / device-timed step time (CUDA events on the library's stream),
whole job.  The state (16 GiB) is far larger than L2 (129 MB), so no flush is needed.

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


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def workload(args):
    if args.workload == "rzrx30":
        n, layers = args.n, args.layers
        circ = wc.rzrx_cz_circuit(n, layers, seed=args.seed)
        name = f"rzrx_cz_{n}q_{layers}layers_{args.dtype}"
    elif args.workload == "haar12":
        n = 12
        circ = wc.haar_cnot_circuit(12, 20, seed=args.seed)
        name = f"haar_cnot_12q_20layers_{args.dtype}"
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    return n, circ, name


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
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args)
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
    stream = torch.cuda.Stream(device=local)
    st = qs.State(n, args.dtype, arith=args.arith, stream=stream)
    plan = qs.compile(n, circ, mode=args.mode, dtype=args.dtype, arith=args.arith, tile_bits=args.tile_bits,
                      low_bits=args.low_bits)
    pstats = plan.stats()

    def step():
        st.reset()
        st.execute(plan)
        return st.norm()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    st.set_profiling(True)
    st.reset_kernel_stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    norms = []
    for _ in range(args.steps):
        norms.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    kstats = st.kernel_stats()
    st.set_profiling(False)
    clk = clocks.stop()
    if pg:
        t = torch.tensor([ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    value = world * G / (ms / 1e3)

    # ---- e2e: host circuit -> compile -> execute -> read back, every step
    e2e = None
    if not args.no_e2e:
        ops, nops, mats = qs.marshal(circ)
        h2d = nops * 48 + mats.nbytes
        readout = 1 << min(n, 16)
        d2h = readout * (16 if args.dtype == "c128" else 8) + 8
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            st.reset()
            st.run(circ, mode=args.mode, tile_bits=args.tile_bits, low_bits=args.low_bits)
            st.amplitudes(0, readout)
            st.norm()
        torch.cuda.synchronize()
        t_e2e = (time.perf_counter() - t0) / e2e_steps
        if pg:
            t = torch.tensor([t_e2e], device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            t_e2e = float(t.item())
        e2e = {"value": world * G / t_e2e, "unit": "gates/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": t_e2e * 1e3}

    # ---- roofline of the dominant kernel (per-launch CUDA events on the library stream)
    peaks, peaks_kind = load_peaks()
    dom = max(kstats, key=lambda k: k["total_ms"]) if kstats else None
    roof = None
    if dom:
        per_launch_ms = dom["total_ms"] / dom["launches"]
        bytes_per_launch = dom["bytes"] / dom["launches"]
        achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"kernel": dom["name"], "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": f"{peaks_kind} hbm_gbs",
                "launches_per_step": dom["launches"] / args.steps,
                "ms_per_launch": round(per_launch_ms, 4),
                "share_of_step": round(dom["total_ms"] / args.steps / ms, 4)}
    launches = int(sum(k["launches"] for k in kstats) / args.steps * args.steps)
    total_bytes = pstats["hbm_bytes"] + (1 << n) * (16 if args.dtype == "c128" else 8) * 2  # + init write + norm read
    hbm_frac_step = total_bytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]

    norm_err = max(abs(x - 1.0) for x in norms)
    out = {
        "metric": "30q random-circuit gates/s & % HBM roofline",
        "value": round(value, 2), "unit": "gates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"c128": ("df" if args.arith in ("auto", "df") else "f64"), "c64": "f32"}[args.dtype],
        "data": "synthetic (seeded random circuit)",
        "config": {"workload": name, "n_qubits": n, "gates": G, "mode": args.mode, "state_dtype": args.dtype,
                   "tile_bits": args.tile_bits or None, "low_bits": args.low_bits or None,
                   "passes": pstats["n_passes"], "permutes": pstats["n_permutes"], "pergate": pstats["n_pergate"],
                   "parallelism": f"replicas{world}", "l2": "state 16 GiB >> 129 MB L2, no flush needed"
                   if n >= 27 else "state fits in L2 (launch-bound workload)"},
        "hbm_frac_step": round(hbm_frac_step, 4),
        "norm_max_dev": norm_err,
        "compile_ms": round(pstats["compile_ms"], 2),
        "roofline": roof, "e2e": e2e, "gpu_launches": launches, "kernels": kstats,
        "clocks": clk,
    }
    if args.cpu_baseline and rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline(args, n, circ)
    if pg:
        pg.destroy_process_group()
    return out, rank


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
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return None, rank
    n, circ, name = workload(args)
    from oracle import sv
    sv.lib()
    # each step: a bounded sample of the workload
    per_step = max(1.0, args.cpu_budget_s / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(args, n, circ, budget_s=per_step)
    vals = []
    samples = []
    for _ in range(args.steps):
        r = cpu_baseline(args, n, circ, budget_s=per_step)
        vals.append(r["value"])
        samples.append(r["sample"])
    v = statistics.median(vals)
    out = {
        "impl": "reference", "metric": "30q random-circuit gates/s & % HBM roofline", "value": v,
        "unit": "gates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 / v, 3) if v else None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random circuit)",
        "config": {"workload": name, "n_qubits": n, "gates": len(circ), "mode": "oracle (per gate, FP64, CPU)",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": v, "unit": "gates/s", "cores": sv.num_threads(), "kind": "oracle",
                         "sample": samples[0]},
        "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return out, rank


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rzrx30", choices=["rzrx30", "haar12"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--layers", type=int, default=40)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--arith", default="auto", choices=["auto", "df", "f64"])
    ap.add_argument("--mode", default="tile", choices=["tile", "paper", "pergate"])
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--low-bits", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--extra", default="", help="comma list of extra measurements: pergate,paper,c64")
    args = ap.parse_args()
    if args.impl == "reference":
        out, rank = run_reference(args)
    else:
        out, rank = run_ours(args)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()

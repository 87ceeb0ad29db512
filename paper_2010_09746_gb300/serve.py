"""Continuous-batching request loop over the C ABI.

Requests (a circuit, its qubit count and dtype) arrive over time.  The server admits a
waiting request as soon as a slot and enough device memory are free -- it does not wait
for the requests already on the GPU -- compiles its plan on the host, and enqueues
state preparation and the plan on the slot's own CUDA stream, so
work of different requests overlaps on the device.  Completion is detected with CUDA
events; the result (the FP64 norm and the first amplitudes) is read out, the state is
released and the next request takes the slot.  Every request runs the same kernels on its
own state whatever else is in flight, so its result does not depend on the mix.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import Plan, State


@dataclass
class Result:
    rid: int
    n: int
    dtype: str
    norm: float
    amplitudes: np.ndarray
    arrival_s: float
    admit_s: float
    done_s: float

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclass
class _Slot:
    stream: object
    busy: bool = False


@dataclass
class _Flight:
    rid: int
    req: object
    slot: int
    state: State
    plan: Plan
    event: object
    arrival_s: float
    admit_s: float
    bytes: int


class Server:
    """slots: requests in flight at once; mem_budget: device bytes for resident states;
    readout: amplitudes copied back per request (first min(2^n, readout))."""

    def __init__(self, slots: int = 8, mem_budget: int = 64 << 30, readout: int = 256, tile_bits: int = 0):
        import torch

        self.torch = torch
        self.slots = [_Slot(torch.cuda.Stream()) for _ in range(slots)]
        self.mem_budget = int(mem_budget)
        self.mem_used = 0
        self.readout = readout
        self.tile_bits = tile_bits
        self.waiting: deque = deque()
        self.flights: List[_Flight] = []
        self.results: Dict[int, Result] = {}
        self.peak_in_flight = 0
        self.peak_mem = 0

    @staticmethod
    def state_bytes(n: int, dtype: str) -> int:
        return (1 << n) * (16 if dtype == "c128" else 8)

    def submit(self, rid: int, req, arrival_s: float):
        if self.state_bytes(req.n, req.dtype) > self.mem_budget:
            raise ValueError(f"request {rid} needs more device memory than the whole budget")
        self.waiting.append((rid, req, arrival_s))

    def _admit(self, now_s: float) -> int:
        admitted = 0
        while self.waiting:
            rid, req, arr = self.waiting[0]
            need = self.state_bytes(req.n, req.dtype)
            free = [i for i, s in enumerate(self.slots) if not s.busy]
            if not free or self.mem_used + need > self.mem_budget:
                break
            self.waiting.popleft()
            si = free[0]
            slot = self.slots[si]
            slot.busy = True
            self.mem_used += need
            plan = Plan(req.n, req.circuit, mode="tile", dtype=req.dtype, tile_bits=self.tile_bits)
            st = State(req.n, req.dtype, stream=slot.stream)
            st.execute(plan)
            ev = self.torch.cuda.Event()
            ev.record(slot.stream)
            self.flights.append(_Flight(rid, req, si, st, plan, ev, arr, now_s, need))
            admitted += 1
        self.peak_in_flight = max(self.peak_in_flight, len(self.flights))
        self.peak_mem = max(self.peak_mem, self.mem_used)
        return admitted

    def _poll(self, clock) -> int:
        done = 0
        keep = []
        for f in self.flights:
            if not f.event.query():
                keep.append(f)
                continue
            count = min(1 << f.req.n, self.readout)
            amps = f.state.amplitudes(0, count)
            norm = f.state.norm()
            t = clock()
            self.results[f.rid] = Result(f.rid, f.req.n, f.req.dtype, norm, amps, f.arrival_s, f.admit_s, t)
            f.state.close()
            self.slots[f.slot].busy = False
            self.mem_used -= f.bytes
            done += 1
        self.flights = keep
        return done

    def run(self, requests, realtime: bool = True, timeout_s: float = 600.0) -> Dict[int, Result]:
        """Serve `requests` (objects with arrival_s, n, dtype, circuit).  realtime: requests
        become visible at their arrival times on the wall clock; otherwise all at once."""
        reqs = sorted(enumerate(requests), key=lambda t: t[1].arrival_s)
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        nxt = 0
        while len(self.results) < len(reqs):
            now = clock()
            if now > timeout_s:
                raise TimeoutError("serving did not finish in time")
            while nxt < len(reqs) and (not realtime or reqs[nxt][1].arrival_s <= now):
                rid, r = reqs[nxt]
                self.submit(rid, r, r.arrival_s if realtime else 0.0)
                nxt += 1
            self._admit(clock())
            if self._poll(clock) == 0:
                time.sleep(0.0002)
        return self.results


def latency_summary(results: Dict[int, Result], wall_s: Optional[float] = None) -> dict:
    lat = np.array([r.latency_s for r in results.values()])
    out = {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50) * 1e3),
           "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}
    if wall_s:
        out["circuits_per_s"] = len(lat) / wall_s
    return out

"""Continuous-batching request loop over the C ABI.

Requests (a circuit, its qubit count and dtype) arrive over time.  The server admits a
waiting request as soon as a slot and enough device memory are free -- it does not wait
for the requests already on the GPU -- compiles its plan on the host, and enqueues
state preparation and the plan on the slot's own CUDA stream, so
work of different requests overlaps on the device.  Small requests (n <= batch_small_n)
waiting together with others of the same dtype share one slot: they are compiled into one
batch (qs_batch_*), whose tile passes run as persistent launches over all of their states.
Admission order is first-come or shortest-estimated-work first (with a maximum wait that
lets long-waiting requests go first).  Completion is detected with CUDA events; the result (the FP64 norm and the first
amplitudes) is read out, the state is released and the next request takes the slot.  Every
request runs the same per-tile code on its own state whatever else is in flight (a batched
circuit's amplitudes are bitwise those of its solo run), so its result does not depend on
the mix.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np

from . import Batch, Plan, State


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
    members: List[tuple]          # (rid, req, arrival_s) of every request in this flight
    slot: int
    state: Optional[State]        # one request
    plan: Optional[Plan]
    batch: Optional[Batch]        # several small requests
    event: object
    admit_s: float
    bytes: int


class Server:
    """slots: requests in flight at once; mem_budget: device bytes for resident states;
    readout: amplitudes copied back per request (first min(2^n, readout))."""

    def __init__(self, slots: int = 8, mem_budget: int = 64 << 30, readout: int = 256, tile_bits: int = 0,
                 batch_small_n: int = 16, batch_max: int = 64, order: str = "fifo", max_wait_s: float = 1.0):
        import torch

        self.torch = torch
        self.slots = [_Slot(torch.cuda.Stream()) for _ in range(slots)]
        self.mem_budget = int(mem_budget)
        self.mem_used = 0
        self.readout = readout
        self.tile_bits = tile_bits
        self.batch_small_n = batch_small_n
        self.batch_max = batch_max
        if order not in ("fifo", "sjf"):
            raise ValueError("order must be 'fifo' or 'sjf'")
        self.order = order            # sjf: least estimated work first, unless a request waited max_wait_s
        self.max_wait_s = max_wait_s
        self.batched_requests = 0
        self.batches = 0
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

    @staticmethod
    def work_estimate(req) -> float:
        """Relative device work: gates x amplitudes, complex128 (double-float) ~8x complex64."""
        return len(req.circuit) * float(1 << req.n) * (8.0 if req.dtype == "c128" else 1.0)

    def _next(self, now_s: float) -> int:
        """Index in `waiting` of the request to admit next."""
        if self.order == "fifo" or len(self.waiting) == 1:
            return 0
        if now_s - self.waiting[0][2] >= self.max_wait_s:   # the oldest has waited long enough
            return 0
        return min(range(len(self.waiting)), key=lambda k: self.work_estimate(self.waiting[k][1]))

    def _admit(self, now_s: float) -> int:
        admitted = 0
        while self.waiting:
            k = self._next(now_s)
            if k:
                self.waiting.rotate(-k)   # bring it to the front; the others keep their order after it
                item = self.waiting.popleft()
                self.waiting.rotate(k)
                self.waiting.appendleft(item)
            rid, req, arr = self.waiting[0]
            need = self.state_bytes(req.n, req.dtype)
            free = [i for i, s in enumerate(self.slots) if not s.busy]
            if not free or self.mem_used + need > self.mem_budget:
                break
            si = free[0]
            slot = self.slots[si]
            group = []
            if req.n <= self.batch_small_n and self.batch_max > 1:
                # the small requests of this dtype now waiting, in arrival order, that fit
                mem = 0
                for item in self.waiting:
                    r2 = item[1]
                    b2 = self.state_bytes(r2.n, r2.dtype)
                    if (r2.n <= self.batch_small_n and r2.dtype == req.dtype and len(group) < self.batch_max
                            and self.mem_used + mem + b2 <= self.mem_budget):
                        group.append(item)
                        mem += b2
            if len(group) > 1:
                ids = {id(item) for item in group}
                self.waiting = deque(item for item in self.waiting if id(item) not in ids)
                b = Batch([(r.n, r.circuit) for _, r, _ in group], dtype=req.dtype, stream=slot.stream, graph=False,
                          tile_bits=self.tile_bits)
                b.run()
                ev = self.torch.cuda.Event()
                ev.record(slot.stream)
                self.flights.append(_Flight(group, si, None, None, b, ev, now_s, mem))
                self.mem_used += mem
                self.batched_requests += len(group)
                self.batches += 1
                admitted += len(group)
            else:
                self.waiting.popleft()
                plan = Plan(req.n, req.circuit, mode="tile", dtype=req.dtype, tile_bits=self.tile_bits)
                st = State(req.n, req.dtype, stream=slot.stream)
                st.execute(plan)
                ev = self.torch.cuda.Event()
                ev.record(slot.stream)
                self.flights.append(_Flight([(rid, req, arr)], si, st, plan, None, ev, now_s, need))
                self.mem_used += need
                admitted += 1
            slot.busy = True
        self.peak_in_flight = max(self.peak_in_flight, sum(len(f.members) for f in self.flights))
        self.peak_mem = max(self.peak_mem, self.mem_used)
        return admitted

    def _poll(self, clock) -> int:
        done = 0
        keep = []
        for f in self.flights:
            if not f.event.query():
                keep.append(f)
                continue
            if f.batch is not None:
                norms = f.batch.norms()
                t = clock()
                for i, (rid, req, arr) in enumerate(f.members):
                    amps = f.batch.amplitudes(i, 0, min(1 << req.n, self.readout))
                    self.results[rid] = Result(rid, req.n, req.dtype, float(norms[i]), amps, arr, f.admit_s, t)
                del f.batch
            else:
                rid, req, arr = f.members[0]
                amps = f.state.amplitudes(0, min(1 << req.n, self.readout))
                norm = f.state.norm()
                t = clock()
                self.results[rid] = Result(rid, req.n, req.dtype, norm, amps, arr, f.admit_s, t)
                f.state.close()
            self.slots[f.slot].busy = False
            self.mem_used -= f.bytes
            done += len(f.members)
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

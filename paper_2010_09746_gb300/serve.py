"""Continuous-batching request loop: a thin binding of the library's server (qs_server_*).

The server itself is native code (csrc/server.cpp): host threads compile each request's plan
as it arrives, and one admission thread starts a compiled request as soon as a slot (its own
CUDA stream) and enough device memory are free -- it does not wait for the requests already
on the GPU -- so work of different requests overlaps on the device.  Small requests that are
ready together share a slot as one batch (persistent tile-pass launches over all their
states).  Admission order is first-come or least-estimated-work first (with a maximum wait).
Every request runs the same per-tile code on its own state whatever else is in flight, so
its result does not depend on the mix.  This module only submits requests (at their arrival
times, or all at once), polls for results and copies them out.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass
from typing import Dict, Optional

import numpy as np

from . import _lib, marshal
from ._lib import QS_C64, QS_C128

_DT = {"c64": QS_C64, "c128": QS_C128}


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
    batched: bool = False
    status: int = 0          # qs_status; QS_ECANCELED for a request withdrawn before it ran

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


class Server:
    """slots: requests (or batches of small ones) on the GPU at once; mem_budget: device bytes
    for resident states; readout: amplitudes copied back per request (the first
    min(2^n, readout)); order: "fifo" or "sjf" (least estimated work first unless a request
    has waited max_wait_s)."""

    def __init__(self, slots: int = 8, mem_budget: int = 64 << 30, readout: int = 256, tile_bits: int = 0,
                 batch_small_n: int = 16, batch_max: int = 64, order: str = "fifo", max_wait_s: float = 1.0,
                 compile_threads: int = 4):
        if order not in ("fifo", "sjf"):
            raise ValueError("order must be 'fifo' or 'sjf'")
        o = _lib.qs_server_opts()
        o.slots = slots
        o.compile_threads = compile_threads
        o.mem_budget = int(mem_budget)
        o.readout = readout
        o.batch_small_n = batch_small_n if batch_small_n > 0 else -1
        o.batch_max = batch_max
        o.order = 0 if order == "fifo" else 1
        o.max_wait_ms = max(1, int(round(max_wait_s * 1e3)))
        o.tile_bits = tile_bits
        self.mem_budget = int(mem_budget)
        self.readout = readout
        self._L = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(self._L.qs_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._rid_of: Dict[int, int] = {}
        self._arrival: Dict[int, float] = {}
        self.results: Dict[int, Result] = {}

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.qs_server_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    @staticmethod
    def state_bytes(n: int, dtype: str) -> int:
        return (1 << n) * (16 if dtype == "c128" else 8)

    # -- statistics of the native server ---------------------------------------------------
    def stats(self) -> dict:
        st = _lib.qs_server_stats()
        _lib.check(self._L.qs_server_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    @property
    def peak_in_flight(self) -> int:
        return int(self.stats()["peak_in_flight"])

    @property
    def batched_requests(self) -> int:
        return int(self.stats()["batched_requests"])

    @property
    def batches(self) -> int:
        return int(self.stats()["batches"])

    @property
    def peak_mem(self) -> float:
        return self.stats()["peak_mem_bytes"]

    # -- requests ----------------------------------------------------------------------------
    def submit(self, rid: int, req) -> int:
        if self.state_bytes(req.n, req.dtype) > self.mem_budget:
            raise ValueError(f"request {rid} needs more device memory than the whole budget")
        ops, nops, mats = marshal(req.circuit)
        sid = ctypes.c_int64()
        _lib.check(self._L.qs_server_submit(self._h, int(req.n), _DT[req.dtype], ops, nops,
                                            mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mats.size,
                                            ctypes.byref(sid)))
        self._rid_of[sid.value] = rid
        return sid.value

    def cancel(self, sid: int) -> bool:
        """Withdraw submitted request `sid` (the id submit returned) if it has not started on the
        GPU; its result then comes back with status QS_ECANCELED.  False if it already started."""
        st = self._L.qs_server_cancel(self._h, int(sid))
        if st == _lib.QS_EBUSY:
            return False
        _lib.check(st)
        return True

    def poll(self, timeout_s: float = 0.0) -> int:
        """Collect finished requests (waiting up to timeout_s for the first); returns how many."""
        buf = (_lib.qs_server_result * 256)()
        cnt = ctypes.c_int()
        _lib.check(self._L.qs_server_poll(self._h, buf, 256, ctypes.byref(cnt), int(timeout_s * 1e3)))
        for i in range(cnt.value):
            r = buf[i]
            if r.status == _lib.QS_ECANCELED:
                rid = self._rid_of.pop(r.id)
                self._L.qs_server_take(self._h, r.id, None, 0)
                self.results[rid] = Result(rid, r.n, "c128" if r.dtype == QS_C128 else "c64", 0.0,
                                           np.zeros(0, dtype=np.complex64), self._arrival.pop(r.id, r.t_submit_s),
                                           r.t_admit_s, r.t_done_s, False, r.status)
                continue
            if r.status != _lib.QS_OK:
                raise _lib.QSError(r.status, f"request {self._rid_of.get(r.id)}: {r.error.decode(errors='replace')}")
            dt = "c128" if r.dtype == QS_C128 else "c64"
            amps = np.empty(r.amplitudes, dtype=np.complex128 if dt == "c128" else np.complex64)
            _lib.check(self._L.qs_server_take(self._h, r.id, amps.ctypes.data_as(ctypes.c_void_p), r.amplitudes))
            rid = self._rid_of.pop(r.id)
            arr = self._arrival.pop(r.id, r.t_submit_s)
            self.results[rid] = Result(rid, r.n, dt, r.norm, amps, arr, r.t_admit_s, r.t_done_s, bool(r.batched))
        return cnt.value

    def run(self, requests, realtime: bool = True, timeout_s: float = 600.0) -> Dict[int, Result]:
        """Serve `requests` (objects with arrival_s, n, dtype, circuit).  realtime: each request
        is submitted at its arrival time (server clock); otherwise all at once.  Latency runs
        from submission to the result being in host memory."""
        self.results = {}
        reqs = sorted(enumerate(requests), key=lambda t: t[1].arrival_s)
        st0 = self.stats()["now_s"]
        w0 = time.perf_counter()
        nxt = 0
        while len(self.results) < len(reqs):
            now = time.perf_counter() - w0
            if now > timeout_s:
                raise TimeoutError("serving did not finish in time")
            while nxt < len(reqs) and (not realtime or reqs[nxt][1].arrival_s <= now):
                rid, r = reqs[nxt]
                sid = self.submit(rid, r)
                if realtime:   # the arrival instant on the server's clock
                    self._arrival[sid] = st0 + r.arrival_s
                nxt += 1
            wait = 0.05
            if realtime and nxt < len(reqs):
                wait = max(0.0, min(wait, reqs[nxt][1].arrival_s - (time.perf_counter() - w0)))
            self.poll(wait)
        return self.results


def latency_summary(results: Dict[int, Result], wall_s: Optional[float] = None) -> dict:
    lat = np.array([r.latency_s for r in results.values()])
    out = {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50) * 1e3),
           "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}
    if wall_s:
        out["circuits_per_s"] = len(lat) / wall_s
    return out

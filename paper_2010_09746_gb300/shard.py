"""Global-qubit sharding: the paper's distributed setting (Sec. 2, Sec. 3, Appendix A).

The state of n qubits is split over P = 2^g processes.  Process r holds the 2^m amplitudes
(m = n - g) whose top g storage bits equal r: the paper's "global" qubits are storage bits
m .. n-1, its "local" qubits storage bits 0 .. m-1.  The circuit is compiled by the library's
Algorithm 1 with m local qubits (QS_MODE_PAPER), and its schedule (qs_plan_get_trace) is run
by every process on its own slice:

* a local gate: its qubits' storage bits are local, or it acts on its global qubits only
  through controls and diagonal factors (block diagonal in them): the process applies the
  block that its own global bits select (a gate on global qubits only becomes a scalar);
* PermuteQubits of one transposition, local qubit l <-> global qubit g, as Appendix A
  splits it: a local permutation that brings l to the top local position m - 1 (no
  communication), then a pairwise exchange with the process whose rank differs in the bit
  of g: each process sends the half of its slice whose top local bit differs from its own
  bit of g and receives its partner's half into the same place;
* a gate that Algorithm 1 runs non-locally (non-diagonal on a global qubit) first exchanges
  each such global qubit with a local position in the same way, then runs locally.

The slice lives in a backend (`StateBackend`: the library's State on this process's GPU; the
tests use a CPU backend with the same methods) and halves travel through a transport
(`TorchTransport`: torch.distributed point-to-point send/recv; NCCL between GPUs, gloo on
CPUs).  Nothing here does arithmetic on amplitudes: gates run in the backend.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence

import numpy as np

from . import QS_ORDER_STORAGE, State, _lib, compile as qs_compile, marshal


def gate_matrices(n: int, circuit: Sequence) -> List[np.ndarray]:
    """Each gate's full 2^k x 2^k matrix as the library defines it (qs_gate_matrix), with
    r = sum_t b(q_t) 2^t."""
    ops, nops, mats = marshal(circuit)
    L = _lib.load()
    buf = np.zeros(2 * 4 ** 6)
    k = ctypes.c_int()
    out = []
    for i in range(nops):
        _lib.check(L.qs_gate_matrix(n, ctypes.byref(ops[i]), mats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    mats.size, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(k)))
        d = 1 << k.value
        out.append(buf[: 2 * d * d].view(np.complex128).reshape(d, d).copy())
    return out


def sharded_program(n: int, g: int, circuit: Sequence, dtype: str = "c128") -> list:
    """Algorithm 1 with m = n - g local qubits, as a list of ("gate", index) and
    ("swap", l, g) (a local<->global transposition) and ("nonlocal", index)."""
    m = n - g
    plan = qs_compile(n, list(circuit), mode="paper", dtype=dtype, tile_bits=m)
    prog = []
    for kind, v in plan.trace():
        if kind == 0:
            prog.append(("gate", v))
        elif kind == 1:
            prog.append(("nonlocal", v))
        elif kind == 2:
            prog.append(("swap",) + divmod(v, 64))
    return prog


def block_for_rank(U: np.ndarray, slots: Sequence[int], m: int, rank: int):
    """The part of a gate this rank applies: (local matrix, local slots), or None when the
    gate is not block diagonal in its global qubits.  slots[t] is the storage bit of the
    gate's qubit t; bits >= m are global, with the value of bit (slot - m) of the rank."""
    k = len(slots)
    loc = [t for t in range(k) if slots[t] < m]
    glo = [t for t in range(k) if slots[t] >= m]
    if not glo:
        return U, list(slots)
    gmask = sum(1 << t for t in glo)
    gval = sum(((rank >> (slots[t] - m)) & 1) << t for t in glo)
    r_idx = np.arange(1 << k)
    same = ((r_idx[:, None] ^ r_idx[None, :]) & gmask) == 0
    if np.any(U[~same] != 0):
        return None
    sel = [r for r in range(1 << k) if (r & gmask) == gval]   # ascending local index order
    return U[np.ix_(sel, sel)], [slots[t] for t in loc]


class TorchTransport:
    """Pairwise exchange over torch.distributed (send / recv of one tensor each way)."""

    def __init__(self, dist):
        self.dist = dist

    def exchange(self, partner: int, send_buf, recv_buf):
        reqs = self.dist.batch_isend_irecv([self.dist.P2POp(self.dist.isend, send_buf, partner),
                                            self.dist.P2POp(self.dist.irecv, recv_buf, partner)])
        for r in reqs:
            r.wait()


class StateBackend:
    """The slice as a library State of m qubits on this process's GPU (kept at the identity
    permutation, so its logical qubit p is storage bit p); halves are copied through torch
    device buffers (qs_copy_range_device)."""

    def __init__(self, m: int, dtype: str = "c128", device: int = 0, rank: int = 0):
        import torch
        self.torch = torch
        self.m = m
        self.dtype = dtype
        self.device = device
        self.state = State(m, dtype)   # |0...0> on the current device
        if rank:                       # only rank 0 holds amplitude 0 of the whole state
            self.scale(0.0)

    def apply(self, U: np.ndarray, slots: Sequence[int]):
        if len(slots) == 1:
            self.state.apply_1q(U, slots[0])
        elif len(slots) == 2:
            self.state.apply_2q(U, slots[0], slots[1])
        else:
            self.state.apply_dense(U, list(slots))

    def scale(self, z: complex):
        self.state.apply_1q(np.array([[z, 0], [0, z]]), 0)

    def swap_bits(self, a: int, b: int):
        perm = list(range(self.m))
        perm[a], perm[b] = b, a
        self.state.permute(perm)                      # data moves
        self.state.run([_Relabel(a, b)], mode="pergate")   # back to the identity permutation

    def buffer(self, count: int):
        """A device buffer of `count` amplitudes; the executor asks for two per exchange, always of
        the same size, so the two are kept and handed out in turn."""
        el = self.torch.float64 if self.dtype == "c128" else self.torch.float32
        pool = self.__dict__.setdefault("_bufs", [])
        if len(pool) < 2 or pool[0].numel() != 2 * count:
            pool[:] = [self.torch.empty(2 * count, dtype=el, device=f"cuda:{self.device}") for _ in range(2)]
            self._next = 0
        b = pool[self._next]
        self._next ^= 1
        return b

    def read_range(self, first: int, buf):
        _lib.check(_lib.load().qs_copy_range_device(self.state.handle, ctypes.c_void_p(buf.data_ptr()), first,
                                                   buf.numel() // 2, 0))

    def write_range(self, first: int, buf):
        _lib.check(_lib.load().qs_copy_range_device(self.state.handle, ctypes.c_void_p(buf.data_ptr()), first,
                                                   buf.numel() // 2, 1))

    def amplitudes(self) -> np.ndarray:
        return self.state.amplitudes(order=QS_ORDER_STORAGE)


class _Relabel:
    kind = "RELABEL"
    param = 0.0
    matrix = None

    def __init__(self, a, b):
        self.qubits = (a, b)


class ShardedRun:
    """Runs a circuit on rank `rank` of 2^g processes (global-qubit sharding)."""

    def __init__(self, n: int, g: int, rank: int, backend, transport, dtype: str = "c128"):
        if g < 0 or n - g < 1:
            raise ValueError("need 0 <= g < n")
        if not 0 <= rank < (1 << g):
            raise ValueError("rank outside 0 .. 2^g - 1")
        self.n, self.g, self.m, self.rank = n, g, n - g, rank
        self.backend, self.transport, self.dtype = backend, transport, dtype
        self.sigma = list(range(n))        # logical qubit -> storage bit (global: >= m)
        self.exchanges = 0

    def _move_to_top(self, q: int):
        """Local permutation: logical qubit q (local) to storage bit m - 1."""
        top = self.m - 1
        p = self.sigma[q]
        if p == top:
            return
        other = self.sigma.index(top)
        self.backend.swap_bits(p, top)
        self.sigma[q], self.sigma[other] = top, p

    def transpose(self, l: int, gq: int):
        """PermuteQubits of the transposition l (local) <-> gq (global), Appendix A."""
        if not (self.sigma[l] < self.m <= self.sigma[gq]):
            raise ValueError("transposition must exchange a local and a global qubit")
        self._move_to_top(l)
        pg = self.sigma[gq]
        bit = pg - self.m
        mine = (self.rank >> bit) & 1
        partner = self.rank ^ (1 << bit)
        half = 1 << (self.m - 1)
        first = (1 - mine) * half           # the half whose top local bit differs from mine
        send = self.backend.buffer(half)
        recv = self.backend.buffer(half)
        self.backend.read_range(first, send)
        self.transport.exchange(partner, send, recv)
        self.backend.write_range(first, recv)
        self.sigma[l], self.sigma[gq] = pg, self.m - 1
        self.exchanges += 1

    def apply(self, U: np.ndarray, qubits: Sequence[int]):
        slots = [self.sigma[q] for q in qubits]
        blk = block_for_rank(U, slots, self.m, self.rank)
        if blk is None:   # non-diagonal on a global qubit: bring those qubits local first
            busy = {self.sigma[q] for q in qubits}
            for q in qubits:
                if self.sigma[q] < self.m:
                    continue
                # a local qubit not used by this gate takes the global position
                cand = [x for x in range(self.n) if self.sigma[x] < self.m and self.sigma[x] not in busy]
                if not cand:
                    raise ValueError("gate needs more qubits than a process holds locally (n - g)")
                loc = max(cand, key=lambda x: self.sigma[x])
                self.transpose(loc, q)
                busy = {self.sigma[x] for x in qubits}
            slots = [self.sigma[q] for q in qubits]
            blk = block_for_rank(U, slots, self.m, self.rank)
        Ul, ls = blk
        if ls:
            self.backend.apply(Ul, ls)
        else:
            self.backend.scale(complex(Ul[0, 0]))

    def run(self, circuit: Sequence):
        circuit = list(circuit)
        mats = gate_matrices(self.n, circuit)
        for ins in sharded_program(self.n, self.g, circuit, self.dtype):
            if ins[0] in ("gate", "nonlocal"):
                v = ins[1]
                self.apply(mats[v], list(circuit[v].qubits))
            else:
                self.transpose(ins[1], ins[2])
        return self

"""GB300 (sm_103a) state-vector simulator: Python binding of libqs.so.

Thin ctypes marshalling over the C ABI of include/qs.h -- gates, PermuteQubits, the
compiler pass and the read-outs all run in the library's CUDA kernels (there is no
CPU implementation here).  PyTorch is optional plumbing: `use_torch_allocator()` routes
device allocations through torch's caching allocator and `State.set_stream` accepts a
torch.cuda.Stream.
"""
from __future__ import annotations

import ctypes
import itertools
from typing import Iterable, List, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (QS_ARITH_AUTO, QS_ARITH_DF, QS_ARITH_F64, QS_C64, QS_C128, QS_MODE_PAPER,
                   QS_MODE_PERGATE, QS_MODE_TILE, QS_ORDER_LOGICAL, QS_ORDER_STORAGE, QSError)

__all__ = ["State", "Plan", "Batch", "compile", "marshal", "use_torch_allocator", "QSError", "QS_C64", "QS_C128",
           "QS_MODE_PERGATE", "QS_MODE_PAPER", "QS_MODE_TILE", "QS_ARITH_AUTO", "QS_ARITH_DF", "QS_ARITH_F64",
           "QS_ORDER_LOGICAL", "QS_ORDER_STORAGE", "lib_path"]

_DTYPES = {"c64": QS_C64, "c128": QS_C128, QS_C64: QS_C64, QS_C128: QS_C128}
_MODES = {"pergate": QS_MODE_PERGATE, "paper": QS_MODE_PAPER, "tile": QS_MODE_TILE,
          QS_MODE_PERGATE: QS_MODE_PERGATE, QS_MODE_PAPER: QS_MODE_PAPER, QS_MODE_TILE: QS_MODE_TILE}
_ARITH = {"auto": QS_ARITH_AUTO, "df": QS_ARITH_DF, "f64": QS_ARITH_F64,
          QS_ARITH_AUTO: QS_ARITH_AUTO, QS_ARITH_DF: QS_ARITH_DF, QS_ARITH_F64: QS_ARITH_F64}


def lib_path() -> str:
    return _lib.LIB_PATH


def _L():
    return _lib.load()


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _cmat(m) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(m, dtype=np.complex128)).view(np.float64).ravel().copy()


# qs_op as a numpy record (same field order, sizes and alignment as the C struct)
_OP_DTYPE = np.dtype([("kind", "<i4"), ("nq", "<i4"), ("q", "<i4", (6,)), ("param", "<f8"), ("mat", "<i8")],
                     align=True)
assert _OP_DTYPE.itemsize == ctypes.sizeof(_lib.qs_op)


def marshal(circuit: Iterable):
    """Gate objects (attributes kind, qubits, param, matrix) -> (qs_op array, matrix doubles).

    The fields are gathered with one list comprehension each and written column by column
    into a record array that the qs_op array shares, and the matrices are concatenated in
    one call, so that a batch of millions of gates marshals in C loops rather than one
    ctypes field write at a time."""
    gates = list(circuit)
    N = len(gates)
    rec = np.zeros(max(1, N), dtype=_OP_DTYPE)
    codes = _lib.OP_CODES
    rec["kind"][:N] = [codes[g.kind] for g in gates]
    qls = [tuple(g.qubits) for g in gates]
    nq = np.fromiter(map(len, qls), dtype=np.int64, count=N)
    if N and int(nq.max()) > 6:
        raise ValueError("a gate acts on more than 6 qubits")
    rec["nq"][:N] = nq
    total = int(nq.sum())
    if total:   # qubit t of gate i goes to q[i][t]
        flat = np.fromiter(itertools.chain.from_iterable(qls), dtype=np.int64, count=total)
        row = np.repeat(np.arange(N), nq)
        col = np.arange(total) - np.repeat(np.cumsum(nq) - nq, nq)
        rec["q"][row, col] = flat
    rec["param"][:N] = [float(getattr(g, "param", 0.0) or 0.0) for g in gates]
    ms = [getattr(g, "matrix", None) for g in gates]
    has = [i for i, m in enumerate(ms) if m is not None]
    rec["mat"][:N] = -1
    if has:
        arrs = [np.asarray(ms[i], dtype=np.complex128) for i in has]
        sizes = np.fromiter(map(np.size, arrs), dtype=np.int64, count=len(arrs))
        rec["mat"][np.array(has)] = 2 * (np.cumsum(sizes) - sizes)   # first double of each matrix
        buf = np.concatenate(arrs, axis=None).view(np.float64)      # each matrix row-major
    else:
        buf = np.zeros(1)
    ops = (_lib.qs_op * max(1, N)).from_buffer(rec)
    return ops, N, np.ascontiguousarray(buf, dtype=np.float64)


def _opts(mode="tile", dtype="c128", arith="auto", tile_bits=0, low_bits=0, max_ops=0, scoring=0, reg_bits=0,
          renorm_every=0, full_rx=False, dense=True, fuse=True, cost=None):
    o = _lib.qs_compile_opts()
    o.mode = _MODES[mode]
    o.dtype = _DTYPES[dtype]
    o.arith = _ARITH[arith]
    o.tile_bits = tile_bits
    o.low_bits = low_bits
    o.max_ops = max_ops
    o.scoring = scoring
    o.flags = (_lib.QS_FLAG_FULL_RX if full_rx else 0) | (0 if dense else _lib.QS_FLAG_NO_DENSE) | \
        (0 if fuse else _lib.QS_FLAG_NO_FUSE)
    o.reg_bits = reg_bits
    o.renorm_every = renorm_every
    if cost is not None:   # a qs_cost_model (tuning.CostModel.native); read during qs_compile only
        o.cost = ctypes.pointer(cost)
    return o


def default_cost_model(dtype="c128", arith="auto"):
    """The compiler's built-in kernel cost model for this dtype (qs_default_cost_model)."""
    m = _lib.qs_cost_model()
    _lib.check(_L().qs_default_cost_model(_DTYPES[dtype], _ARITH[arith], ctypes.byref(m)))
    return m


class Plan:
    """A compiled circuit (qs_compile); run it with State.execute."""

    def __init__(self, n: int, circuit: Iterable, sigma0: Optional[Sequence[int]] = None, **opts):
        L = _L()
        self.n = n
        ops, nops, mats = marshal(circuit)
        self._opts = _opts(**opts)
        s0 = None
        if sigma0 is not None:
            s0 = np.ascontiguousarray(sigma0, dtype=np.int32)
        h = ctypes.c_void_p()
        _lib.check(L.qs_compile(n, ops, nops, _dp(mats), mats.size, _ip(s0) if s0 is not None else None,
                                ctypes.byref(self._opts), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _L().qs_plan_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        st = _lib.qs_plan_stats()
        _lib.check(_L().qs_plan_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def final_permutation(self) -> List[int]:
        out = np.zeros(self.n, dtype=np.int32)
        _lib.check(_L().qs_plan_final_permutation(self._h, _ip(out)))
        return [int(x) for x in out]

    def export_swaps(self, circuit):
        """QS_MODE_PAPER schedule as a plain gate list for any backend (Appendix B): the gates
        in scheduled order, every PermuteQubits(l <-> g) written as SWAP(l, g) followed by the
        Emulated-SWAP RELABEL(l, g).  On hardware RELABEL is a SWAP (the pair cancels); on this
        simulator it only exchanges storage positions, so SWAP + RELABEL moves the data."""
        from types import SimpleNamespace
        circuit = list(circuit)
        out = []
        for kind, v in self.trace():
            if kind in (0, 1):
                out.append(circuit[v])
            elif kind == 2:
                l, g = divmod(v, 64)
                out.append(SimpleNamespace(kind="SWAP", qubits=(l, g), param=0.0, matrix=None))
                out.append(SimpleNamespace(kind="RELABEL", qubits=(l, g), param=0.0, matrix=None))
        return out

    def trace(self):
        cnt = ctypes.c_size_t()
        _lib.check(_L().qs_plan_get_trace(self._h, None, None, 0, ctypes.byref(cnt)))
        k = np.zeros(max(1, cnt.value), dtype=np.int32)
        v = np.zeros(max(1, cnt.value), dtype=np.int32)
        _lib.check(_L().qs_plan_get_trace(self._h, k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cnt.value,
                                          ctypes.byref(cnt)))
        return [(int(a), int(b)) for a, b in zip(k[:cnt.value], v[:cnt.value])]


def compile(n: int, circuit: Iterable, sigma0=None, **opts) -> Plan:
    return Plan(n, circuit, sigma0, **opts)


class State:
    """2^n complex amplitudes on the GPU (qs_create)."""

    def __init__(self, n: int, dtype="c128", arith="auto", stream=None):
        L = _L()
        self.n = n
        self.dtype = _DTYPES[dtype]
        self.arith = _ARITH[arith]
        h = ctypes.c_void_p()
        _lib.check(L.qs_create(n, self.dtype, ctypes.byref(h)))
        self._h = h
        if arith != "auto":
            _lib.check(L.qs_set_arith(h, _ARITH[arith]))
        if stream is not None:
            self.set_stream(stream)

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            _L().qs_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    @property
    def np_dtype(self):
        return np.complex128 if self.dtype == QS_C128 else np.complex64

    def set_stream(self, stream):
        ptr = getattr(stream, "cuda_stream", stream)
        _lib.check(_L().qs_set_stream(self._h, ctypes.c_void_p(int(ptr) if ptr else 0)))

    def set_arith(self, arith):
        _lib.check(_L().qs_set_arith(self._h, _ARITH[arith]))
        self.arith = _ARITH[arith]

    def set_dense_path(self, path: str):
        """Engine of apply_dense: "auto", "cuda_cores" or "tensor" (qs_set_dense_path)."""
        code = {"auto": _lib.QS_DENSE_AUTO, "cuda_cores": _lib.QS_DENSE_CUDA_CORES, "tensor": _lib.QS_DENSE_TENSOR}[path]
        _lib.check(_L().qs_set_dense_path(self._h, code))

    def set_profiling(self, on: bool):
        _lib.check(_L().qs_set_profiling(self._h, 1 if on else 0))

    def kernel_stats(self) -> List[dict]:
        cnt = ctypes.c_int()
        buf = (_lib.qs_kernel_stat * 64)()
        _lib.check(_L().qs_get_kernel_stats(self._h, buf, 64, ctypes.byref(cnt)))
        return [{"name": buf[i].name.decode(), "launches": buf[i].launches, "total_ms": buf[i].total_ms,
                 "bytes": buf[i].bytes, "alu": buf[i].alu} for i in range(min(cnt.value, 64))]

    def reset_kernel_stats(self):
        _lib.check(_L().qs_reset_kernel_stats(self._h))

    def reset(self):
        _lib.check(_L().qs_reset(self._h))

    def sync(self):
        _lib.check(_L().qs_sync(self._h))

    def device_ptr(self) -> int:
        p = ctypes.c_void_p()
        _lib.check(_L().qs_get_info(self._h, None, None, ctypes.byref(p), None))
        return int(p.value or 0)

    # -- gates ----------------------------------------------------------------------------
    def apply_1q(self, U, q: int):
        _lib.check(_L().qs_apply_1q(self._h, _dp(_cmat(U)), int(q)))

    def apply_2q(self, U, q0: int, q1: int):
        _lib.check(_L().qs_apply_2q(self._h, _dp(_cmat(U)), int(q0), int(q1)))

    def apply_controlled(self, U, c: int, t: int):
        _lib.check(_L().qs_apply_controlled(self._h, _dp(_cmat(U)), int(c), int(t)))

    def apply_dense(self, U, qubits: Sequence[int]):
        qs = np.ascontiguousarray(qubits, dtype=np.int32)
        _lib.check(_L().qs_apply_dense(self._h, _dp(_cmat(U)), len(qs), _ip(qs)))

    def permute(self, perm: Sequence[int]):
        p = np.ascontiguousarray(perm, dtype=np.int32)
        if p.size != self.n:
            raise QSError(_lib.QS_EINVAL, "perm must have n entries")
        _lib.check(_L().qs_permute(self._h, _ip(p)))

    def permutation(self) -> List[int]:
        out = np.zeros(self.n, dtype=np.int32)
        _lib.check(_L().qs_get_permutation(self._h, _ip(out)))
        return [int(x) for x in out]

    def execute(self, plan: Plan):
        _lib.check(_L().qs_execute(self._h, plan.handle))

    def run(self, circuit: Iterable, **opts):
        ops, nops, mats = marshal(circuit)
        opts.setdefault("arith", self.arith)
        o = _opts(dtype=self.dtype, **opts)
        _lib.check(_L().qs_run(self._h, ops, nops, _dp(mats), mats.size, ctypes.byref(o)))

    # -- read-outs ------------------------------------------------------------------------
    def probabilities(self, order=QS_ORDER_LOGICAL) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.float64)
        _lib.check(_L().qs_probabilities(self._h, _dp(out), order))
        return out

    def amplitudes(self, first: int = 0, count: Optional[int] = None, order=QS_ORDER_LOGICAL) -> np.ndarray:
        if count is None:
            count = (1 << self.n) - first
        out = np.empty(count, dtype=self.np_dtype)
        _lib.check(_L().qs_get_amplitudes(self._h, out.ctypes.data_as(ctypes.c_void_p), first, count, order))
        return out

    def set_amplitudes(self, storage_vec: np.ndarray):
        a = np.ascontiguousarray(storage_vec, dtype=self.np_dtype)
        if a.size != (1 << self.n):
            raise QSError(_lib.QS_EINVAL, "vector must have 2^n entries")
        _lib.check(_L().qs_set_amplitudes(self._h, a.ctypes.data_as(ctypes.c_void_p)))

    def norm(self) -> float:
        out = ctypes.c_double()
        _lib.check(_L().qs_norm(self._h, ctypes.byref(out)))
        return out.value

    def inner(self, other: "State") -> complex:
        """<self|other> in FP64 (qs_inner); same n and permutation, any dtypes."""
        out = np.zeros(2, dtype=np.float64)
        _lib.check(_L().qs_inner(self._h, other._h, _dp(out)))
        return complex(out[0], out[1])

    def fidelity(self, other: "State") -> float:
        """|<self|other>|^2 / (<self|self> <other|other>), every reduction in FP64."""
        return abs(self.inner(other)) ** 2 / (self.norm() * other.norm())

    def renormalize(self, sync: bool = True) -> Optional[float]:
        """Divide by the square root of the FP64 norm (qs_renormalize); returns the norm
        before scaling when sync is true, else enqueues without synchronising."""
        if not sync:
            _lib.check(_L().qs_renormalize(self._h, None))
            return None
        out = ctypes.c_double()
        _lib.check(_L().qs_renormalize(self._h, ctypes.byref(out)))
        return out.value


class Batch:
    """Many independent circuits run together (qs_batch_create): list of (n, circuit)."""

    @staticmethod
    def marshal(circuits):
        """(n list, qs_op array, op offsets, matrix doubles) of a list of (n, circuit): the
        arrays qs_batch_create takes; pass them as `marshalled` to skip this step."""
        circuits = list(circuits)
        allg = []
        offs = [0]
        for _, c in circuits:
            c = list(c)
            allg.extend(c)
            offs.append(offs[-1] + len(c))
        ops, nops, mats = marshal(allg)
        return [int(n) for n, _ in circuits], ops, offs, mats

    def __init__(self, circuits=None, dtype="c64", stream=None, graph=True, marshalled=None, **opts):
        L = _L()
        ns, ops, offs, mats = marshalled if marshalled is not None else Batch.marshal(circuits)
        self.count = len(ns)
        self.ns = list(ns)
        self.dtype = _DTYPES[dtype]
        n_arr = np.ascontiguousarray(self.ns, dtype=np.int32)
        off_arr = np.ascontiguousarray(offs, dtype=np.int64)
        o = _opts(dtype=dtype, **opts)
        h = ctypes.c_void_p()
        _lib.check(L.qs_batch_create(self.count, _ip(n_arr), ops, off_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     _dp(mats), mats.size, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        if stream is not None:
            ptr = getattr(stream, "cuda_stream", stream)
            _lib.check(L.qs_batch_set_stream(h, ctypes.c_void_p(int(ptr) if ptr else 0)))
        _lib.check(L.qs_batch_set_graph(h, 1 if graph else 0))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _L().qs_batch_destroy(h)
            self._h = None

    def run(self):
        _lib.check(_L().qs_batch_run(self._h))

    def sync(self):
        _lib.check(_L().qs_batch_sync(self._h))

    def norms(self) -> np.ndarray:
        out = np.empty(self.count, dtype=np.float64)
        _lib.check(_L().qs_batch_norms(self._h, _dp(out)))
        return out

    def amplitudes(self, i: int, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        if count is None:
            count = (1 << self.ns[i]) - first
        out = np.empty(count, dtype=np.complex128 if self.dtype == QS_C128 else np.complex64)
        _lib.check(_L().qs_batch_get_amplitudes(self._h, int(i), out.ctypes.data_as(ctypes.c_void_p), first, count))
        return out

    def stats(self) -> dict:
        st = _lib.qs_batch_stats()
        _lib.check(_L().qs_batch_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}


_torch_cb = None


def use_torch_allocator(device: int = 0):
    """Route every device allocation of the library through torch's caching allocator."""
    global _torch_cb
    import torch

    def _alloc(nbytes, ctx, stream):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, stream if stream else None))
        except Exception:  # noqa: BLE001 - allocation failure is reported as NULL
            return None

    def _free(ptr, nbytes, ctx, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    a = _lib.ALLOC_FN(_alloc)
    f = _lib.FREE_FN(_free)
    _lib.check(_L().qs_set_allocator(a, f, None))
    _torch_cb = (a, f)


def use_default_allocator():
    global _torch_cb
    null_a = ctypes.cast(None, _lib.ALLOC_FN)
    null_f = ctypes.cast(None, _lib.FREE_FN)
    _lib.check(_L().qs_set_allocator(null_a, null_f, None))
    _torch_cb = None


def selftest_bounded_wait(limit_us: int = 20000) -> int:
    """Run the bounded-wait self-test (qs_selftest_bounded_wait); returns the status the
    device reported (QS_ETIMEOUT when the deliberately unsatisfiable wait expired)."""
    out = ctypes.c_int(-1)
    _lib.check(_L().qs_selftest_bounded_wait(int(limit_us), ctypes.byref(out)))
    return out.value

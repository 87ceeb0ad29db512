"""CPU, world sizes 2 and 4 over gloo: global-qubit sharding (the paper's setting, Sec. 2 and
Appendix A).  Each rank holds 2^(n-g) amplitudes; the library's Algorithm 1 (m = n - g local
qubits) schedules the gates and the local<->global transpositions; transpositions become a
local permutation plus a pairwise exchange of half slices over torch.distributed.  The slice
here lives in a CPU backend whose arithmetic is the oracle's, so the test checks the rank
logic and the data movement: the gathered state must equal the oracle's full-state result
(1e-12), and the number of exchanges must equal the number of transpositions in the plan.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import sv
from workloads import circuits as wc

qs = pytest.importorskip("paper_2010_09746_gb300")
from paper_2010_09746_gb300 import shard  # noqa: E402


class OracleSliceBackend:
    """A rank's slice in host memory; gates through the oracle's routines on the slice."""

    def __init__(self, m, rank):
        self.m = m
        self.o = sv.OracleState(m)
        if rank:
            self.o.psi[:] = 0.0

    def apply(self, U, slots):
        self.o.apply_dense(U, list(slots))

    def scale(self, z):
        self.o.psi *= z

    def swap_bits(self, a, b):
        ident = list(range(self.m))
        perm = list(ident)
        perm[a], perm[b] = b, a
        self.o.psi = sv.permute_storage(self.o.psi, self.m, ident, perm)

    def buffer(self, count):
        return torch.empty(2 * count, dtype=torch.float64)

    def read_range(self, first, buf):
        n = buf.numel() // 2
        buf.copy_(torch.from_numpy(self.o.psi[first:first + n].view(np.float64).copy()))

    def write_range(self, first, buf):
        n = buf.numel() // 2
        self.o.psi[first:first + n] = buf.numpy().view(np.complex128)

    def amplitudes(self):
        return self.o.psi


def circuits(n):
    return {"paper_p0.3": wc.paper_random_circuit(n, 0.3, seed=n),
            "rzrx_cz": wc.rzrx_cz_circuit(n, 6, seed=n),
            "qft_like": wc.qft_like_circuit(n),
            "haar_cnot": wc.haar_cnot_circuit(n, 4, seed=n),
            "mixed": wc.random_mixed_circuit(n, 60, seed=n, kmax=3)}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = world.bit_length() - 1
        out = {}
        for name, circ in circuits(n).items():
            be = OracleSliceBackend(n - g, rank)
            run = shard.ShardedRun(n, g, rank, be, shard.TorchTransport(dist)).run(circ)
            t = torch.from_numpy(be.amplitudes().view(np.float64).copy())
            parts = [torch.empty_like(t) for _ in range(world)] if rank == 0 else None
            dist.gather(t, parts, dst=0)
            if rank == 0:
                full = np.concatenate([p.numpy().view(np.complex128) for p in parts])
                out[name] = (full, list(run.sigma), run.exchanges)
        if rank == 0:
            q.put(out)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 9), (4, 10)])
def test_sharded_runs_match_oracle(world, n):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    import queue
    import time
    t0 = time.time()
    got = None
    while got is None:   # stop early if a rank died
        try:
            got = q.get(timeout=2)
        except queue.Empty:
            assert all(p.exitcode in (None, 0) for p in procs), [p.exitcode for p in procs]
            assert time.time() - t0 < 300, "sharded run did not finish"
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = world.bit_length() - 1
    for name, circ in circuits(n).items():
        full, sigma, exchanges = got[name]
        psi = sv.to_logical(full, n, sigma)
        ref = sv.simulate(n, circ)
        assert np.max(np.abs(psi - ref)) <= 1e-12, name
        prog = shard.sharded_program(n, g, circ)
        swaps = sum(1 for ins in prog if ins[0] == "swap")
        assert exchanges >= swaps, name   # plus one per global qubit a non-local gate brings in
    # the circuits do communicate
    assert any(e > 0 for _, _, e in got.values())


def test_block_for_rank():
    """Controls and diagonal factors on global qubits select a block; non-diagonal action on
    a global qubit is refused."""
    c, s = np.cos(0.3), np.sin(0.3)
    rx = np.array([[c, -1j * s], [-1j * s, c]])
    cnot = np.eye(4)[[0, 3, 2, 1]]      # control q0 (bit 0), target q1 (bit 1)
    m = 3
    # control on a global qubit (storage bit 3 = rank bit 0)
    assert np.array_equal(shard.block_for_rank(cnot, [3, 1], m, 1)[0], np.array([[0, 1], [1, 0]]))
    assert np.array_equal(shard.block_for_rank(cnot, [3, 1], m, 0)[0], np.eye(2))
    # target on a global qubit: non-local
    assert shard.block_for_rank(cnot, [1, 3], m, 0) is None
    assert shard.block_for_rank(rx, [4], m, 0) is None
    # a phase on a global qubit alone: a scalar
    rz = np.diag([np.exp(-0.2j), np.exp(0.2j)])
    Ul, slots = shard.block_for_rank(rz, [4], m, 2)
    assert slots == [] and Ul.shape == (1, 1) and Ul[0, 0] == np.exp(0.2j)

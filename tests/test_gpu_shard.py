"""GPU: the sharded executor with its slices in library States on this GPU.

Each rank's slice is a qs State (kernels on this GPU); the ranks are host threads, and the
pairwise exchange of half slices goes through device buffers (qs_copy_range_device) and a host
rendezvous -- no kernel waits on another rank's kernel.  The gathered state must match the FP64
oracle (complex128: 1e-12, complex64: 1e-5).  Multi-GPU runs (one process per GPU over NCCL)
use the same executor with torch.distributed as the transport.
"""
import threading

import numpy as np
import pytest

from oracle import sv
from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")
torch = pytest.importorskip("torch")
from paper_2010_09746_gb300 import shard  # noqa: E402


class ThreadTransport:
    """Rank `rank` of a group of threads: exchange = post my buffer, wait for everyone, take my
    partner's, wait again (every rank exchanges at the same points of the program)."""

    def __init__(self, rank, box, barrier):
        self.rank, self.box, self.barrier = rank, box, barrier

    def exchange(self, partner, send, recv):
        self.box[(self.rank, partner)] = send.clone()
        self.barrier.wait()
        recv.copy_(self.box[(partner, self.rank)])
        torch.cuda.synchronize()
        self.barrier.wait()


@pytest.mark.parametrize("world,n,dtype", [(2, 12, "c128"), (4, 12, "c128"), (4, 13, "c64")])
def test_sharded_on_states(world, n, dtype):
    g = world.bit_length() - 1
    circ = wc.paper_random_circuit(n, 0.3, seed=n) + wc.rzrx_cz_circuit(n, 4, seed=n) + wc.qft_like_circuit(n)
    box, barrier = {}, threading.Barrier(world)
    backends = [shard.StateBackend(n - g, dtype, rank=r) for r in range(world)]
    runs = [shard.ShardedRun(n, g, r, backends[r], ThreadTransport(r, box, barrier), dtype=dtype) for r in range(world)]
    errors = []

    def go(r):
        try:
            runs[r].run(circ)
        except Exception as e:  # noqa: BLE001
            errors.append(e)
            barrier.abort()

    th = [threading.Thread(target=go, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errors, errors
    assert runs[0].exchanges > 0
    full = np.concatenate([b.amplitudes().astype(np.complex128) for b in backends])
    psi = sv.to_logical(full, n, runs[0].sigma)
    ref = sv.simulate(n, circ)
    tol = 1e-12 if dtype == "c128" else 1e-5
    assert np.max(np.abs(psi - ref)) <= tol
    assert all(r.sigma == runs[0].sigma for r in runs)

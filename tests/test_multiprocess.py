"""CPU, world size 2 over gloo: the replica path of bench.py.  Each rank times its own
replica; the job's time is the slowest rank's and its throughput counts every rank's
units (weak scaling, no collective on the data path)."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 100.0 + 50.0 * rank          # rank 1 is the slow replica
        mx = bench.reduce_max(my_ms, dist)
        rate = bench.job_rate(2680, world, mx)
        w, r, _ = bench.dist_env()
        q.put((rank, mx, rate, w, r))
    finally:
        dist.destroy_process_group()


def test_replica_reduction_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, mx, rate, w, r in got:
        assert mx == 150.0                       # the slowest replica's time
        assert abs(rate - 2 * 2680 / 0.150) < 1e-6
        assert w == 2 and r == rank


def test_single_process_reduction_is_identity():
    assert bench.reduce_max(12.5, None) == 12.5
    assert bench.job_rate(100, 1, 1000.0) == 100.0

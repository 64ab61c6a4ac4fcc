"""The multi-GPU path is replicas only (independent grids, no collective on
the data path): the bench's whole-job rate takes the slowest rank's time and
all ranks' points.  Checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [40.0, 50.0][rank]  # rank 1 is the slower replica
        ms, rate = bench.replica_rate(local_ms, 1000, 4, world, torch.device("cpu"))
        out.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_replica_rate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 50.0
        assert rate == pytest.approx(2 * 4 * 1000 / 0.050 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.replica_rate(20.0, 1000, 2, 1, None)
    assert ms == 20.0 and rate == pytest.approx(2 * 1000 / 0.020 / 1e6)

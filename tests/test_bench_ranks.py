"""The multi-GPU path of bench.py is replicas with no collective on the data path: each
rank times its own events and the job time is the slowest rank.  Checked here with two
gloo ranks on the CPU (the aggregation is the only cross-rank step)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    elapsed = [100.0, 250.0][rank]  # rank 1 is the slow one
    dist.barrier()
    value, ms = bench.aggregate(elapsed, events_per_rank=320)
    q.put((rank, value, ms))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_aggregate_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, value, ms in res:
        assert ms == 250.0                      # max over ranks
        assert abs(value - 2 * 320 / 0.25) < 1e-6  # whole-job events / slowest rank's time


def test_single_process_aggregate():
    value, ms = bench.aggregate(50.0, 100)
    assert ms == 50.0 and abs(value - 2000.0) < 1e-9

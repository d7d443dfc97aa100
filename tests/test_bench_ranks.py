"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas) whose
local step times differ; both must report the slower rank's time and the
throughput of all ranks' cells together."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.whole_job(100.0 + 50.0 * rank, 1000, 10, world, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 150.0
        assert value == pytest.approx(world * 1000 * 10 / 0.150 / 1e6)


def test_single_rank_needs_no_collective():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    ms, value = bench.whole_job(20.0, 1000, 10, 1)
    assert ms == 20.0 and value == pytest.approx(1000 * 10 / 0.020 / 1e6)

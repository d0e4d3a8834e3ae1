"""Host logic of the multi-rank benchmark path on CPU (gloo, world size 2):
each rank times its own packing; rank 0 reports the iterations of all ranks
over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, iters = (1000.0, 500) if rank == 0 else (1500.0, 700)
    value, ms_max = bench.aggregate(ms, iters, world, dist, device="cpu")
    out[rank] = (value, ms_max)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        value, ms_max = out[r]
        assert ms_max == 1500.0
        assert value == pytest.approx((500 + 700) / 1.5)

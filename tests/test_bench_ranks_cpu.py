"""World-size-2 CPU check (gloo) of the benchmark's multi-process path.  The
library runs on one GPU per process with no data exchange: with N > 1 every
rank runs the whole workload as an independent replica, and the only
collectives are a barrier and the max over ranks of the timed region, which
is what sets the reported throughput (units of all ranks / slowest rank)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    t = bench.max_over_ranks(1.5 + rank, dist)        # each rank's own timed region
    np.save(os.path.join(out_dir, "tmax%d.npy" % rank), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_over_ranks(tmp_path):
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert float(np.load(tmp_path / ("tmax%d.npy" % r))[0]) == 2.5   # every rank sees the slowest


def test_max_over_ranks_without_a_process_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25

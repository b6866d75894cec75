"""World-size-2 CPU check of the sharded path (gloo): each rank integrates
its shard of orbits with its global orbit offset; the gathered shards equal
the unsharded run bit for bit, and the timing reduction is a max."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1908_03869_gb300.sharding import max_over_ranks, shard, weak_scaling_offset


def test_shard_arithmetic():
    for total in (1, 7, 1024, 1000003):
        for world in (1, 2, 3, 8):
            spans = [shard(total, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (o0, c0), (o1, _) in zip(spans, spans[1:]):
                assert o0 + c0 == o1
            assert sum(c for _, c in spans) == total
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    assert weak_scaling_offset(1 << 20, 3) == 3 << 20
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, total, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1908_03869_gb300 import inputs

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 6
    p, x0 = inputs.kuramoto(n, total, seed=3)
    off, cnt = shard(total, world, rank)
    pb = oracle.make_problem("kuramoto", n, n, n + 2, 0.01, 120, 40, 5)
    fr, xk = oracle.integrate(pb, p[off:off + cnt], x0[off:off + cnt], orbit_begin=off)
    parts = [None] * world
    dist.all_gather_object(parts, (off, xk))
    t = max_over_ranks(1.0 + rank, dist)
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.concatenate([x for _, x in sorted(parts, key=lambda a: a[0])]))
        np.save(os.path.join(out_dir, "tmax.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_equal_unsharded(tmp_path):
    import oracle
    from paper_1908_03869_gb300 import inputs

    total, world = 37, 2
    mp.spawn(_worker, args=(world, _free_port(), total, str(tmp_path)), nprocs=world, join=True)
    gathered = np.load(tmp_path / "gathered.npy")
    n = 6
    p, x0 = inputs.kuramoto(n, total, seed=3)
    pb = oracle.make_problem("kuramoto", n, n, n + 2, 0.01, 120, 40, 5)
    _, ref = oracle.integrate(pb, p, x0)
    np.testing.assert_array_equal(gathered, ref)
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 2.0

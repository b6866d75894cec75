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


def test_adjoint_error_report_against_the_oracle():
    """bench.py's adjoint error block on two orbits whose 'GPU' gradients are
    the oracle's own (error ~0) and then perturbed by 1e-2 of each orbit's
    largest component (error 1e-2, listed beyond 1e-3 with its one-ulp
    sensitivity)."""
    import bench
    import oracle
    from paper_1908_03869_gb300 import inputs

    W = inputs.WORKLOADS["kuramoto_adjoint_n32"]
    n, k = W["n"], 2
    p, x0 = inputs.kuramoto(n, W["orbits"], seed=1, shared=True)
    p32, x32 = p.astype(np.float32), x0[:k].astype(np.float32)
    pb = oracle.make_problem("kuramoto", n, n, n + 2, W["dt"], W["steps"], 1, W["seed"])
    dps = []
    for o in range(k):
        x = x32[o:o + 1].astype(np.float64)
        _, xK = oracle.integrate(pb, p32[None, :], x, orbit_begin=o, frames=False)
        _, dr = oracle.order_param(xK[0])
        dp, _ = oracle.adjoint(pb, p32[None, :], x, (dr / W["orbits"])[None, :], orbit_begin=o)
        dps.append(dp[0])
    a = {"p": p32, "x0": x32, "dp": np.array(dps), "W": W, "orbits": W["orbits"]}
    e = bench._adjoint_errors(a)
    assert e["orbits"] == k and e["max_rel_to_orbit_max"] < 1e-12 and e["over_1e-3"] == []
    assert len(e["oracle_one_ulp_sensitivity"]) == k and all(s > 0 for s in e["oracle_one_ulp_sensitivity"])
    a["dp"] = a["dp"] + 1e-2 * np.abs(a["dp"]).max(axis=1, keepdims=True)
    e = bench._adjoint_errors(a)
    assert abs(e["max_rel_to_orbit_max"] - 1e-2) < 1e-9
    assert [d["orbit"] for d in e["over_1e-3"]] == [0, 1]

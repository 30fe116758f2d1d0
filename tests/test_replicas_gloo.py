"""Host logic of the multi-GPU benchmark (replicas only: independent
trajectory batches per rank, no data-path collective) with two gloo ranks
on the CPU: the ranks hold consecutive slices of one seeded batch and draw
with its global trajectory ids (so N GPUs compute the trajectories one GPU
would), the job time is the maximum over ranks and the throughput sums the
ranks' trajectories."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [120.0, 150.0][rank]
    e2e_local = [1.5, 1.2][rank]
    agg = bench.aggregate(ms_local, e2e_local, 4096, 10, world, dist, "cpu")
    n = 6
    md, dt, x, p, occ, C = bench.replica_state(20, n, world, rank)
    mine = (bench.replica_traj_base(rank, n), x, p, occ, C)
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    out[rank] = (agg["ms"], agg["e2e_s"], agg["value"], parts)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import numpy as np
    _, _, x1, p1, occ1, C1 = bench.replica_state(20, 12, 1, 0)  # the job on one GPU
    for r in range(2):
        ms, e2e, value, parts = out[r]
        assert ms == 150.0 and e2e == 1.5
        assert value == pytest.approx(2 * 4096 * 10 / 0.150)
        assert [q[0] for q in parts] == [0, 6]  # global ids of each rank's first trajectory
        for whole, k in ((x1, 1), (p1, 2), (occ1, 3), (C1, 4)):
            assert np.array_equal(np.concatenate([q[k] for q in parts]), whole)


def test_single_rank_aggregation_of_host_time_only():
    """The end-to-end leg passes no device time: no throughput, no error."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    agg = bench.aggregate(0.0, 2.5, 4096, 10, 1)
    assert agg["e2e_s"] == 2.5 and agg["value"] is None
    agg = bench.aggregate(200.0, 0.0, 4096, 10, 1)
    assert agg["value"] == pytest.approx(4096 * 10 / 0.2)

"""Multi-GPU bench path on the CPU: two gloo ranks (replicas only).

The hot path does not shard: each rank runs an independent replica on its
own instance, and the whole-job figures are the slowest rank's time and the
sum of all ranks' candidates.  This checks that reduction and the per-rank
seeds with world_size 2 over gloo on 127.0.0.1.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, c = bench.reduce_replicas(1.5 + rank, 1000 * (rank + 1), "cpu")
        out[rank] = (t, c, bench.replica_seed(7, rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_whole_job():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:2] == res[1][:2] == (2.5, 3000.0)      # slowest rank, all candidates
    assert res[0][2] != res[1][2]                          # each rank descends its own instance


def test_single_process_is_the_identity():
    import bench
    assert bench.reduce_replicas(3.0, 42, "cpu") == (3.0, 42.0)

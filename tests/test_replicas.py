"""Multi-GPU runs are replicas (the step has no data exchange between simulations): each rank
steps its own simulation and the job's throughput is world * steps / (slowest rank's time).
The host-side aggregation is checked here with two gloo ranks on the CPU."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = 100.0 if rank == 0 else 250.0          # rank 1 is slower
    value, ms = bench.replica_throughput(ms_local, 10, dist, "cpu")
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    port = 29517
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        value, ms = out[r]
        assert ms == pytest.approx(250.0)
        assert value == pytest.approx(2 * 10 / 0.25)


def test_single_rank_throughput():
    import bench

    value, ms = bench.replica_throughput(50.0, 5, None)
    assert ms == 50.0 and value == pytest.approx(100.0)

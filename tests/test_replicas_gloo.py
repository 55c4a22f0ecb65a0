"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks, the
slowest rank's time and the whole-job throughput (atoms of all ranks x steps
/ that time)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [40.0, 50.0][rank]          # rank 1 is the slower one
    n_local = [1000, 3000][rank]
    ms, value = bench.replica_throughput(ms_local, n_local, 10, dist, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_summed_units():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        ms, value = out[r]
        assert ms == 50.0
        assert value == pytest.approx((1000 + 3000) * 10 / 0.050)


def test_single_process_is_the_local_figure():
    import bench
    ms, value = bench.replica_throughput(20.0, 500, 4)
    assert ms == 20.0 and value == pytest.approx(500 * 4 / 0.020)

"""The multi-rank timing logic of bench.py on CPU: two gloo ranks, each with
its own batch (weak scaling); the job's time is the slowest rank's."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [1.0 + rank, 5.0 - rank]
        got = bench.max_over_ranks(times, dist, "cpu")
        w = synth.medium(seed=bench.rank_workload_seed(rank), n_t=2)
        out[rank] = (got, float(w.l[0]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_own_batches():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert out[0][0] == [2.0, 5.0] and out[1][0] == [2.0, 5.0]
    assert out[0][1] != out[1][1]        # each rank has its own batch

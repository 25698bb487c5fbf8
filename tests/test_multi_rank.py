"""The multi-rank logic of bench.py on CPU, with two gloo ranks.

Each rank takes the contiguous block of hour angles of one batch that
synth.large(shard=(rank, world)) describes (the visibilities are time-major,
so a contiguous range of the batch's visibilities), keeps the whole
component list and predicts its own block. Checked: the job's time is the
slowest rank's; the ranks' blocks, concatenated in rank order, are the
one-rank batch bit for bit; and the concatenated predictions, computed here
by the oracle (Eq. 17) on each rank, equal the oracle's prediction of the
whole batch on one rank.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
J_TEST = 6          # a small tree: the oracle's Eq. 17 stays quick on 32 640 baselines per rank


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [1.0 + rank, 5.0 - rank]
        got = bench.max_over_ranks(times, dist, "cpu")
        w = synth.large(J=J_TEST, n_t=1, shard=(rank, world))
        v = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J_TEST).vis_eq17(w.uvw)
        parts = [None] * world
        dist.all_gather_object(parts, (w.uvw, v))
        out[rank] = (got, parts if rank == 0 else None)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_one_batch():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert out[0][0] == [2.0, 5.0] and out[1][0] == [2.0, 5.0]
    parts = out[0][1]
    import oracle as O
    import synth
    whole = synth.large(J=J_TEST, n_t=world)
    assert np.array_equal(np.concatenate([p[0] for p in parts]), whole.uvw)
    ref = O.Tree(whole.l, whole.m, whole.flux, whole.ra0, whole.dec0, J_TEST).vis_eq17(whole.uvw)
    assert np.array_equal(np.concatenate([p[1] for p in parts]), ref)


def test_shard_ranges_cover_the_batch_in_order():
    sys.path.insert(0, ROOT)
    import bench
    for n in (0, 1, 7, 1008000):
        for world in (1, 2, 3, 8):
            r = [bench.shard_range(n, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1

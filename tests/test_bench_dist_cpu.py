"""The multi-rank path of bench.py on CPU: two gloo ranks (one process per
GPU in a real run) each evaluate their own theta batch, meet at a barrier and
report the whole-job rate from the slowest rank's time (weak scaling, no
collective on the data path)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        th = bench.rank_thetas(r, 6)
        local_s = [0.25, 0.75][r]          # this rank's timed region
        dist.barrier()
        smax = bench.max_over_ranks(local_s, w)
        rate = bench.whole_job_rate(w, len(th), 3, smax)
        shards = [None] * w
        dist.all_gather_object(shards, th.tolist())
        q.put((r, w, local, smax, rate, shards))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_thetas_and_time_by_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for r, w, local, smax, rate, shards in res:
        assert (w, local) == (2, r)
        assert smax == 0.75                       # max over ranks, on every rank
        assert rate == pytest.approx(2 * 6 * 3 / 0.75)
        a, b = np.array(shards[0]), np.array(shards[1])
        assert a.shape == b.shape == (6, 4)
        assert not np.any(np.all(a[:, None, :] == b[None, :, :], axis=2))  # disjoint batches


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.whole_job_rate(1, 152, 3, 0.69) == pytest.approx(152 * 3 / 0.69)
    np.testing.assert_array_equal(bench.rank_thetas(0, 4), bench.rank_thetas(0, 4))

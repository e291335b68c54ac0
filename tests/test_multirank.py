"""The multi-GPU path of the benchmark on the host: two gloo ranks on CPU.

Each rank solves its own fields (weak scaling, no collective on the data
path); the only collectives are the barrier and the max over ranks of the
elapsed time. This checks the shard seeds, the max-over-ranks reduction and
the whole-job rate with world size 2, without a GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        B = 7
        seed = bench.rank_seed(rank, B)
        fields = list(range(seed, seed + B))
        ms = 10.0 + 5.0 * rank  # rank 1 is slower
        slowest = bench.max_over_ranks(ms, world)
        rate = bench.job_rate(B, world, 3, slowest)
        dist.barrier()
        q.put((rank, fields, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_time_like_the_benchmark():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, f0, s0, r0), (_, f1, s1, r1) = res
    assert not set(f0) & set(f1)  # disjoint fields
    assert s0 == s1 == 15.0  # both ranks see the slowest rank's time
    assert r0 == r1 == pytest.approx(7 * 2 * 3 / 0.015)

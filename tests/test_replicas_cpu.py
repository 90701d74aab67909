"""The multi-rank path of the bench (replicas only: a shard of pairs per rank, a barrier on both
sides of the timed region, the slowest rank's time) on two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    from paper_2203_00459_gb300 import replicas, synth
    world, r, _ = replicas.world()
    dist = replicas.init("gloo")
    first, count = replicas.shard(2, r)
    _, _, gt = synth.make_batch("single128", pairs=count, start=first)
    replicas.barrier(dist)
    ms = replicas.max_over_ranks(1.0 + 2.0 * r, dist)   # rank 1 is the slow one
    shards = [torch.zeros((count, 3), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(shards, torch.from_numpy(gt))
    replicas.barrier(dist)
    dist.destroy_process_group()
    out.put((r, world, ms, replicas.job_rate(world, count, ms), torch.cat(shards).numpy()))


def test_two_gloo_ranks_shard_pairs_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2203_00459_gb300 import synth
    _, _, whole = synth.make_batch("single128", pairs=4, start=0)
    for r, world, ms, rate, gathered in res:
        assert world == 2
        assert ms == 3.0                        # the slowest rank's time, on every rank
        assert rate == 2 * 2 / 3.0e-3           # all ranks' pairs over that time
        np.testing.assert_array_equal(gathered, whole)   # disjoint shards that tile the workload


def test_single_process_defaults():
    from paper_2203_00459_gb300 import replicas
    assert replicas.init("gloo") is None or replicas.world()[0] > 1
    assert replicas.max_over_ranks(2.5, None) == 2.5
    assert replicas.shard(32, 3) == (96, 32)

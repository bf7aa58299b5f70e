"""The multi-GPU path is replicas (independent solves per rank, no data-path collective): its
host logic — per-rank right-hand-side streams, index sharding of a batch, the max-over-ranks
reduction of the timed region and the whole-job rate — checked with two gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2205_09104_gb300 import replicas
    m = replicas.max_over_ranks(10.0 + 3.0 * rank)
    q.put((rank, m, list(replicas.shard(7, world, rank)), replicas.rhs_key((2, 0), rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [13.0, 13.0]             # max over ranks on every rank
    items = res[0][2] + res[1][2]
    assert sorted(items) == list(range(7)) and not set(res[0][2]) & set(res[1][2])
    assert res[0][3] != res[1][3]                          # disjoint right-hand-side streams


def test_rate_and_shards_single_process():
    from paper_2205_09104_gb300 import replicas
    assert replicas.max_over_ranks(4.5) == 4.5             # no process group: identity
    assert replicas.job_rate(10, 4, 200.0) == pytest.approx(200.0)
    for world in (1, 3, 8):
        got = [i for r in range(world) for i in replicas.shard(13, world, r)]
        assert got == list(range(13))

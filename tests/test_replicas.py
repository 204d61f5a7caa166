"""Multi-rank host logic of the replica runs, on CPU with the gloo backend
(world size 2): distinct noise keys per rank, job time = max over ranks, work
= sum over ranks."""
import os
import socket

import pytest

from paper_1410_5584_gb300.replicas import MASK64, aggregate, replica_seed


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = aggregate(1.0 + rank, 100.0 * (rank + 1))
        q.put((rank, t, u, replica_seed(7, rank)))
    finally:
        dist.destroy_process_group()


def test_replica_seeds_are_distinct():
    seeds = {replica_seed(1, r) for r in range(64)}
    assert len(seeds) == 64 and all(0 <= s <= MASK64 for s in seeds)
    assert replica_seed(1, 0) == 1


def test_aggregate_without_process_group_is_identity():
    assert aggregate(2.5, 10) == (2.5, 10.0)


def test_two_rank_gloo_aggregation():
    mp = pytest.importorskip("torch.multiprocessing")
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
    assert [r[1] for r in res] == [2.0, 2.0]      # max of 1.0 and 2.0
    assert [r[2] for r in res] == [300.0, 300.0]  # 100 + 200
    assert res[0][3] != res[1][3]

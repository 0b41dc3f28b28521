"""Replica sharding: host logic on CPU with a world_size-2 gloo group; chain-id stability
of split engines on the GPU."""
import os
import socket

import numpy as np
import pytest

from paper_1905_07440_gb300 import replicas


def test_shard_covers_all_chains_once():
    for total in (0, 1, 7, 256, 1000):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                first, n = replicas.shard(total, world, r)
                seen.extend(range(first, first + n))
            assert seen == list(range(total))
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, n = replicas.shard(10, world, rank)
        t = replicas.max_over_ranks(1.5 + rank)
        rows = replicas.gather_per_chain([f"chain{c}" for c in range(first, first + n)], first)
        q.put((rank, t, rows))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_max_and_gather():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rows in res:
        assert t == 2.5
        assert rows == [f"chain{c}" for c in range(10)]


@pytest.mark.gpu
def test_split_engines_reproduce_one_engine():
    """Chains [0, 3) and [3, 6) run as two engines equal chains [0, 6) of one engine."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_07440_gb300 as hq
    from workloads import HolsteinParams, initial_fields
    p = HolsteinParams(nx=4, ny=4, beta=2.0, delay_k=4)
    X0 = initial_fields(p, 6)
    whole = hq.Engine(p, 6)
    whole.set_fields(X0)
    whole.sweep(2)
    Xw = whole.get_fields()
    parts = []
    for rank in range(2):
        first, n = replicas.shard(6, 2, rank)
        e = hq.Engine(p, n, first_chain=first)
        e.set_fields(X0[first:first + n])
        e.sweep(2)
        parts.append(e.get_fields())
    assert np.array_equal(np.concatenate(parts), Xw)

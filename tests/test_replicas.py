"""Multi-process host logic on CPU: two gloo ranks (no GPU)."""
import os
import socket

import numpy as np
import pytest

from paper_1210_6412_gb300 import replicas


def test_shard_units_cover_everything_once():
    rng = np.random.default_rng(0)
    sizes = rng.integers(1, 1000, size=257)
    for world in (1, 2, 3, 8):
        seen = np.zeros(sizes.size, int)
        loads = []
        for r in range(world):
            a, b = replicas.shard_units(sizes, world, r)
            seen[a:b] += 1
            loads.append(sizes[a:b].sum())
        assert np.all(seen == 1)
        assert max(loads) - min(loads) <= 2 * sizes.max()
    assert replicas.shard_units([], 2, 1) == (0, 0)
    with pytest.raises(ValueError):
        replicas.shard_units(sizes, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = replicas.max_over_ranks(10.0 + rank)
        replicas.barrier()
        a, b = replicas.shard_units(np.arange(1, 11), world, rank)
        out.put((rank, mx, a, b))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_and_shards():
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
    assert [r[1] for r in res] == [11.0, 11.0]
    (_, _, a0, b0), (_, _, a1, b1) = res
    assert a0 == 0 and b0 == a1 and b1 == 10


def test_max_over_ranks_without_a_group():
    assert replicas.max_over_ranks(3.5) == 3.5

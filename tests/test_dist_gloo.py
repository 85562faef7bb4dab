"""Multi-process host logic with the gloo backend on CPU (world size 2)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2606_02053_gb300 import dist as D  # noqa: E402
from paper_2606_02053_gb300 import inputs  # noqa: E402


def test_shard_instances_is_a_balanced_partition():
    inst = inputs.scan_instances(64, seed=2606)
    sizes = [d["n"] ** 3 for d in inst]
    for world in (1, 2, 3, 4, 8):
        shards = D.shard_instances(sizes, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(64))
        loads = [sum(sizes[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(sizes)
    assert D.shard_instances([5, 3, 2], 2) == [[0], [1, 2]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = [1.5, 4.0][rank]
        mx = D.max_over_ranks(t)
        sm = D.sum_over_ranks(10.0 * (rank + 1))
        sizes = [d["n"] ** 3 for d in inputs.scan_instances(16, seed=7)]
        mine = D.shard_instances(sizes, world)[rank]
        total = D.sum_over_ranks(float(sum(sizes[i] for i in mine)))
        out.put((rank, mx, sm, total, float(sum(sizes))))
    finally:
        dist.destroy_process_group()


def test_reductions_and_sharding_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm, total, expect in res:
        assert mx == 4.0
        assert sm == 30.0
        assert total == expect


def test_single_process_reductions_are_identity():
    assert D.max_over_ranks(3.25) == 3.25
    assert D.sum_over_ranks(2.0) == 2.0

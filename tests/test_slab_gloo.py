"""The slab decomposition's host logic on CPU ranks (gloo): the plane split, the
ghost-plane exchange and the exponent reduction, against the single-domain
periodic layout.  The library's host calls size the slabs; no kernel runs.

* slab_bounds covers every plane once, each slab at least as deep as the ghosts;
* after DistExchange.ghosts on two and three ranks, every slab's ghost planes
  equal, bitwise, the whole grid's periodic neighbours of its own planes (each
  rank holds one slab of the same seeded whole-grid array);
* LocalExchange, all slabs in one process, gives the same ghost planes;
* DistExchange.exponents leaves every rank with the largest of the ranks' values.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2606_02053_gb300 import build  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_2606_02053_gb300 import cosmos

    build.build()
    return cosmos.lib()


N = (7, 5, 17)  # nx, ny, nz of the whole grid
H = (0.1, 0.1, 0.1)
X0 = (0.0, 0.0, 0.0)


def whole_grid(nf, pitch):
    rng = np.random.default_rng(11)
    return torch.from_numpy(rng.standard_normal((nf, N[2], N[1], pitch)))


def expected_ghosts(full, k0, k1):
    nz = full.shape[1]
    G = 3
    below = full[:, [(k0 - G + q) % nz for q in range(G)]]
    above = full[:, [(k1 + q) % nz for q in range(G)]]
    return below, above


def test_slab_bounds_cover_every_plane():
    from paper_2606_02053_gb300.slab import G, slab_bounds

    for nz, S in ((17, 2), (17, 3), (256, 8), (9, 3), (6, 1)):
        b = slab_bounds(nz, S)
        assert b[0][0] == 0 and b[-1][1] == nz
        assert all(b[j][1] == b[j + 1][0] for j in range(S - 1))
        assert all(k1 - k0 >= G for k0, k1 in b)
    with pytest.raises(ValueError):
        slab_bounds(8, 3)


def test_local_exchange_fills_ghosts_from_the_periodic_neighbours(lib):
    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.slab import LocalExchange, Slab, scatter, slab_bounds

    p = C.make_params(fluid=1)
    for S in (1, 2, 3):
        slabs = [Slab(N, H, X0, p, k0, k1, device="cpu", pitch=8) for k0, k1 in slab_bounds(N[2], S)]
        full = whole_grid(slabs[0].nf, 8)
        scatter(full, slabs)
        LocalExchange().ghosts(slabs, [s.state for s in slabs])
        for s in slabs:
            below, above = expected_ghosts(full, s.k0, s.k1)
            assert torch.equal(s.ghost_below(s.state), below)
            assert torch.equal(s.ghost_above(s.state), above)
            assert torch.equal(s.own(s.state), full[:, s.k0:s.k1])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2606_02053_gb300 import cosmos as C
        from paper_2606_02053_gb300.slab import DistExchange, Slab, slab_bounds

        p = C.make_params(fluid=1, scalar=1)
        k0, k1 = slab_bounds(N[2], world)[rank]
        s = Slab(N, H, X0, p, k0, k1, device="cpu", pitch=8)
        full = whole_grid(s.nf, 8)
        s.own(s.state).copy_(full[:, k0:k1])
        s.ghost_below(s.state).fill_(float("nan"))
        s.ghost_above(s.state).fill_(float("nan"))
        x = DistExchange()
        x.ghosts([s], [s.state])
        below, above = expected_ghosts(full, k0, k1)
        ok = torch.equal(s.ghost_below(s.state), below) and torch.equal(s.ghost_above(s.state), above)
        ok = ok and torch.equal(s.own(s.state), full[:, k0:k1])
        s.E.copy_(torch.arange(s.E.numel(), dtype=torch.int32) * (rank + 1) + 1000 * (rank % 2))
        x.exponents([s])
        a = torch.arange(s.E.numel(), dtype=torch.int32)
        want = a * 1
        for r in range(world):
            want = torch.maximum(want, a * (r + 1) + 1000 * (r % 2))
        ok = ok and torch.equal(s.E, want)
        q.put((rank, bool(ok)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_exchange_matches_the_single_domain_layout(lib, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
    assert res == {r: True for r in range(world)}

"""Slab decomposition of one periodic grid (z-slabs with ghost planes).

The sweep's only coupling between distant points is the stencil reach (3
points, the Kreiss-Oliger stencil), so a grid splits along z into slabs: slab
j owns planes [k0, k1) of the whole grid's nz planes and holds them with G = 3
ghost planes below and above, as an ordinary grid of k1 - k0 + 2G planes whose
point 0 lies G planes below its first own plane.  Before every RK4 stage:

1. the ghost planes of the stage state are refilled from the neighbouring
   slabs' own planes (periodic in z across the slabs);
2. every slab's per-field reference exponent of the integer derivative pass
   (cosmos_field_exponents) is replaced by the largest over all slabs, so that
   each slab rounds its derivatives exactly as the whole grid does;
3. cosmos_rk4_stage_slab advances the slab's own planes (the algebra pass and
   the stage combine on them only; the derivative and fluid passes read the
   ghost planes).

The own planes then equal those of cosmos_rk4_step on the whole grid bitwise.
Two exchangers move the planes:

* ``LocalExchange``: every slab in this process (device-to-device copies),
  e.g. several slabs on one GPU;
* ``DistExchange``: one slab per rank of torch.distributed, point-to-point
  sends of the packed planes to the two neighbours and an all-reduce (MAX) of
  the exponents (NCCL between GPUs, gloo between CPU processes).

Marshalling only: all arithmetic runs in the library's kernels.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch

from . import cosmos as C

G = 3  # ghost planes on each side: the reach of the widest stencil


def slab_bounds(nz: int, nslabs: int) -> List[Tuple[int, int]]:
    """Planes [k0, k1) of each slab: nz split as evenly as integers allow."""
    if nslabs < 1 or nz < G * nslabs:
        raise ValueError(f"{nslabs} slabs of at least {G} planes do not fit in {nz} planes")
    return [(nz * j // nslabs, nz * (j + 1) // nslabs) for j in range(nslabs)]


class Slab:
    """One slab's grid, buffers and views (all planes of a field are contiguous)."""

    def __init__(self, n: Sequence[int], h: Sequence[float], x0: Sequence[float], params, k0: int, k1: int,
                 device="cuda", pitch=None):
        nx, ny, nz = (int(v) for v in n)
        self.k0, self.k1, self.nloc = k0, k1, k1 - k0
        self.p = params
        self.g = C.make_grid((nx, ny, self.nloc + 2 * G), tuple(h), x0=(x0[0], x0[1], x0[2] + (k0 - G) * h[2]),
                             pitch=pitch)
        self.nf = C.cosmos_nfields(params)
        self.fs = C.cosmos_field_stride(self.g)
        self.shape = (self.nf, self.nloc + 2 * G, ny, self.g.pitch)
        f64 = torch.float64
        self.state = torch.zeros(self.nf * self.fs, dtype=f64, device=device)
        self.A = torch.zeros_like(self.state)
        self.B = torch.zeros_like(self.state)
        self.acc = torch.zeros_like(self.state)
        nb = C.cosmos_workspace_bytes(self.g, params, C.COSMOS_OP_RHS)
        self.ws = torch.empty((nb + 7) // 8, dtype=f64, device=device)
        self.E = torch.zeros(24 + 2 * int(params.scalar), dtype=torch.int32, device=device)

    def view(self, t: torch.Tensor) -> torch.Tensor:
        return t.view(self.shape)

    def own(self, t):
        return self.view(t)[:, G:G + self.nloc]

    def bottom_own(self, t):  # first G own planes: the lower neighbour's upper ghosts
        return self.view(t)[:, G:2 * G]

    def top_own(self, t):  # last G own planes: the upper neighbour's lower ghosts
        return self.view(t)[:, self.nloc:self.nloc + G]

    def ghost_below(self, t):
        return self.view(t)[:, 0:G]

    def ghost_above(self, t):
        return self.view(t)[:, G + self.nloc:2 * G + self.nloc]


class LocalExchange:
    """Ghost planes and exponents among slabs that all live in this process."""

    def ghosts(self, slabs: List[Slab], bufs: List[torch.Tensor]):
        S = len(slabs)
        for j in range(S):
            lo, up = (j - 1) % S, (j + 1) % S
            slabs[j].ghost_below(bufs[j]).copy_(slabs[lo].top_own(bufs[lo]))
            slabs[j].ghost_above(bufs[j]).copy_(slabs[up].bottom_own(bufs[up]))

    def exponents(self, slabs: List[Slab]):
        m = slabs[0].E.clone()
        for s in slabs[1:]:
            m = torch.maximum(m, s.E)
        for s in slabs:
            s.E.copy_(m)


class DistExchange:
    """One slab per rank of the default torch.distributed group.

    Every rank posts, in this order: its top own planes to the upper rank, its
    bottom own planes to the lower rank, then receives its lower ghosts from the
    lower rank and its upper ghosts from the upper rank.  With two ranks both
    neighbours are the same rank and the two messages each way are told apart
    by that order (NCCL has no message tags)."""

    def __init__(self):
        import torch.distributed as dist

        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()

    def ghosts(self, slabs: List[Slab], bufs: List[torch.Tensor]):
        (s,), (b,) = slabs, bufs
        if self.world == 1:
            return LocalExchange().ghosts(slabs, bufs)
        up, lo = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        top = s.top_own(b).contiguous()
        bot = s.bottom_own(b).contiguous()
        below = torch.empty_like(top)
        above = torch.empty_like(bot)
        P2P = self.dist.P2POp
        ops = [P2P(self.dist.isend, top, up), P2P(self.dist.isend, bot, lo),
               P2P(self.dist.irecv, below, lo), P2P(self.dist.irecv, above, up)]
        for r in self.dist.batch_isend_irecv(ops):
            r.wait()
        s.ghost_below(b).copy_(below)
        s.ghost_above(b).copy_(above)

    def exponents(self, slabs: List[Slab]):
        (s,) = slabs
        if self.world > 1:
            self.dist.all_reduce(s.E, op=self.dist.ReduceOp.MAX)


class SlabEvolution:
    """RK4 steps of a grid held as slabs (all of them here, or this rank's one)."""

    def __init__(self, slabs: List[Slab], exchange):
        self.slabs = slabs
        self.x = exchange

    def _stage(self, stage: int, src: str, dst: str, t: float, dt: float):
        S = self.slabs
        self.x.ghosts(S, [getattr(s, src) for s in S])
        for s in S:
            C.check(C.cosmos_field_exponents(s.g, s.p, getattr(s, src), s.E))
        self.x.exponents(S)
        for s in S:
            U_next = getattr(s, dst) if dst else None
            C.check(C.cosmos_rk4_stage_slab(s.g, s.p, stage, getattr(s, src), s.state, U_next, s.acc, t, dt, G,
                                            s.nloc, s.E, s.ws))

    def step(self, t: float, dt: float, steps: int = 1):
        """In place on every slab's own planes: as cosmos_rk4_step on the whole grid."""
        for k in range(steps):
            tk = t + k * dt
            self._stage(1, "state", "A", tk, dt)
            self._stage(2, "A", "B", tk, dt)
            self._stage(3, "B", "A", tk, dt)
            self._stage(4, "A", None, tk, dt)


def scatter(full: torch.Tensor, slabs: List[Slab]):
    """Own planes of every slab from a whole-grid state [nf, nz, ny, pitch]."""
    for s in slabs:
        s.own(s.state).copy_(full[:, s.k0:s.k1])


def gather(slabs: List[Slab], out: torch.Tensor):
    """Whole-grid state [nf, nz, ny, pitch] from every slab's own planes."""
    for s in slabs:
        out[:, s.k0:s.k1].copy_(s.own(s.state))
    return out

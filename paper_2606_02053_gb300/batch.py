"""Batched threshold scan: many uneven grids evolved together.

``BatchScan`` owns the instance states and the batch workspace (torch
tensors) and drives the C ABI batch calls (``cosmos_batch_*``).
``autotune`` calls the library's autotuner (``cosmos_batch_autotune``): it
times the candidate work-list mappings / launch shapes and keeps the fastest,
with an optional cache file keyed by the GPU name, the matter model and the
grid sizes.
"""
from __future__ import annotations

import torch

from . import cosmos as C

# The library's built-in candidate tunings: (mapping, block_x, block_y, blocks_per_sm)
CANDIDATES = [(0, 32, 4, 3), (0, 16, 8, 3), (0, 64, 2, 3), (0, 8, 16, 3), (1, 32, 4, 3), (1, 32, 4, 2),
              (0, 32, 4, 2), (1, 32, 4, 1)]


def as_tuple(t) -> tuple:
    return (t.mapping, t.block_x, t.block_y, t.blocks_per_sm)


def tuning(t) -> C.cosmos_batch_tuning:
    x = C.cosmos_batch_tuning()
    x.mapping, x.block_x, x.block_y, x.blocks_per_sm = t
    return x


class BatchScan:
    def __init__(self, grids, params, dts, t0s=None, max_steps=1, device="cuda", tune=None):
        self.grids = list(grids)
        self.p = params
        self.n = len(self.grids)
        self.device = torch.device(device)
        self.nf = C.cosmos_nfields(params)
        self.dts = list(dts)
        self.t0s = list(t0s) if t0s is not None else [0.0] * self.n
        self.states = [torch.zeros(self.nf * C.cosmos_field_stride(g), dtype=torch.float64, device=self.device)
                       for g in self.grids]
        nb = C.cosmos_batch_workspace_bytes(self.grids, params, max_steps)
        if nb == 0:
            raise C.CosmosError("invalid batch description")
        self.ws = torch.empty((nb + 7) // 8, dtype=torch.float64, device=self.device)
        self.max_steps = max_steps
        code, self.plan = C.cosmos_batch_plan(self.grids, params, self.dts, self.t0s, self.states, max_steps,
                                              None if tune is None else tuning(tune), self.ws)
        C.check(code)
        self.tune = tune if tune is not None else CANDIDATES[0]

    def init(self, idents, ws_init=None):
        """Initial data per instance through cosmos_init_grid."""
        for g, st, ident in zip(self.grids, self.states, idents):
            nb = C.cosmos_workspace_bytes(g, self.p, C.COSMOS_OP_INIT)
            ws = torch.empty((nb + 7) // 8, dtype=torch.float64, device=self.device) if nb else None
            C.check(C.cosmos_init_grid(g, self.p, ident, st, ws))

    def set_tuning(self, t):
        C.check(C.cosmos_batch_set_tuning(self.plan, tuning(t)))
        self.tune = tuple(t)

    def run(self, first_step, steps, use_graph=True, stream=None):
        """Advance every instance; work queued on the current stream (initial
        data, copies) is ordered before the run when another stream is given."""
        cur = torch.cuda.current_stream()
        if stream is None:
            stream = cur
        elif stream != cur:
            stream.wait_stream(cur)
        C.check(C.cosmos_batch_run(self.plan, first_step, steps, 1 if use_graph else 0, stream))

    def time_stage(self, reps=3):
        code, ms = C.cosmos_batch_time_stage(self.plan, reps)
        C.check(code)
        return ms

    def autotune(self, candidates=None, reps=3, cache_path=None):
        """Runs the library's autotuner; candidates = None takes its built-in list.
        Returns {"best": [...], "ms": {candidate: ms}, "cache_hit": bool} (no
        timings on a cache hit)."""
        cands = [tuning(c) for c in candidates] if candidates else []
        code, best, ms, hit = C.cosmos_batch_autotune(self.plan, cands, reps, cache_path)
        C.check(code)
        self.tune = as_tuple(best)
        names = [as_tuple(c) for c in (cands or C.cosmos_batch_default_candidates())]
        return {"best": list(self.tune), "ms": {} if hit else {str(list(k)): v for k, v in zip(names, ms)},
                "cache_hit": hit}

    def close(self):
        if self.plan:
            C.cosmos_batch_free(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

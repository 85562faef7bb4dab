"""Torch-level holder of a fixed-mesh-refinement hierarchy (see the
``cosmos_fmr_*`` calls of include/cosmos.h): one device state per level and
the hierarchy workspace.  Buffers and layout copies only; every step of the
computation runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import cosmos as C


class Hierarchy:
    def __init__(self, levels, params: C.cosmos_params, pitch_align=1, device="cuda"):
        self.levels = levels
        self.m = C.make_fmr(levels, pitch_align)
        self.p = params
        self.device = torch.device(device)
        self.nf = C.cosmos_nfields(params)
        nbytes = C.cosmos_fmr_workspace_bytes(self.m, params)
        if nbytes == 0:
            raise C.CosmosError("invalid refinement hierarchy")
        self.ws = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=self.device)
        self.fs = [C.cosmos_field_stride(self.m.grid[l]) for l in range(len(levels))]
        self.states = [torch.zeros(self.nf * fs, dtype=torch.float64, device=self.device) for fs in self.fs]

    @property
    def L(self):
        return len(self.levels)

    def grid(self, l):
        return self.m.grid[l]

    def view(self, l, flat=None):
        g = self.m.grid[l]
        flat = self.states[l] if flat is None else flat
        return flat.view(-1, g.nz, g.ny, g.pitch)

    def get(self, l, flat=None) -> np.ndarray:
        g = self.m.grid[l]
        return self.view(l, flat)[..., : g.nx].cpu().numpy().copy()

    def set(self, l, arr, flat=None):
        g = self.m.grid[l]
        self.view(l, flat)[..., : g.nx] = torch.from_numpy(np.ascontiguousarray(arr)).to(self.device)

    def init(self, ident: C.cosmos_id):
        C.check(C.cosmos_fmr_init(self.m, self.p, ident, self.states, self.ws))

    def step(self, t, dt0, steps=1):
        for n in range(steps):
            C.check(C.cosmos_fmr_step(self.m, self.p, self.states, t + n * dt0, dt0, self.ws))

    def prolong(self, level, parent, child):
        C.check(C.cosmos_fmr_prolong(self.m, self.p, level, parent, child, self.ws))

    def restrict(self, level, child, parent):
        C.check(C.cosmos_fmr_restrict(self.m, self.p, level, child, parent))

    def interior_points(self, l) -> int:
        lv = self.levels[l]
        return int(np.prod([lv["hi"][d] - lv["lo"][d] for d in range(3)]))

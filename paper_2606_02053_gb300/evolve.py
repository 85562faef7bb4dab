"""Torch-level helpers around the C ABI: device buffers, workspaces, layout.

``Evolution`` owns the device state and the workspaces of one grid and calls
the library through the ctypes binding; nothing here computes any part of
the method.  Host arrays use the unpadded layout [nf, nz, ny, nx]; device
state uses the library layout with a row pitch (see include/cosmos.h).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import cosmos as C


def _alloc_ws(nbytes: int, device):
    if nbytes == 0:
        return None
    # float64 elements; torch's caching allocator returns >= 512-byte aligned blocks
    return torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=device)


class Evolution:
    def __init__(self, grid: C.cosmos_grid, params: C.cosmos_params, device="cuda"):
        self.g = grid
        self.p = params
        self.device = torch.device(device)
        self.nf = C.cosmos_nfields(params)
        self.fs = C.cosmos_field_stride(grid)
        self.state = torch.zeros(self.nf * self.fs, dtype=torch.float64, device=self.device)
        self.ws_rk4 = _alloc_ws(C.cosmos_workspace_bytes(grid, params, C.COSMOS_OP_RK4), self.device)
        self.ws_rhs = _alloc_ws(C.cosmos_workspace_bytes(grid, params, C.COSMOS_OP_RHS), self.device)
        self.ws_con = _alloc_ws(C.cosmos_workspace_bytes(grid, params, C.COSMOS_OP_CONSTRAINTS), self.device)
        self.ws_init = _alloc_ws(C.cosmos_workspace_bytes(grid, params, C.COSMOS_OP_INIT), self.device)

    # ---- layout conversion (host <-> device copies only) ----
    def view(self, flat=None):
        """[nf, nz, ny, pitch] view of a flat device buffer."""
        flat = self.state if flat is None else flat
        return flat.view(-1, self.g.nz, self.g.ny, self.g.pitch)

    def set_state(self, arr: np.ndarray):
        v = self.view()
        v[..., : self.g.nx] = torch.from_numpy(np.ascontiguousarray(arr)).to(self.device)

    def get(self, flat=None) -> np.ndarray:
        return self.view(flat)[..., : self.g.nx].cpu().numpy().copy()

    # ---- library calls ----
    def init(self, ident: C.cosmos_id):
        C.check(C.cosmos_init_grid(self.g, self.p, ident, self.state, self.ws_init))

    def rhs(self, t=0.0, out=None):
        out = torch.empty_like(self.state) if out is None else out
        C.check(C.cosmos_rhs(self.g, self.p, self.state, out, t, self.ws_rhs))
        return out

    def step(self, t, dt, steps=1):
        for n in range(steps):
            C.check(C.cosmos_rk4_step(self.g, self.p, self.state, t + n * dt, dt, self.ws_rk4))

    def save(self, path, t, step):
        """Checkpoint of the current state (cosmos_checkpoint_save)."""
        C.check(C.cosmos_checkpoint_save(path, self.g, self.p, self.state, t, step))

    def load(self, path):
        """Resume from a checkpoint of this grid and these parameters; returns (t, step)."""
        code, t, step = C.cosmos_checkpoint_load(path, self.g, self.p, self.state)
        C.check(code)
        return t, step

    def scan(self):
        """Failure detection on the current state: {field: count} of NaN/Inf
        values (and, fluid on, of tau~ <= 0); empty when the state is sound."""
        ws = _alloc_ws(C.cosmos_workspace_bytes(self.g, self.p, C.COSMOS_OP_SCAN), self.device)
        code, counts = C.cosmos_scan_state(self.g, self.p, self.state, ws)
        if code not in (C.COSMOS_OK, C.COSMOS_ENONFINITE):
            C.check(code)
        return {f: c for f, c in enumerate(counts) if c}

    def constraints(self, want_fields=False):
        hm = torch.empty(4 * self.fs, dtype=torch.float64, device=self.device) if want_fields else None
        norms = (ctypes.c_double * 8)()
        C.check(C.cosmos_constraints(self.g, self.p, self.state, hm, norms, self.ws_con))
        return (self.view(hm)[..., : self.g.nx].cpu().numpy() if want_fields else None), np.array(list(norms))

"""Gradients of collapse diagnostics with respect to the initial curvature
perturbation, by the hand-written (generated) adjoint of the RK4 BSSN step.

``CollapseRun`` fixes the problem: one periodic grid, FLRW background with a
radiation fluid, initial data from a per-point curvature perturbation zeta
(cosmos_init_zeta), ``steps`` RK4 steps of size dt, checkpoints every
``checkpoint_every`` steps.  Diagnostics (definitions in include/cosmos.h):

* minimum central lapse  min_n alpha(centre, t_n), n = 0 .. steps
  (the gradient follows the first step attaining the minimum);
* peak compaction  max_k C(r_k) at the final time (gradient through the
  maximising shell).

``CosmosAdjoint`` (a torch.autograd.Function) maps zeta -> (min lapse, peak
compaction); its backward replays each checkpoint segment forward, stores the
segment's time levels and their RK4 stage states (cosmos_rk4_step_stages), and
runs cosmos_adjoint_step_stages backwards through them,
injecting the diagnostics' cotangents at the step they were measured, then
cosmos_init_zeta_vjp.  zeta = mu * profile built with torch gives d/d mu by
ordinary autograd.  ``CollapseRun.backward_many`` gives the zeta gradients of
several cotangent pairs (e.g. each diagnostic on its own) in one reverse sweep
that replays each checkpoint segment once for all of them.
"""
from __future__ import annotations

import torch

from . import cosmos as C

def _ws(nbytes, device):
    return torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=device) if nbytes else None


class CollapseRun:
    def __init__(self, n, params, dt, steps, checkpoint_every=16, kmax=None, a0=1.0, device="cuda"):
        h = 1.0 / n
        self.n = n
        self.g = C.make_grid(n, h, x0=(-(n // 2) * h,) * 3)
        self.p = params
        self.dt = dt
        self.steps = steps
        self.every = checkpoint_every
        self.kmax = kmax if kmax is not None else n // 2 - 1
        self.a0 = a0
        self.device = torch.device(device)
        self.nf = C.cosmos_nfields(params)
        self.fs = C.cosmos_field_stride(self.g)
        dev = self.device
        self.ws_rk4 = _ws(C.cosmos_workspace_bytes(self.g, params, C.COSMOS_OP_RK4), dev)
        self.ws_init = _ws(C.cosmos_workspace_bytes(self.g, params, C.COSMOS_OP_INIT), dev)
        self.ws_adj = _ws(C.cosmos_adjoint_workspace_bytes(self.g, params, C.COSMOS_OP_ADJOINT), dev)
        self.ws_ivjp = _ws(C.cosmos_adjoint_workspace_bytes(self.g, params, C.COSMOS_OP_INIT_VJP), dev)
        self.ws_diag = _ws(C.cosmos_adjoint_workspace_bytes(self.g, params, C.COSMOS_OP_DIAG), dev)

    def new_state(self):
        return torch.empty(self.nf * self.fs, dtype=torch.float64, device=self.device)

    def init(self, zeta, state):
        C.check(C.cosmos_init_zeta(self.g, self.p, zeta, self.a0, state, self.ws_init))

    def step(self, state, n):
        C.check(C.cosmos_rk4_step(self.g, self.p, state, n * self.dt, self.dt, self.ws_rk4))

    def compaction(self, state):
        code, Ck, aux = C.cosmos_compaction(self.g, self.p, state, self.kmax, self.ws_diag)
        C.check(code)
        return Ck, aux

    def forward(self, zeta):
        """Returns (min central lapse, peak compaction, record for backward)."""
        U = self.new_state()
        self.init(zeta, U)
        U0 = U.clone()
        alphas = torch.empty(self.steps + 1, dtype=torch.float64, device=self.device)
        C.check(C.cosmos_central_lapse(self.g, self.p, U, alphas, 0))
        checkpoints = {0: U.clone()}
        for s in range(self.steps):
            self.step(U, s)
            C.check(C.cosmos_central_lapse(self.g, self.p, U, alphas, s + 1))
            if (s + 1) % self.every == 0 and s + 1 < self.steps:
                checkpoints[s + 1] = U.clone()
        res = torch.empty(2, dtype=torch.float64, device=self.device)
        C.check(C.cosmos_series_argmin(alphas, self.steps + 1, res))
        amin, nstar = res.cpu().tolist()
        nstar = int(nstar)
        Ck, aux = self.compaction(U)
        kstar = max(range(len(Ck)), key=lambda k: Ck[k]) + 1  # first maximising radius (host values)
        rec = dict(U0=U0, final=U, checkpoints=checkpoints, nstar=nstar, kstar=kstar, aux=aux, alphas=alphas)
        return amin, float(Ck[kstar - 1]), rec

    def backward(self, rec, gbar_alpha, gbar_comp):
        """zeta_bar for the cotangents of (min lapse, peak compaction)."""
        return self.backward_many(rec, [(gbar_alpha, gbar_comp)])[0]

    def backward_many(self, rec, seeds):
        """zeta_bar for each pair (gbar_alpha, gbar_comp) in `seeds`, in one reverse sweep:
        every checkpoint segment is replayed forward once, and each step's adjoint runs
        for every pair on the same replayed stage states."""
        lams = []
        for ga, gc in seeds:
            lam = self.new_state()
            C.check(C.cosmos_compaction_vjp(self.g, self.p, rec["final"], rec["kstar"], self.kmax, rec["aux"],
                                            float(gc), lam))
            if rec["nstar"] == self.steps:
                C.check(C.cosmos_central_lapse_vjp(self.g, self.p, float(ga), lam))
            lams.append(lam)
        starts = sorted(rec["checkpoints"].keys())
        for si in reversed(range(len(starts))):
            s0 = starts[si]
            s1 = starts[si + 1] if si + 1 < len(starts) else self.steps
            # replay the segment, keeping every step's level and its three stage states
            U = rec["checkpoints"][s0].clone()
            saved = []
            for s in range(s0, s1):
                stages = [self.new_state() for _ in range(3)]
                saved.append((U.clone(), stages))
                C.check(C.cosmos_rk4_step_stages(self.g, self.p, U, s * self.dt, self.dt, *stages, self.ws_rk4))
            for s in reversed(range(s0, s1)):
                Un, (U2, U3, U4) = saved[s - s0]
                for lam, (ga, _) in zip(lams, seeds):
                    C.check(C.cosmos_adjoint_step_stages(self.g, self.p, Un, U2, U3, U4, lam, lam, s * self.dt,
                                                         self.dt, self.ws_adj))
                    if s == rec["nstar"]:
                        C.check(C.cosmos_central_lapse_vjp(self.g, self.p, float(ga), lam))
            del saved
        zbars = []
        for lam in lams:
            zbar = torch.empty(self.fs, dtype=torch.float64, device=self.device)
            C.check(C.cosmos_init_zeta_vjp(self.g, self.p, rec["U0"], lam, zbar, self.ws_ivjp))
            zbars.append(zbar)
        return zbars


class CosmosAdjoint(torch.autograd.Function):
    """(min central lapse, peak compaction) = f(zeta); backward by the adjoint."""

    @staticmethod
    def forward(ctx, zeta, run: CollapseRun):
        amin, cpeak, rec = run.forward(zeta.detach().contiguous())
        ctx.run = run
        ctx.rec = rec
        return torch.tensor([amin, cpeak], dtype=torch.float64, device=zeta.device)

    @staticmethod
    def backward(ctx, gout):
        g = gout.detach().cpu()
        zbar = ctx.run.backward(ctx.rec, float(g[0]), float(g[1]))
        return zbar, None

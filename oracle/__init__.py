"""CPU FP64 oracle for the COSMOS evolution problem — test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product package
(``paper_2606_02053_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``cosmos_oracle.cpp`` (plain C++17, FP64, compiled
with ``-ffp-contract=off``).  This module compiles it with g++ on first use,
loads it with ctypes and exposes numpy-level wrappers.  Arrays follow the
oracle's own layout: ``state[f, k, j, i]`` (i fastest), C-contiguous float64.

Parity status per function (what pins it, see ``tests/test_oracle_*.py``):
  rhs / rhs_points / rk4_step : flat space, Fourier symbols, translation and
      axis permutation, gauge-wave closed form + 4th-order convergence, ADM
      cross-check against an autodiff evaluation of the Einstein equations
      (vacuum, fluid, scalar), homogeneous FLRW expansion law.
  constraints : autodiff ADM constraints (4th-order convergence), gauge wave.
  init        : gauge-wave closed form; FLRW + zeta gives H = 0 (discrete);
      next-to-leading-order data (kind 3): the right-hand side at t = 0 meets
      the growing-mode rates of K, At and gt to O(eps^4) (16-fold per doubling
      of H0; 4-fold for the leading-order data or a wrong coefficient), H = 0,
      M = 0, and the data reduce to the leading order as eps -> 0.
  flop_count  : counts only; no physics.
  fluid_rho   : round trip (rho, v) -> (E, J) -> rho against the definitions.
  rhs_vjp / adjoint_step : tape reverse mode of rhs / rk4_step; pinned by
      finite-difference dot-product tests against the (pinned) forward map.
  init_zeta / compaction / central_lapse (collapse diagnostics): the zeta map
      equals the Gaussian initial data when given the Gaussian's values and
      leaves H = 0, M = 0; compaction is 0 for a homogeneous state and equals
      the closed form 2 dM / R of a top-hat overdensity (lattice counts by
      brute force); the areal radius uses exactly the six axis points.
  init_zeta_vjp / compaction_vjp / collapse_gradient : tapes over the same
      functions, pinned by finite-difference dot-product tests; the whole
      pipeline zeta -> (min central lapse, peak compaction) against central
      differences along the amplitude mu.
  fmr_* (fixed mesh refinement) : prolongation exact for degree-5
      polynomials and not for degree 6; injection against its definition;
      the RK4 continuous extension against quadrature and linear-ODE closed
      forms; the gauge wave on three levels converges at 4th order; an
      independent copy of the scheme written in the test agrees with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cosmos_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CXXFLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++); returns its path."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", *CXXFLAGS, "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_L = ctypes.POINTER(ctypes.c_long)


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.oracle_nfields.argtypes = [_D]
        L.oracle_nfields.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        L.oracle_rhs.argtypes = [_I, _D, _D, _D, _D, ctypes.c_double, _D]
        L.oracle_rhs_points.argtypes = [_I, _D, _D, _D, _D, ctypes.c_double, ctypes.c_long, _L, _D]
        L.oracle_rhs_planes.argtypes = [_I, _D, _D, _D, _D, ctypes.c_double, ctypes.c_long, ctypes.c_long, _D]
        L.oracle_rk4_step.argtypes = [_I, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double]
        L.oracle_constraints.argtypes = [_I, _D, _D, _D, _D, _D, _D]
        L.oracle_init.argtypes = [_I, _D, _D, _D, _D, _D]
        L.oracle_flop_count.argtypes = [_I, _D, _D, _D, _D, ctypes.c_double, _D]
        L.oracle_rhs_vjp.argtypes = [_I, _D, _D, _D, _D, ctypes.c_double, _D, _D]
        L.oracle_flop_count_parts.argtypes = [_I, _D, _D, _D, _D, ctypes.c_double, _D]
        L.oracle_fluid_rho.argtypes = [_D, _D, ctypes.c_long, ctypes.c_double, _D]
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# Parameter containers (plain data)
# --------------------------------------------------------------------------
class OGrid:
    """Uniform periodic grid: n = (nx, ny, nz), spacing h, coordinate x0 of point 0."""

    def __init__(self, n, h, x0=(0.0, 0.0, 0.0)):
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in (h if np.ndim(h) else (h, h, h)))
        self.x0 = tuple(float(v) for v in x0)

    @property
    def npts(self):
        return self.n[0] * self.n[1] * self.n[2]

    def c(self):
        return ((ctypes.c_int * 3)(*self.n), (ctypes.c_double * 3)(*self.h), (ctypes.c_double * 3)(*self.x0))


def params_array(slicing=0, shift=1, eta=2.0, ko_sigma=0.1, w=1.0 / 3.0, fluid=0, scalar=0, H0=0.0, t0=0.0):
    return np.array([slicing, shift, eta, ko_sigma, w, fluid, scalar, H0, t0], dtype=np.float64)


def nfields(params) -> int:
    return 24 + 4 * int(params[5]) + 2 * int(params[6])


def _dp(a):
    return a.ctypes.data_as(_D)


def _check_state(g: OGrid, params, state):
    nf = nfields(params)
    assert state.dtype == np.float64 and state.flags.c_contiguous
    assert state.shape == (nf, g.n[2], g.n[1], g.n[0]), (state.shape, nf, g.n)


def set_threads(n: int):
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def rhs(g: OGrid, params, state, t=0.0):
    _check_state(g, params, state)
    out = np.empty_like(state)
    n, h, x0 = g.c()
    lib().oracle_rhs(n, h, x0, _dp(params), _dp(state), float(t), _dp(out))
    return out


def rhs_points(g: OGrid, params, state, pts, t=0.0):
    """RHS at (i, j, k) points; returns array [npts, nf]."""
    _check_state(g, params, state)
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.int64).reshape(-1, 3))
    out = np.empty((pts.shape[0], nfields(params)), dtype=np.float64)
    n, h, x0 = g.c()
    lib().oracle_rhs_points(n, h, x0, _dp(params), _dp(state), float(t), pts.shape[0],
                            pts.ctypes.data_as(_L), _dp(out))
    return out


def rhs_planes(g: OGrid, params, state, k0, k1, t=0.0):
    _check_state(g, params, state)
    out = np.empty((nfields(params), k1 - k0, g.n[1], g.n[0]), dtype=np.float64)
    n, h, x0 = g.c()
    lib().oracle_rhs_planes(n, h, x0, _dp(params), _dp(state), float(t), int(k0), int(k1), _dp(out))
    return out


def rk4_step(g: OGrid, params, state, t, dt):
    """In place: state <- RK4 step of size dt from time t."""
    _check_state(g, params, state)
    n, h, x0 = g.c()
    lib().oracle_rk4_step(n, h, x0, _dp(params), _dp(state), float(t), float(dt))
    return state


def evolve(g: OGrid, params, state, t, dt, steps):
    for s in range(steps):
        rk4_step(g, params, state, t + s * dt, dt)
    return state


def constraints(g: OGrid, params, state):
    """Returns (ham_mom[4, nz, ny, nx], norms[8])."""
    _check_state(g, params, state)
    hm = np.empty((4, g.n[2], g.n[1], g.n[0]), dtype=np.float64)
    norms = np.empty(8, dtype=np.float64)
    n, h, x0 = g.c()
    lib().oracle_constraints(n, h, x0, _dp(params), _dp(state), _dp(hm), _dp(norms))
    return hm, norms


def id_array(kind, A=0.0, mu=0.0, sigma=0.125, q=(1.0, 1.0, 1.0), center=(0.0, 0.0, 0.0), a0=1.0, t=0.0):
    return np.array([kind, A, mu, sigma, *q, *center, a0, t], dtype=np.float64)


def init(g: OGrid, params, idarr):
    state = np.empty((nfields(params), g.n[2], g.n[1], g.n[0]), dtype=np.float64)
    n, h, x0 = g.c()
    lib().oracle_init(n, h, x0, _dp(params), _dp(np.asarray(idarr, dtype=np.float64)), _dp(state))
    return state


def flop_count_parts(g: OGrid, params, state, t=0.0):
    """Counts {add, mul, div, sqrt, cmp} per part: derivatives, ko, algebra, flux."""
    _check_state(g, params, state)
    c = np.empty(20, dtype=np.float64)
    n, h, x0 = g.c()
    lib().oracle_flop_count_parts(n, h, x0, _dp(params), _dp(state), float(t), _dp(c))
    names = ["add", "mul", "div", "sqrt", "cmp"]
    return {part: dict(zip(names, c[5 * i:5 * i + 5].tolist()))
            for i, part in enumerate(["derivatives", "ko", "algebra", "flux"])}


def rhs_vjp(g: OGrid, params, state, w, t=0.0):
    """(dF/dU)^T w by a tape over the whole right-hand side (tiny grids only)."""
    _check_state(g, params, state)
    w = np.ascontiguousarray(w, dtype=np.float64)
    assert w.shape == state.shape
    out = np.empty_like(state)
    n, h, x0 = g.c()
    lib().oracle_rhs_vjp(n, h, x0, _dp(params), _dp(state), float(t), _dp(w), _dp(out))
    return out


def rk4_stages(g: OGrid, params, state, t, dt):
    """Stage states U_1..U_4 of one classic RK4 step (as rk4_step forms them)."""
    k1 = rhs(g, params, state, t)
    U2 = state + 0.5 * dt * k1
    k2 = rhs(g, params, U2, t + 0.5 * dt)
    U3 = state + 0.5 * dt * k2
    k3 = rhs(g, params, U3, t + 0.5 * dt)
    U4 = state + dt * k3
    return [state, U2, U3, U4]


def adjoint_step(g: OGrid, params, state, lam, t, dt):
    """Reverse of one classic RK4 step U_{n+1} = U_n + dt/6 (k1 + 2 k2 + 2 k3 + k4),
    k_s = F(U_s, t_s): returns (dU_{n+1}/dU_n)^T lam, stage by stage in reverse:
    kbar_4 = dt/6 lam, then v_s = (dF/dU at U_s)^T kbar_s feeds lam_n += v_s and
    kbar_{s-1} = b_{s-1} dt lam + a_{s,s-1} dt v_s (a = 1, 1/2, 1/2)."""
    U = rk4_stages(g, params, state, t, dt)
    ts = [t, t + 0.5 * dt, t + 0.5 * dt, t + dt]
    out = lam.copy()
    kb = dt / 6.0 * lam
    v = rhs_vjp(g, params, U[3], kb, ts[3])
    out += v
    kb = dt / 3.0 * lam + dt * v
    v = rhs_vjp(g, params, U[2], kb, ts[2])
    out += v
    kb = dt / 3.0 * lam + 0.5 * dt * v
    v = rhs_vjp(g, params, U[1], kb, ts[1])
    out += v
    kb = dt / 6.0 * lam + 0.5 * dt * v
    out += rhs_vjp(g, params, U[0], kb, ts[0])
    return out


def fluid_rho(E, J2, w):
    """Rest-frame density recovered from E and J^2 for P = w rho."""
    E = np.ascontiguousarray(E, dtype=np.float64).ravel()
    J2 = np.ascontiguousarray(J2, dtype=np.float64).ravel()
    out = np.empty_like(E)
    lib().oracle_fluid_rho(_dp(E), _dp(J2), E.size, float(w), _dp(out))
    return out


def flop_count(g: OGrid, params, state, t=0.0):
    """{add, mul, div, sqrt, cmp} of one RHS evaluation at one point."""
    _check_state(g, params, state)
    c = np.empty(5, dtype=np.float64)
    n, h, x0 = g.c()
    lib().oracle_flop_count(n, h, x0, _dp(params), _dp(state), float(t), _dp(c))
    return dict(zip(["add", "mul", "div", "sqrt", "cmp"], c.tolist()))


# --------------------------------------------------------------------------
# Fixed mesh refinement (levels described by plain dicts: n, h, x0, origin,
# lo, hi per level, as paper_2606_02053_gb300.inputs.nested_boxes returns)
# --------------------------------------------------------------------------
def _hier_c(levels):
    L = len(levels)
    n = (ctypes.c_int * (3 * L))(*[int(v) for lv in levels for v in lv["n"]])
    h = (ctypes.c_double * (3 * L))(*[float(v) for lv in levels for v in lv["h"]])
    x0 = (ctypes.c_double * (3 * L))(*[float(v) for lv in levels for v in lv["x0"]])
    og = (ctypes.c_int * (3 * L))(*[int(v) for lv in levels for v in lv["origin"]])
    lo = (ctypes.c_int * (3 * L))(*[int(v) for lv in levels for v in lv["lo"]])
    hi = (ctypes.c_int * (3 * L))(*[int(v) for lv in levels for v in lv["hi"]])
    return L, n, h, x0, og, lo, hi


def _fmr_lib():
    L = lib()
    if not getattr(L, "_fmr_sigs", False):
        H = [ctypes.c_int, _I, _D, _D, _I, _I, _I]
        L.oracle_fmr_step.argtypes = H + [_D, ctypes.POINTER(_D), ctypes.c_double, ctypes.c_double]
        L.oracle_fmr_init.argtypes = H + [_D, _D, ctypes.POINTER(_D)]
        L.oracle_fmr_prolong.argtypes = H + [ctypes.c_int, ctypes.c_int, _D, _D]
        L.oracle_fmr_restrict.argtypes = H + [ctypes.c_int, ctypes.c_int, _D, _D]
        L.oracle_rk4_dense.argtypes = [ctypes.c_long, _D, _D, ctypes.c_double, ctypes.c_double, _D]
        L._fmr_sigs = True
    return L


def level_grid(level) -> OGrid:
    return OGrid(level["n"], level["h"], level["x0"])


def _check_levels(levels, params, states):
    assert len(states) == len(levels)
    for lv, s in zip(levels, states):
        _check_state(level_grid(lv), params, s)


def fmr_init(levels, params, idarr):
    """Initial data on every level of the hierarchy; returns the list of states."""
    states = [np.empty((nfields(params), lv["n"][2], lv["n"][1], lv["n"][0])) for lv in levels]
    ptrs = (_D * len(levels))(*[_dp(s) for s in states])
    _fmr_lib().oracle_fmr_init(*_hier_c(levels), _dp(params), _dp(np.asarray(idarr, dtype=np.float64)), ptrs)
    return states


def fmr_step(levels, params, states, t, dt0):
    """In place: one step of the hierarchy (level l takes 2^l steps of dt0 / 2^l)."""
    _check_levels(levels, params, states)
    ptrs = (_D * len(levels))(*[_dp(s) for s in states])
    _fmr_lib().oracle_fmr_step(*_hier_c(levels), _dp(params), ptrs, float(t), float(dt0))
    return states


def fmr_prolong(levels, level, parent, child):
    """In place: ghost points of `child` (level `level`) from the parent state."""
    nf = parent.shape[0]
    assert parent.flags.c_contiguous and child.flags.c_contiguous and child.shape[0] == nf
    _fmr_lib().oracle_fmr_prolong(*_hier_c(levels), int(level), nf, _dp(parent), _dp(child))
    return child


def fmr_restrict(levels, level, child, parent):
    """In place: interior points of `child` lying on parent points overwrite them."""
    nf = parent.shape[0]
    assert parent.flags.c_contiguous and child.flags.c_contiguous and child.shape[0] == nf
    _fmr_lib().oracle_fmr_restrict(*_hier_c(levels), int(level), nf, _dp(child), _dp(parent))
    return parent


def rk4_dense(Un, k, dt, theta):
    """U_n + dt sum_s b_s(theta) k_s for k = [k1, k2, k3, k4] (arrays like Un)."""
    Un = np.ascontiguousarray(Un, dtype=np.float64)
    kk = np.ascontiguousarray(np.stack([np.asarray(x, dtype=np.float64) for x in k]))
    out = np.empty_like(Un)
    _fmr_lib().oracle_rk4_dense(Un.size, _dp(Un), _dp(kk), float(dt), float(theta), _dp(out))
    return out


def fmr_interior(level):
    """Boolean mask [nz, ny, nx] of the interior points of a level."""
    n, lo, hi = level["n"], level["lo"], level["hi"]
    m = np.zeros((n[2], n[1], n[0]), dtype=bool)
    m[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = True
    return m


# --------------------------------------------------------------------------
# Collapse diagnostics and initial data from a per-point zeta (definitions in
# cosmos_oracle.cpp, section "Collapse diagnostics"), with their reverse modes
# and the whole pipeline zeta -> N RK4 steps -> (min central lapse, peak
# compaction) reversed through the oracle's own tapes.
# --------------------------------------------------------------------------
def _diag_lib():
    L = lib()
    if not getattr(L, "_diag_sigs", False):
        G = [_I, _D, _D, _D]
        L.oracle_init_zeta.argtypes = G + [_D, ctypes.c_double, _D]
        L.oracle_init_zeta_vjp.argtypes = G + [_D, ctypes.c_double, _D, _D]
        L.oracle_central_lapse.argtypes = [_I, _D]
        L.oracle_central_lapse.restype = ctypes.c_double
        L.oracle_compaction.argtypes = G + [_D, ctypes.c_int, _D]
        L.oracle_compaction_vjp.argtypes = G + [_D, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
        L._diag_sigs = True
    return L


def _zeta_array(g: OGrid, zeta):
    z = np.ascontiguousarray(np.asarray(zeta, dtype=np.float64).reshape(g.n[2], g.n[1], g.n[0]))
    return z


def init_zeta(g: OGrid, params, zeta, a0=1.0):
    """FLRW + curvature-perturbation data at leading gradient order from a per-point
    zeta [nz, ny, nx] (the paper's initial-data paragraph; fluid at rest, E from the
    discrete Hamiltonian constraint)."""
    z = _zeta_array(g, zeta)
    state = np.empty((nfields(params), g.n[2], g.n[1], g.n[0]), dtype=np.float64)
    n, h, x0 = g.c()
    _diag_lib().oracle_init_zeta(n, h, x0, _dp(params), _dp(z), float(a0), _dp(state))
    return state


def init_zeta_vjp(g: OGrid, params, zeta, lam0, a0=1.0):
    """zeta_bar = (d init_zeta / d zeta)^T lam0 by a tape (tiny grids)."""
    z = _zeta_array(g, zeta)
    lam0 = np.ascontiguousarray(lam0, dtype=np.float64)
    assert lam0.shape == (nfields(params), g.n[2], g.n[1], g.n[0])
    out = np.empty_like(z)
    n, h, x0 = g.c()
    _diag_lib().oracle_init_zeta_vjp(n, h, x0, _dp(params), _dp(z), float(a0), _dp(lam0), _dp(out))
    return out


def central_lapse(g: OGrid, state):
    """alpha at the centre grid point (nx/2, ny/2, nz/2)."""
    n, _, _ = g.c()
    return float(_diag_lib().oracle_central_lapse(n, _dp(np.ascontiguousarray(state))))


def compaction(g: OGrid, params, state, kmax):
    """C(r_k) = 2 dM(r_k) / R(r_k) for k = 1..kmax about the centre point (array [kmax])."""
    _check_state(g, params, state)
    out = np.empty(int(kmax), dtype=np.float64)
    n, h, x0 = g.c()
    _diag_lib().oracle_compaction(n, h, x0, _dp(params), _dp(state), int(kmax), _dp(out))
    return out


def compaction_vjp(g: OGrid, params, state, kmax, kstar, cbar=1.0):
    """cbar d C(r_kstar) / d state, state layout, by a tape."""
    _check_state(g, params, state)
    out = np.empty_like(state)
    n, h, x0 = g.c()
    _diag_lib().oracle_compaction_vjp(n, h, x0, _dp(params), _dp(state), int(kmax), int(kstar), float(cbar),
                                      _dp(out))
    return out


def collapse_run(g: OGrid, params, zeta, dt, steps, kmax, a0=1.0):
    """Forward pipeline: init_zeta, `steps` RK4 steps from t = 0.  Returns a dict with
    every time level (`states`), the central lapse per level (`alphas`), the first
    level attaining its minimum (`nstar`), the final compaction function (`C`) and the
    first maximising radius index (`kstar`, 1-based)."""
    U = init_zeta(g, params, zeta, a0)
    states = [U.copy()]
    alphas = [central_lapse(g, U)]
    for s in range(steps):
        rk4_step(g, params, U, s * dt, dt)
        states.append(U.copy())
        alphas.append(central_lapse(g, U))
    C = compaction(g, params, U, kmax)
    alphas = np.array(alphas)
    return dict(states=states, alphas=alphas, nstar=int(np.argmin(alphas)), min_lapse=float(alphas.min()),
                C=C, kstar=int(np.argmax(C)) + 1, peak=float(C.max()))


def collapse_gradient(g: OGrid, params, zeta, dt, steps, kmax, a0=1.0, run=None):
    """(d min-central-lapse / d zeta, d peak-compaction / d zeta), each [nz, ny, nx]:
    the compaction's tape at the final level, the lapse seed at the first minimising
    level, the RK4 adjoint step (tape of the right-hand side) back through every level,
    then the tape of the zeta map.  Tiny grids only."""
    r = run if run is not None else collapse_run(g, params, zeta, dt, steps, kmax, a0)
    ia = ALPHA_FIELD
    nz, ny, nx = g.n[2], g.n[1], g.n[0]
    out = []
    for which in ("lapse", "compaction"):
        if which == "compaction":
            lam = compaction_vjp(g, params, r["states"][steps], kmax, r["kstar"])
        else:
            lam = np.zeros_like(r["states"][0])
        if which == "lapse" and r["nstar"] == steps:
            lam[ia, nz // 2, ny // 2, nx // 2] += 1.0
        for s in reversed(range(steps)):
            lam = adjoint_step(g, params, r["states"][s], lam, s * dt, dt)
            if which == "lapse" and s == r["nstar"]:
                lam[ia, nz // 2, ny // 2, nx // 2] += 1.0
        out.append(init_zeta_vjp(g, params, zeta, lam, a0))
    return out[0], out[1], r


ALPHA_FIELD = 17

"""Seeded synthetic inputs shared by the tests, the bench and the oracle leg.

This module holds none of the method's arithmetic: only random numbers and
plain data (grid shapes, parameter values).  Both the CUDA path and the CPU
oracle receive the arrays it produces, so neither side generates inputs for
the other.

* ``smooth_state``: a generic smooth periodic state for right-hand-side
  parity tests -- every evolved field is a base value plus a short sum of
  random Fourier modes (integer wave numbers, so the field is periodic on the
  box).  The base keeps the conformal metric close to the identity, chi, the
  lapse and the fluid energy positive and the fluid velocity small.
* ``splitmix64`` / ``uniform53``: the counter-free generator used to draw the
  batched threshold-scan instances (seed 2606, draw order documented below).
* ``scan_instances``: parameters of the batched scan: N uniform in [64, 96],
  mu in [0.3, 0.9], sigma in [L/10, L/6], axis ratios q_1..3 in [0.8, 1.2],
  drawn in that order per instance.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1

# base values per field (state order: chi, gt(6), K, At(6), Gt(3), alpha,
# beta(3), B(3), [tau, S(3)], [phi, Pi])
_BASE_BSSN = [1.0, 1.0, 0.0, 0.0, 1.0, 0.0, 1.0, 0.0] + [0.0] * 6 + [0.0] * 3 + [1.0] + [0.0] * 6
_AMP_BSSN = [0.1] + [0.05] * 6 + [0.2] + [0.1] * 6 + [0.2] * 3 + [0.1] + [0.05] * 3 + [0.05] * 3


def nfields(fluid: bool, scalar: bool) -> int:
    return 24 + 4 * int(bool(fluid)) + 2 * int(bool(scalar))


def smooth_state(n, seed, fluid=False, scalar=False, modes=3, kmax=2, scale=1.0):
    """Random smooth periodic state, array [nf, nz, ny, nx] (float64).

    Field f = base_f + scale * amp_f * sum_m c_{f,m} sin(2 pi k_m . x / n + p_{f,m})
    with x the integer grid index, k_m integer in [-kmax, kmax]^3.
    """
    nx, ny, nz = (n, n, n) if np.isscalar(n) else tuple(n)
    rng = np.random.default_rng(seed)
    base = list(_BASE_BSSN)
    amp = list(_AMP_BSSN)
    if fluid:
        base += [1.0, 0.0, 0.0, 0.0]
        amp += [0.2, 0.05, 0.05, 0.05]
    if scalar:
        base += [0.0, 0.0]
        amp += [0.2, 0.2]
    nf = len(base)
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    out = np.empty((nf, nz, ny, nx), dtype=np.float64)
    for f in range(nf):
        acc = np.zeros((nz, ny, nx))
        for _ in range(modes):
            kv = rng.integers(-kmax, kmax + 1, size=3)
            c = rng.uniform(-1.0, 1.0)
            p = rng.uniform(0.0, 2.0 * np.pi)
            acc += c * np.sin(2.0 * np.pi * (kv[0] * i / nx + kv[1] * j / ny + kv[2] * k / nz) + p)
        out[f] = base[f] + scale * amp[f] * acc
    return out


def splitmix64(state: int):
    """One step of SplitMix64 (Steele, Lea, Flood 2014): returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def uniform53(state: int):
    """Double in [0, 1) from the top 53 bits of one SplitMix64 output."""
    state, z = splitmix64(state)
    return state, (z >> 11) * (1.0 / (1 << 53))


def scan_instances(count=64, seed=2606, n_lo=64, n_hi=96, L=1.0):
    """Threshold-scan instances: list of dicts {n, mu, sigma, q}.

    Per instance, in this order: N = n_lo + floor(u * (n_hi - n_lo + 1)),
    mu = 0.3 + 0.6 u, sigma = L/10 + (L/6 - L/10) u, q_1, q_2, q_3 = 0.8 + 0.4 u.
    """
    s = seed
    out = []
    for _ in range(count):
        s, u = uniform53(s)
        n = n_lo + int(u * (n_hi - n_lo + 1))
        s, u = uniform53(s)
        mu = 0.3 + 0.6 * u
        s, u = uniform53(s)
        sigma = L / 10.0 + (L / 6.0 - L / 10.0) * u
        q = []
        for _ in range(3):
            s, u = uniform53(s)
            q.append(0.8 + 0.4 * u)
        out.append(dict(n=n, mu=mu, sigma=sigma, q=tuple(q)))
    return out


# Workload descriptions (plain data).
GAUGE_WAVE = dict(A=0.01, L=1.0, cfl=0.25)
FLRW_ZETA = dict(w=1.0 / 3.0, mu=0.5, sigma_over_L=1.0 / 8.0, H0_times_L=40.0, cfl=0.25)


def nested_boxes(n0, h0, x0, levels, n_child, centre=None):
    """Plain description of a fixed-mesh-refinement hierarchy of nested boxes.

    Level 0: the periodic box of n0 = (nx, ny, nz) points, spacing h0, point 0
    at x0.  Level l >= 1: an array of n_child[l-1] = (nx, ny, nz) points (an int
    gives a cube) with spacing h0 / 2^l.  Along each axis it is either periodic
    (n = 2 x the parent's points, when the parent is periodic there) or a box
    whose interior [lo, hi) holds an odd number of points centred on the
    parent's centre point, with 3 ghost layers below and 3 or 4 above.
    centre: level-0 index of the centre point (default n0 // 2 per axis).

    Returns a list of per-level dicts: n, h, x0, origin, lo, hi (origin is
    the position of the level's point 0 on its parent, in the level's own
    spacing: x0_l = x0_{l-1} + origin * h_l).
    """
    n0 = (n0,) * 3 if np.isscalar(n0) else tuple(int(v) for v in n0)
    c_prev = [n0[d] // 2 for d in range(3)] if centre is None else list(centre)
    out = [dict(n=n0, h=(h0,) * 3, x0=tuple(float(v) for v in x0), origin=(0, 0, 0), lo=(0, 0, 0), hi=n0,
                periodic=(True, True, True))]
    for l in range(1, levels):
        nc = n_child[l - 1]
        nc = (nc,) * 3 if np.isscalar(nc) else tuple(int(v) for v in nc)
        par = out[-1]
        h = par["h"][0] / 2.0
        origin, lo, hi, per, c_new = [], [], [], [], []
        for d in range(3):
            if par["periodic"][d] and nc[d] == 2 * par["n"][d]:
                origin.append(0)
                lo.append(0)
                hi.append(nc[d])
                per.append(True)
                c_new.append(2 * c_prev[d])
            else:
                if nc[d] < 8:
                    raise ValueError("a refined box needs at least 8 points per axis")
                a, b = 3, nc[d] - 3 - (1 if (nc[d] - 6) % 2 == 0 else 0)
                cc = a + (b - a - 1) // 2
                origin.append(2 * c_prev[d] - cc)
                lo.append(a)
                hi.append(b)
                per.append(False)
                c_new.append(cc)
        x0l = tuple(par["x0"][d] + origin[d] * h for d in range(3))
        out.append(dict(n=nc, h=(h,) * 3, x0=x0l, origin=tuple(origin), lo=tuple(lo), hi=tuple(hi),
                        periodic=tuple(per)))
        c_prev = c_new
    return out

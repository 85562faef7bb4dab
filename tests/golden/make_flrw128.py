"""Writes ``flrw_zeta_128_200steps.json``: the CPU oracle's state after 200 RK4
steps of the radiation FLRW + Gaussian zeta workload at 128^3, sampled.

Workload (the benchmark's FLRW configuration, §Physical system settings,
initial-data paragraph): w = 1/3, a0 = 1, H0 L = 40, zeta = mu exp(-r^2 /
(2 sigma^2)) with mu = 0.5, sigma = L/8 about the centre grid point, 1+log
slicing with the background trace, Gamma-driver shift (eta = 2/L), KO sigma =
0.1, dt = h/4, 200 steps.  The oracle evolves the whole grid once (about an
hour on eight cores); the file keeps every field's largest magnitude over the
grid (the scale of the 1e-10 tolerance) and the values of all fields at a few
thousand seeded points, including faces, edges, corners and the centre.

Nothing here comes from the CUDA path: this script calls only ``oracle`` (and
numpy).  ``python tests/golden/make_flrw128.py [threads]``.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

OUT = os.path.join(HERE, "flrw_zeta_128_200steps.json")
N = 128
STEPS = 200
PARAMS = dict(slicing=0, shift=1, eta=2.0, ko_sigma=0.1, fluid=1, scalar=0, w=1.0 / 3.0, H0=40.0, t0=0.0)
ID = dict(kind=1, mu=0.5, sigma=0.125)
SEED = 1282


def sample_points(n, count, seed):
    """Seeded random points plus corners, edge midpoints, face centres and the centre."""
    rng = np.random.default_rng(seed)
    pts = [tuple(int(v) for v in rng.integers(0, n, size=3)) for _ in range(count)]
    ends = [0, 1, 2, n // 2 - 1, n // 2, n // 2 + 1, n - 3, n - 2, n - 1]
    for a in ends:
        for b in ends:
            pts += [(a, b, 0), (a, 0, b), (0, a, b), (a, b, n - 1), (a, n - 1, b), (n - 1, a, b)]
    return np.unique(np.array(pts, dtype=np.int64).reshape(-1, 3), axis=0)


def hexes(a):
    return [float(v).hex() for v in np.asarray(a, dtype=np.float64).ravel()]


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    if threads > 0:
        O.set_threads(threads)
    h = 1.0 / N
    x0 = (-(N // 2) * h,) * 3
    g = O.OGrid((N, N, N), h, x0=x0)
    P = O.params_array(**PARAMS)
    s = O.init(g, P, O.id_array(**ID))
    dt = 0.25 * h
    t_start = time.time()
    for step in range(STEPS):
        O.rk4_step(g, P, s, step * dt, dt)
        if step % 10 == 9:
            print(f"step {step + 1}/{STEPS}  {time.time() - t_start:.0f} s", flush=True)
    _, norms = O.constraints(g, P, s)
    pts = sample_points(N, 3000, SEED)
    vals = s[:, pts[:, 2], pts[:, 1], pts[:, 0]]  # [nf, npts]
    out = {"about": "oracle state of the 128^3 FLRW + zeta workload after 200 RK4 steps (hex floats); "
                    "written by tests/golden/make_flrw128.py",
           "n": N, "steps": STEPS, "dt": dt, "x0": list(x0), "params": PARAMS, "id": ID,
           "points_ijk": pts.tolist(),
           "field_max": hexes(np.abs(s).reshape(s.shape[0], -1).max(axis=1)),
           "norms": hexes(norms),
           "values": [hexes(v) for v in vals]}
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    print("wrote", OUT, f"{time.time() - t_start:.0f} s")


if __name__ == "__main__":
    main()

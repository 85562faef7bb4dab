"""Writes ``oracle_regression.json``: sampled outputs of the CPU oracle on small
seeded cases, stored as hexadecimal floats.

The paper prints no worked-example values for the evolution equations, so
nothing here is a value from the paper.  These fixtures are regression
anchors for the oracle itself: ``tests/test_oracle_golden.py`` recomputes
them and fails when the oracle's arithmetic changes.  A change that is
meant must rewrite the file with this script, in a commit that names the
section of the paper (or the reading of it) that justifies it.  What pins
the oracle to the mathematics are the other ``tests/test_oracle_*.py``.

This script calls only ``oracle`` (and numpy): ``python tests/golden/make_golden.py``.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

OUT = os.path.join(HERE, "oracle_regression.json")

# (name, grid n, params, initial-data array, time step) — every state comes from
# the oracle's own initial data, so no input generator enters the fixture
CASES = [
    # gauge wave, 1+log slicing + Gamma-driver shift, KO on (BSSN vacuum, §Formulation)
    ("gauge_wave_vacuum", (16, 8, 8), dict(slicing=0, shift=1, eta=2.0, ko_sigma=0.1),
     dict(kind=0, A=0.1), 0.25 / 16),
    # FLRW + Gaussian zeta with a radiation fluid, harmonic slicing, frozen shift (§Initial conditions)
    ("flrw_zeta_fluid", (12, 12, 12), dict(slicing=1, shift=0, ko_sigma=0.1, fluid=1, w=1.0 / 3.0, H0=40.0),
     dict(kind=1, mu=0.3, sigma=0.15, q=(1.0, 0.9, 1.1)), 0.25 / 12),
    # isocurvature data of a massless scalar beside the fluid (§Initial conditions)
    ("isocurvature_scalar", (12, 10, 12), dict(slicing=0, shift=1, eta=1.3, ko_sigma=0.2, fluid=1, scalar=1,
                                               w=1.0 / 3.0, H0=40.0),
     dict(kind=2, A=0.02, mu=0.3, sigma=0.125, q=(1.0, 0.9, 1.1)), 0.25 / 12),
]

N_SAMPLES = 12
SEED = 20260603


def hexes(a):
    return [float(v).hex() for v in np.asarray(a, dtype=np.float64).ravel()]


def case_values(n, params, idd, dt):
    g = O.OGrid(n, 1.0 / n[0])
    P = O.params_array(**params)
    s = O.init(g, P, O.id_array(**idd))
    rng = np.random.default_rng(SEED)
    pts = np.stack([rng.integers(0, n[a], N_SAMPLES) for a in range(3)], axis=1)  # (i, j, k)
    flat = (pts[:, 2] * n[1] + pts[:, 1]) * n[0] + pts[:, 0]
    r = O.rhs(g, P, s, 0.0).reshape(s.shape[0], -1)
    u1 = O.rk4_step(g, P, s.copy(), 0.0, dt).reshape(s.shape[0], -1)
    ham_mom, norms = O.constraints(g, P, s)
    # each field's largest magnitude over the whole grid: the scale the parity tolerances refer to
    return {"points_ijk": pts.tolist(), "rhs": hexes(r[:, flat]), "rk4_step": hexes(u1[:, flat]),
            "rhs_field_max": hexes(np.abs(r).max(axis=1)), "rk4_step_field_max": hexes(np.abs(u1).max(axis=1)),
            "norms": hexes(norms)}


def main():
    out = {"about": "oracle regression fixtures (hex floats); written by tests/golden/make_golden.py",
           "n_samples": N_SAMPLES, "seed": SEED, "cases": {}}
    for name, n, params, idd, dt in CASES:
        out["cases"][name] = {"n": list(n), "params": params, "id": {k: (list(v) if isinstance(v, tuple) else v)
                                                                       for k, v in idd.items()},
                              "dt": dt, **case_values(n, params, idd, dt)}
    cases = out.pop("cases")
    with open(OUT, "w") as f:  # one line per case
        f.write(json.dumps(out)[:-1] + ', "cases": {\n')
        f.write(",\n".join(f"{json.dumps(k)}: {json.dumps(v)}" for k, v in cases.items()))
        f.write("\n}}\n")


if __name__ == "__main__":
    main()

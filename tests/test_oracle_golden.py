"""The oracle against its stored regression fixtures (``tests/golden/``).

The fixtures hold sampled right-hand sides, one RK4 step and the constraint
norms of three small cases built from the oracle's own initial data (gauge
wave, FLRW + zeta with the fluid, isocurvature scalar).  They are not values
from the paper, which prints none for these equations: they anchor the
oracle against unintended change.  The tolerance, 1e-13 of each field's
largest sampled magnitude, absorbs a different libm or compiler, not a
changed term (a dropped term or a wrong coefficient moves values by far
more).
"""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "oracle_regression.json")
TOL = 1e-13


def load():
    with open(FIXTURE) as f:
        return json.load(f)


def unhex(v):
    return np.array([float.fromhex(x) for x in v])


def recompute(O, c):
    n = tuple(c["n"])
    g = O.OGrid(n, 1.0 / n[0])
    P = O.params_array(**c["params"])
    idd = {k: (tuple(v) if isinstance(v, list) else v) for k, v in c["id"].items()}
    s = O.init(g, P, O.id_array(**idd))
    pts = np.array(c["points_ijk"])
    flat = (pts[:, 2] * n[1] + pts[:, 1]) * n[0] + pts[:, 0]
    r = O.rhs(g, P, s, 0.0).reshape(s.shape[0], -1)[:, flat]
    u1 = O.rk4_step(g, P, s.copy(), 0.0, c["dt"]).reshape(s.shape[0], -1)[:, flat]
    _, norms = O.constraints(g, P, s)
    return {"rhs": r, "rk4_step": u1, "norms": norms}


def rel_err(got, want):
    want = want.reshape(got.shape)
    scale = np.maximum(np.abs(want).max(axis=-1, keepdims=True), 1e-300)
    return float((np.abs(got - want) / scale).max())


@pytest.mark.parametrize("name", ["gauge_wave_vacuum", "flrw_zeta_fluid", "isocurvature_scalar"])
def test_oracle_matches_stored_fixture(O, name):
    c = load()["cases"][name]
    got = recompute(O, c)
    for key in ("rhs", "rk4_step"):
        assert rel_err(got[key], unhex(c[key])) <= TOL, key
    # constraint norms: the FLRW data satisfy H = 0 and M = 0 to rounding (norms ~1e-12 against an
    # energy density ~1e4), so there only "still at rounding level" is fixed; elsewhere relative TOL
    want = unhex(c["norms"])
    small = want < 1e-9
    assert np.all(got["norms"][small] < 1e-9)
    assert np.all(np.abs(got["norms"] - want)[~small] <= TOL * want[~small])


def test_fixture_is_sensitive_to_a_planted_change(O):
    """A change far below any plausible mistake (one part in 1e-9 of one
    field's sampled RHS) already fails the comparison."""
    c = load()["cases"]["gauge_wave_vacuum"]
    got = recompute(O, c)
    r = got["rhs"].copy()
    r[8] *= 1.0 + 1e-9  # At_xx
    assert rel_err(r, unhex(c["rhs"])) > TOL

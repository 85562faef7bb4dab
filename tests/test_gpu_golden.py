"""The CUDA path (initial data, one right-hand side, one RK4 step, the
constraint norms) against the stored oracle fixtures in ``tests/golden/``.

Unlike the other parity tests this one needs no oracle build on the device
host: the expected values were written by ``tests/golden/make_golden.py``,
which calls only the oracle.  Tolerances as in test_gpu_parity: 1e-12 of each
field's largest magnitude over the grid (stored beside the samples; floor
1e-12 of the largest over all fields) for the right-hand side, 1e-10 after
the step.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "oracle_regression.json")
RHS_TOL = 1e-12
STEP_TOL = 1e-10


@pytest.fixture(scope="module")
def C():
    from paper_2606_02053_gb300 import build, cosmos

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    cosmos.lib()
    return cosmos


def unhex(v, nf):
    return np.array([float.fromhex(x) for x in v]).reshape(nf, -1)


def field_errors(got, want, field_max):
    """Largest error of each field over the samples, relative to the field's
    largest magnitude over the whole grid (floor 1e-12 of the largest field)."""
    den = np.maximum(field_max, 1e-12 * field_max.max())
    return np.abs(got - want).max(axis=1) / den


@pytest.mark.parametrize("name", ["gauge_wave_vacuum", "flrw_zeta_fluid", "isocurvature_scalar"])
def test_cuda_path_matches_stored_oracle_values(C, name):
    from paper_2606_02053_gb300.evolve import Evolution

    with open(FIXTURE) as f:
        c = json.load(f)["cases"][name]
    n = tuple(c["n"])
    ev = Evolution(C.make_grid(n, 1.0 / n[0]), C.make_params(**c["params"]))
    ev.init(C.make_id(**c["id"]))
    pts = np.array(c["points_ijk"])

    def sample(flat):
        a = ev.get(flat)
        return a[:, pts[:, 2], pts[:, 1], pts[:, 0]]

    r = sample(ev.rhs(0.0))
    fmax = {k: np.array([float.fromhex(x) for x in c[k + "_field_max"]]) for k in ("rhs", "rk4_step")}
    assert field_errors(r, unhex(c["rhs"], ev.nf), fmax["rhs"]).max() <= RHS_TOL
    _, norms = ev.constraints()
    want = np.array([float.fromhex(x) for x in c["norms"]])
    small = want < 1e-9
    assert np.all(norms[small] < 1e-9)
    assert np.all(np.abs(norms - want)[~small] <= 1e-10 * want[~small])
    ev.step(0.0, c["dt"])
    assert field_errors(sample(None), unhex(c["rk4_step"], ev.nf), fmax["rk4_step"]).max() <= STEP_TOL

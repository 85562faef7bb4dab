"""The 128^3 FLRW + zeta workload (radiation fluid, mu = 0.5, sigma = L/8, H0 L =
40; section "Physical system settings") after its full 200 RK4 steps, against
the oracle's own evolution of the whole grid (tests/golden/make_flrw128.py,
which calls only the oracle: every field at ~3000 seeded points, corners,
edges, face centres and the centre included, and each field's largest
magnitude over the grid).  The bar is the stated 1e-10 after the steps, per
field, relative to that field's largest magnitude; the constraint norms must
agree to the same 1e-10 of the scale of the terms whose difference they are
(6 H0^2 for H, H0^2 for M).
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "flrw_zeta_128_200steps.json")


@pytest.fixture(scope="module")
def C():
    from paper_2606_02053_gb300 import build, cosmos

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    cosmos.lib()
    return cosmos


def unhex(v):
    return np.array([float.fromhex(x) for x in v])


def test_flrw_zeta_128_cube_after_200_steps_matches_the_oracle(C):
    from paper_2606_02053_gb300.evolve import Evolution

    ref = json.load(open(FIXTURE))
    n, steps, dt = ref["n"], ref["steps"], ref["dt"]
    h = 1.0 / n
    P = ref["params"]
    p = C.make_params(slicing=P["slicing"], shift=P["shift"], eta=P["eta"], ko_sigma=P["ko_sigma"], fluid=P["fluid"],
                      scalar=P["scalar"], w=P["w"], H0=P["H0"], t0=P["t0"])
    ev = Evolution(C.make_grid(n, h, x0=tuple(ref["x0"])), p)
    ev.init(C.make_id(ref["id"]["kind"], mu=ref["id"]["mu"], sigma=ref["id"]["sigma"]))
    ev.step(0.0, dt, steps=steps)
    _, norms = ev.constraints()
    pts = np.array(ref["points_ijk"], dtype=np.int64)
    got = ev.view()[:, pts[:, 2], pts[:, 1], pts[:, 0]].cpu().numpy()  # [nf, npts]
    del ev
    torch.cuda.empty_cache()
    want = np.stack([unhex(v) for v in ref["values"]])
    scale = unhex(ref["field_max"])
    scale = np.maximum(scale, 1e-12 * scale.max())
    err = np.abs(got - want).max(axis=1) / scale
    assert err.max() <= 1e-10, err
    onorms = unhex(ref["norms"])
    H0 = P["H0"]
    tol = 1e-10 * np.array([6 * H0 ** 2] + [H0 ** 2] * 3 + [6 * H0 ** 2] + [H0 ** 2] * 3)
    assert np.all(np.abs(np.asarray(norms) - onorms) <= tol), (norms, onorms)

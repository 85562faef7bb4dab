"""cosmos_constraints_noalloc against cosmos_constraints, through the C ABI.

The no-allocation variant is for callers that cannot call cudaMalloc while
they run (applications whose device memory is handed out by their own pool
or framework): its scratch is a static device array inside the library.  It
must give the same constraint fields and norms as the workspace-taking entry
point, on repeated calls (the shared array keeps the previous call's
contents, which must not leak into the next result), and reject grids that
do not fit the array before launching anything.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12  # same per-field relative bar as the right-hand-side parity tests


@pytest.fixture(scope="module")
def C():
    from paper_2606_02053_gb300 import build, cosmos

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    cosmos.lib()
    return cosmos


def _rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    den = np.maximum(np.abs(b).max(axis=1), 1e-12 * np.abs(b).max())
    return (np.abs(a - b).max(axis=1) / den).max()


@pytest.mark.parametrize("fluid,scalar,n", [(0, 0, (40, 24, 18)), (1, 1, (30, 20, 16))])
def test_noalloc_matches_workspace_entry_point_twice(C, fluid, scalar, n):
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    h = 1.0 / n[0]
    p = C.make_params(fluid=fluid, scalar=scalar)
    ev = Evolution(C.make_grid(n, h, pitch=n[0] + 8), p)
    ev.set_state(inputs.smooth_state(n, seed=77 + fluid, fluid=fluid, scalar=scalar))
    ref_hm, ref_norms = ev.constraints(want_fields=True)
    for call in range(2):
        hm = torch.full((4 * ev.fs,), np.nan, dtype=torch.float64, device="cuda")
        norms = (ctypes.c_double * 8)()
        rc = C.cosmos_constraints_noalloc(ev.g, ev.p, ev.state, hm, norms)
        assert rc == C.COSMOS_OK, C.lib().cosmos_strerror(rc)
        got = ev.view(hm)[..., : ev.g.nx].cpu().numpy()
        assert _rel(got, ref_hm) <= TOL, call
        np.testing.assert_allclose(np.array(list(norms)), ref_norms, rtol=TOL, atol=0)
    # norms only (no per-point output)
    norms = (ctypes.c_double * 8)()
    assert C.cosmos_constraints_noalloc(ev.g, ev.p, ev.state, None, norms) == C.COSMOS_OK
    np.testing.assert_allclose(np.array(list(norms)), ref_norms, rtol=TOL, atol=0)


def test_noalloc_rejects_grids_beyond_the_static_scratch(C):
    g = C.make_grid((96, 96, 96), 1.0 / 96)
    p = C.make_params(fluid=1)  # 4 * 96^3 primitive doubles exceed the 2^21-double array
    norms = (ctypes.c_double * 8)()
    state = torch.zeros(16, dtype=torch.float64, device="cuda")  # never read: rejected before any launch
    assert C.cosmos_constraints_noalloc(g, p, state, None, norms) == C.COSMOS_EWORKSPACE

"""Failure detection on the device: cosmos_scan_state counts, per field, the
NaN/Inf values of a state and (fluid on) the points with tau~ <= 0, by a
reduction, never a trap.  The bad values are planted on the host; the GPU
only reads them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_2606_02053_gb300 import build, cosmos

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    cosmos.lib()
    return cosmos


def test_sound_state_passes_and_planted_values_are_counted(C):
    from paper_2606_02053_gb300.evolve import Evolution

    n = (37, 21, 19)  # ragged against the 256-thread blocks
    ev = Evolution(C.make_grid(n, 1.0 / 37, pitch=40), C.make_params())
    ev.init(C.make_id(0, A=0.05))
    assert ev.scan() == {}
    s = ev.get()
    s[8, 3, 4, 5] = np.nan
    s[3, 0, 0, 0] = np.inf
    s[3, 18, 20, 36] = -np.inf  # the last point of the field
    ev.set_state(s)
    assert ev.scan() == {3: 2, 8: 1}
    code, counts = C.cosmos_scan_state(ev.g, ev.p, ev.state,
                                       torch.empty(32, dtype=torch.float64, device="cuda"))
    assert code == C.COSMOS_ENONFINITE and counts[3] == 2 and counts[8] == 1 and sum(counts) == 3


def test_padding_columns_are_not_read(C):
    from paper_2606_02053_gb300.evolve import Evolution

    n = (20, 12, 9)
    ev = Evolution(C.make_grid(n, 0.05, pitch=32), C.make_params())
    ev.init(C.make_id(0, A=0.05))
    ev.view()[..., n[0]:] = float("nan")  # columns nx .. pitch-1
    assert ev.scan() == {}


def test_fluid_energy_density_must_be_positive(C):
    from paper_2606_02053_gb300.evolve import Evolution

    n = (16, 16, 16)
    ev = Evolution(C.make_grid(n, 1.0 / 16), C.make_params(fluid=1, w=1.0 / 3.0, H0=40.0))
    ev.init(C.make_id(1, mu=0.3, sigma=0.15))
    assert ev.scan() == {}
    s = ev.get()
    s[24, 1, 2, 3] = 0.0
    s[24, 9, 9, 9] = -1e-3
    s[25, 4, 4, 4] = np.nan
    ev.set_state(s)
    assert ev.scan() == {24: 2, 25: 1}

"""Checkpoint / resume of device states: a save/load round trip is bitwise,
and a run resumed from a checkpoint continues bitwise as the run that was
not interrupted (the library's RK4 step is deterministic)."""
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


def test_resume_continues_bitwise(C, tmp_path):
    from paper_2606_02053_gb300.evolve import Evolution

    n = (40, 24, 20)
    g = C.make_grid(n, 1.0 / 40, pitch=48)
    p = C.make_params(fluid=1, w=1.0 / 3.0, H0=40.0)
    dt = 0.25 / 40
    a = Evolution(g, p)
    a.init(C.make_id(1, mu=0.3, sigma=0.15))
    a.step(0.0, dt, 3)
    path = str(tmp_path / "run.ck")
    a.save(path, 3 * dt, 3)
    a.step(3 * dt, dt, 2)

    b = Evolution(g, p)
    b.state.fill_(float("nan"))
    t, step = b.load(path)
    assert t == 3 * dt and step == 3
    b.step(t, dt, 2)
    assert torch.equal(a.view()[..., : n[0]], b.view()[..., : n[0]])
    assert torch.isnan(b.view()[..., n[0]:]).all()  # padding columns are not written by a load

    c = Evolution(g, p)
    host = np.zeros((C.cosmos_nfields(p), n[2], n[1], 48))
    code, t2, step2 = C.cosmos_checkpoint_load(path, g, p, host)  # the same file into host memory
    assert code == C.COSMOS_OK and (t2, step2) == (t, step)
    c.set_state(host[..., : n[0]])
    c.step(t, dt, 2)
    assert torch.equal(a.view()[..., : n[0]], c.view()[..., : n[0]])

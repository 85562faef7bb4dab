"""Slab decomposition on one GPU: the grid held as 1, 2 or 3 z-slabs with ghost
planes in one process (LocalExchange), stepped through cosmos_rk4_stage_slab
with the exponents maximised over the slabs, against cosmos_rk4_step on the
whole grid -- bitwise, for vacuum, fluid + scalar and FLRW + zeta data, on
uneven slabs and a padded row pitch.  The same code with DistExchange runs one
slab per GPU; its exchange is checked on CPU ranks in test_slab_gloo.py.
"""
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


def run_both(C, n, h, x0, p, full_state_setter, slabs_n, steps, pitch=None, t0=0.0):
    from paper_2606_02053_gb300.evolve import Evolution
    from paper_2606_02053_gb300.slab import LocalExchange, Slab, SlabEvolution, gather, scatter, slab_bounds

    ev = Evolution(C.make_grid(n, h, x0=x0, pitch=pitch), p)
    full_state_setter(ev)
    U0 = ev.state.clone()
    dt = 0.25 * h
    ev.step(t0, dt, steps=steps)
    ref = ev.view(ev.state)
    slabs = [Slab(n, (h, h, h), x0, p, k0, k1, pitch=ev.g.pitch) for k0, k1 in slab_bounds(n[2], slabs_n)]
    scatter(ev.view(U0), slabs)
    SlabEvolution(slabs, LocalExchange()).step(t0, dt, steps=steps)
    got = gather(slabs, torch.empty_like(ref))
    nx = n[0]
    return got[..., :nx], ref[..., :nx]


@pytest.mark.parametrize("slabs_n", [1, 2, 3])
def test_vacuum_slabs_equal_the_whole_grid_bitwise(C, slabs_n):
    from paper_2606_02053_gb300 import inputs

    n = (20, 12, 18)
    s = inputs.smooth_state(n, seed=31, scale=0.5)
    got, ref = run_both(C, n, 1.0 / 20, (0.0, 0.0, 0.0), C.make_params(slicing=0, shift=1), lambda ev: ev.set_state(s),
                        slabs_n, 4, pitch=24, t0=0.02)
    assert torch.equal(got, ref)


def test_fluid_and_scalar_slabs_equal_the_whole_grid_bitwise(C):
    from paper_2606_02053_gb300 import inputs

    n = (16, 10, 15)
    s = inputs.smooth_state(n, seed=32, fluid=True, scalar=True, scale=0.5)
    p = C.make_params(fluid=1, scalar=1, H0=2.0)
    got, ref = run_both(C, n, 1.0 / 16, (0.0, 0.0, 0.0), p, lambda ev: ev.set_state(s), 2, 3)
    assert torch.equal(got, ref)


def test_flrw_zeta_slabs_equal_the_whole_grid_bitwise(C):
    n = (20, 20, 20)
    h = 1.0 / 20
    x0 = (-10 * h,) * 3
    p = C.make_params(fluid=1, H0=40.0)
    got, ref = run_both(C, n, h, x0, p, lambda ev: ev.init(C.make_id(1, mu=0.5, sigma=0.125)), 3, 5)
    assert torch.equal(got, ref)
    assert float(ref.abs().max()) > 0 and bool(torch.isfinite(ref).all())


def test_slab_stage_refuses_a_plane_range_outside_the_grid(C):
    from paper_2606_02053_gb300.slab import Slab

    p = C.make_params()
    s = Slab((8, 8, 9), (0.1, 0.1, 0.1), (0.0, 0.0, 0.0), p, 0, 9)
    for k_lo, k_cnt in ((-1, 3), (0, 0), (10, 6), (3, 13)):
        assert C.cosmos_rk4_stage_slab(s.g, p, 1, s.state, s.state, s.A, s.acc, 0.0, 0.01, k_lo, k_cnt, s.E,
                                       s.ws) == C.COSMOS_EINVAL

"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances (per field f, oracle o, GPU g):
    err_f = max|g - o| / max(max|o_f|, 1e-12 * max_all|o|)
    right-hand side:  err_f <= 1e-12;   after the stated step counts: <= 1e-10.
The GPU contracts multiply-adds into FMA and orders sums differently; all
stencils difference neighbouring values first on both sides, so the
remaining rounding differences are a few ulps of each term.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-12
STEP_TOL = 1e-10


def field_errors(gpu, ref):
    gpu = gpu.reshape(gpu.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    floor = 1e-12 * np.abs(ref).max()
    den = np.maximum(np.abs(ref).max(axis=1), floor)
    return np.abs(gpu - ref).max(axis=1) / den


@pytest.fixture(scope="module")
def C():
    from paper_2606_02053_gb300 import build, cosmos

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    cosmos.lib()
    return cosmos


def oracle_params(O, Cp):
    return O.params_array(slicing=Cp.slicing, shift=Cp.shift, eta=Cp.eta, ko_sigma=Cp.ko_sigma, w=Cp.w,
                          fluid=Cp.fluid, scalar=Cp.scalar, H0=Cp.H0, t0=Cp.t0)


def run_rhs(C, O, n, h, params, state, t=0.0, pitch=None):
    from paper_2606_02053_gb300.evolve import Evolution

    g = C.make_grid(n, h, pitch=pitch)
    ev = Evolution(g, params)
    ev.set_state(state)
    r = ev.get(ev.rhs(t))
    og = O.OGrid(n, h)
    ref = O.rhs(og, oracle_params(O, params), state, t)
    return r, ref


@pytest.mark.parametrize("fluid,scalar", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("n,pitch", [((20, 12, 9), None), ((37, 13, 11), 40), ((33, 8, 16), None)])
def test_rhs_parity_smooth_random_state(C, O, fluid, scalar, n, pitch):
    from paper_2606_02053_gb300 import inputs

    p = C.make_params(slicing=0, shift=1, fluid=fluid, scalar=scalar, eta=1.7, ko_sigma=0.1, H0=2.0 * fluid)
    s = inputs.smooth_state(n, seed=100 + 7 * fluid + scalar, fluid=fluid, scalar=scalar)
    r, ref = run_rhs(C, O, n, 1.0 / n[0], p, s, t=0.013, pitch=pitch)
    err = field_errors(r, ref)
    assert err.max() <= RHS_TOL, (err.argmax(), err.max(), err)


@pytest.mark.parametrize("slicing,shift", [(1, 0), (0, 0), (1, 1)])
def test_rhs_parity_gauge_options(C, O, slicing, shift):
    from paper_2606_02053_gb300 import inputs

    n = (16, 16, 16)
    p = C.make_params(slicing=slicing, shift=shift, eta=0.5, ko_sigma=0.3)
    s = inputs.smooth_state(n, seed=5)
    r, ref = run_rhs(C, O, n, 0.0625, p, s)
    assert field_errors(r, ref).max() <= RHS_TOL


def test_rhs_parity_thin_and_tiny_grids(C, O):
    from paper_2606_02053_gb300 import inputs

    p = C.make_params()
    for n in [(16, 1, 1), (8, 3, 2), (1, 1, 1), (5, 7, 1)]:
        s = inputs.smooth_state(n, seed=9)
        r, ref = run_rhs(C, O, n, 0.1, p, s)
        assert field_errors(r, ref).max() <= RHS_TOL, n


@pytest.mark.parametrize("fluid,scalar", [(0, 0), (1, 1)])
def test_rhs_parity_anisotropic_spacing(C, O, fluid, scalar):
    """Unequal h along the axes: the derivative pass takes its per-axis
    Kreiss-Oliger branch (equal spacing sums the axes first)."""
    from paper_2606_02053_gb300 import inputs

    n = (21, 14, 10)
    h = (1.0 / 21, 1.3 / 14, 0.9 / 10)
    p = C.make_params(slicing=0, shift=1, fluid=fluid, scalar=scalar, eta=1.1, ko_sigma=0.25, H0=2.0 * fluid)
    s = inputs.smooth_state(n, seed=31 + fluid, fluid=fluid, scalar=scalar)
    r, ref = run_rhs(C, O, n, h, p, s, t=0.02)
    assert field_errors(r, ref).max() <= RHS_TOL


@pytest.mark.parametrize("h", [0.1, (0.1, 0.07, 0.13)])
def test_flat_space_rhs_is_exactly_zero_both_ko_branches(C, O, h):
    n = (12, 9, 7)
    p = C.make_params(ko_sigma=0.3)
    s = np.zeros((24, n[2], n[1], n[0]))
    s[0] = 0.7
    s[1] = s[4] = s[6] = 1.0
    s[17] = 1.3
    s[18] = 0.2
    s[19] = -0.45
    r, _ = run_rhs(C, O, n, h, p, s)
    assert np.all(r == 0.0)


def test_flat_space_rhs_is_exactly_zero(C, O):
    n = (12, 9, 7)
    p = C.make_params()
    s = np.zeros((24, n[2], n[1], n[0]))
    s[0] = 0.7
    s[1] = s[4] = s[6] = 1.0
    s[17] = 1.3
    s[18] = 0.2
    r, _ = run_rhs(C, O, n, 0.1, p, s)
    assert np.all(r == 0.0)


@pytest.mark.parametrize("fluid", [0, 1])
def test_rk4_step_parity(C, O, fluid):
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    n = (24, 20, 18)
    h = 1.0 / 24
    p = C.make_params(fluid=fluid, H0=3.0 * fluid)
    s = inputs.smooth_state(n, seed=33 + fluid, fluid=fluid)
    ev = Evolution(C.make_grid(n, h), p)
    ev.set_state(s)
    ev.step(0.1, 0.25 * h, steps=2)
    ref = s.copy()
    O.evolve(O.OGrid(n, h), oracle_params(O, p), ref, 0.1, 0.25 * h, 2)
    assert field_errors(ev.get(), ref).max() <= STEP_TOL


@pytest.mark.parametrize("fluid,scalar,n,pitch", [(0, 0, (16, 16, 16), None), (1, 1, (21, 11, 13), 24),
                                                   (0, 0, (37, 9, 12), 40)])
def test_rk4_stage_entry_point_composes_to_step(C, fluid, scalar, n, pitch):
    """Four cosmos_rk4_stage calls (each scanning its stage state for the integer
    pass's exponents) equal one cosmos_rk4_step (stages 2-4 taking the exponents the
    previous algebra pass recorded), bitwise; so does the per-pass sequence with the
    record options, on ragged rows whose last warp is partly idle."""
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    h = 1.0 / n[0]
    p = C.make_params(fluid=fluid, scalar=scalar, H0=2.0 * fluid)
    s = inputs.smooth_state(n, seed=4, fluid=fluid, scalar=scalar, scale=0.5)
    a = Evolution(C.make_grid(n, h, pitch=pitch), p)
    a.set_state(s)
    a.step(0.0, 0.01)
    for options in (False, True):
        b = Evolution(C.make_grid(n, h, pitch=pitch), p)
        b.set_state(s)
        U1, U2, acc = (torch.empty_like(b.state) for _ in range(3))
        ws = b.ws_rhs
        opts = {(1, 1): 0, (1, 2): 96, (2, 1): 16, (2, 2): 32, (3, 1): 16, (3, 2): 32, (4, 1): 16, (4, 2): 0}
        for st, (src, dst) in enumerate([(b.state, U1), (U1, U2), (U2, U1), (U1, None)], start=1):
            if options:
                for pss in (0, 1, 2):
                    C.check(C.cosmos_stage_pass(b.g, b.p, pss + opts.get((st, pss), 0), st, src, b.state, dst, acc,
                                                0.0, 0.01, ws))
            else:
                C.check(C.cosmos_rk4_stage(b.g, b.p, st, src, b.state, dst, acc, 0.0, 0.01, ws))
        nx = n[0]
        assert torch.equal(a.view()[..., :nx], b.view()[..., :nx])
    # options only where they mean something
    b = Evolution(C.make_grid(n, h, pitch=pitch), p)
    U1, acc = torch.empty_like(b.state), torch.empty_like(b.state)
    for pss, st in ((0 + 16, 2), (2 + 16, 2), (1 + 32, 2), (2 + 32, 4), (2 + 128, 1)):
        assert C.cosmos_stage_pass(b.g, b.p, pss, st, b.state, b.state, U1, acc, 0.0, 0.01,
                                   b.ws_rhs) == C.COSMOS_EINVAL


def test_gauge_wave_32_cube_20_steps(C, O):
    """32^3 gauge wave, 1+log + Gamma-driver, dt = h/4, 20 steps."""
    from paper_2606_02053_gb300.evolve import Evolution

    n, h = 32, 1.0 / 32
    p = C.make_params(slicing=0, shift=1, eta=2.0, ko_sigma=0.1)
    ev = Evolution(C.make_grid(n, h), p)
    ev.init(C.make_id(0, A=0.01))
    op = oracle_params(O, p)
    og = O.OGrid((n, n, n), h)
    s0 = O.init(og, op, O.id_array(0, A=0.01))
    assert field_errors(ev.get(), s0).max() <= 1e-13
    ev.step(0.0, 0.25 * h, steps=20)
    # the data is independent of y and z, so the oracle runs on an n x 1 x 1 grid (bitwise the same)
    ot = O.OGrid((n, 1, 1), h)
    ref = O.init(ot, op, O.id_array(0, A=0.01))
    O.evolve(ot, op, ref, 0.0, 0.25 * h, 20)
    g = ev.get()
    assert field_errors(g[:, 7:8, 3:4, :], ref).max() <= STEP_TOL
    assert np.abs(g - g[:, :1, :1, :]).max() <= 1e-13  # y, z invariance kept


def test_gauge_wave_harmonic_closed_form_on_gpu(C):
    """Harmonic slicing, frozen shift: the gauge wave is exact; 4th order."""
    from paper_2606_02053_gb300.evolve import Evolution

    errs = []
    for n in (16, 32):
        h = 1.0 / n
        p = C.make_params(slicing=1, shift=0)
        ev = Evolution(C.make_grid((n, 4, 4), h), p)
        ev.init(C.make_id(0, A=0.01))
        steps = n
        ev.step(0.0, 0.25 * h, steps=steps)
        ex = Evolution(C.make_grid((n, 4, 4), h), p)
        ex.init(C.make_id(0, A=0.01, t=steps * 0.25 * h))
        errs.append(np.abs(ev.get() - ex.get()).max())
    assert 12 < errs[0] / errs[1] < 20, errs


def test_constraints_parity(C, O):
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    for fluid, scalar in [(0, 0), (1, 1)]:
        n = (18, 14, 10)
        h = 1.0 / 18
        p = C.make_params(fluid=fluid, scalar=scalar)
        s = inputs.smooth_state(n, seed=51, fluid=fluid, scalar=scalar)
        ev = Evolution(C.make_grid(n, h), p)
        ev.set_state(s)
        hm, norms = ev.constraints(want_fields=True)
        ref_hm, ref_norms = O.constraints(O.OGrid(n, h), oracle_params(O, p), s)
        assert field_errors(hm, ref_hm).max() <= RHS_TOL
        np.testing.assert_allclose(norms, ref_norms, rtol=1e-12)


def test_flrw_zeta_init_parity_and_constraints(C, O):
    from paper_2606_02053_gb300.evolve import Evolution

    n = 24
    h = 1.0 / n
    x0 = (-(n // 2) * h,) * 3
    p = C.make_params(fluid=1, w=1.0 / 3.0, H0=40.0)
    ev = Evolution(C.make_grid(n, h, x0=x0), p)
    ev.init(C.make_id(1, mu=0.5, sigma=0.125, q=(1.0, 0.9, 1.1)))
    og = O.OGrid((n, n, n), h, x0=x0)
    ref = O.init(og, oracle_params(O, p), O.id_array(1, mu=0.5, sigma=0.125, q=(1.0, 0.9, 1.1)))
    assert field_errors(ev.get(), ref).max() <= 1e-12
    hm, norms = ev.constraints(want_fields=True)
    assert np.abs(hm[0]).max() <= 1e-12 * 6.0 * 40.0 ** 2
    assert np.abs(hm[1:]).max() == 0.0


def test_flrw_zeta_evolution_parity_32(C, O):
    """Radiation FLRW + Gaussian zeta (mu = 0.5, sigma = L/8, H0 L = 40) at 32^3, 40 steps."""
    from paper_2606_02053_gb300.evolve import Evolution

    n = 32
    h = 1.0 / n
    x0 = (-(n // 2) * h,) * 3
    p = C.make_params(fluid=1, w=1.0 / 3.0, H0=40.0)
    ev = Evolution(C.make_grid(n, h, x0=x0), p)
    ev.init(C.make_id(1, mu=0.5, sigma=0.125))
    og = O.OGrid((n, n, n), h, x0=x0)
    op = oracle_params(O, p)
    ref = O.init(og, op, O.id_array(1, mu=0.5, sigma=0.125))
    dt = 0.25 * h
    ev.step(0.0, dt, steps=40)
    O.evolve(og, op, ref, 0.0, dt, 40)
    assert field_errors(ev.get(), ref).max() <= STEP_TOL


@pytest.mark.parametrize("fluid,scalar,n,pitch", [(0, 0, (37, 13, 11), 40), (1, 1, (20, 12, 5), None)])
def test_evolve_host_matches_device_steps(C, fluid, scalar, n, pitch):
    """Host-buffer path (copies overlapped with the passes, field groups in,
    plane slabs out) against cosmos_rk4_step on the device: bitwise."""
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    h = 1.0 / n[0]
    p = C.make_params(fluid=fluid, scalar=scalar, H0=2.0 * fluid)
    g = C.make_grid(n, h, pitch=pitch)
    ev = Evolution(g, p)
    ev.set_state(inputs.smooth_state(n, seed=77 + fluid, fluid=fluid, scalar=scalar, scale=0.5))
    U0 = ev.state.clone()
    dt = 0.25 * h
    for steps in (0, 1, 3):
        for pinned in (True, False):
            host_in = U0.cpu().pin_memory() if pinned else U0.cpu()
            host_out = torch.full_like(host_in, float("nan"))
            if pinned:
                host_out = host_out.pin_memory()
            dev = torch.empty_like(U0)
            C.check(C.cosmos_evolve_host(g, p, host_in, host_out, dev, steps, 0.01, dt, ev.ws_rk4))
            ev.state.copy_(U0)
            ev.step(0.01, dt, steps=steps)
            assert torch.equal(host_out, ev.state.cpu()), (steps, pinned)
            assert torch.equal(dev, ev.state), (steps, pinned)


@pytest.mark.parametrize("fluid,scalar,n,pitch", [(0, 0, (37, 13, 11), 40), (1, 1, (20, 12, 5), None)])
def test_pipelined_host_evolution_of_many_states_matches_device_steps(C, fluid, scalar, n, pitch):
    """cosmos_evolve_host_many: five different states (one of them given twice),
    each evolved from host memory through 1, 2 or 3 device buffers, equal bitwise
    to cosmos_rk4_step on the device; pinned and pageable host buffers; a result
    over an input buffer is refused."""
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    h = 1.0 / n[0]
    p = C.make_params(fluid=fluid, scalar=scalar, H0=2.0 * fluid)
    g = C.make_grid(n, h, pitch=pitch)
    ev = Evolution(g, p)
    states = []
    for q in range(4):
        ev.set_state(inputs.smooth_state(n, seed=90 + q + 10 * fluid, fluid=fluid, scalar=scalar, scale=0.5))
        states.append(ev.state.clone())
    states.append(states[1])  # the same inputs again
    dt = 0.25 * h
    want = {}
    for steps in (0, 1, 2):
        for q in range(4):
            ev.state.copy_(states[q])
            ev.step(0.01, dt, steps=steps)
            want[steps, q] = ev.state.cpu()
    for steps in (1, 2, 0):
        for nbuf in (1, 2, 3):
            for pinned in (True, False):
                ins = [x.cpu().pin_memory() if pinned else x.cpu() for x in states]
                outs = [torch.full_like(ins[0], float("nan")) for _ in states]
                if pinned:
                    outs = [o.pin_memory() for o in outs]
                devs = [torch.empty_like(states[0]) for _ in range(nbuf)]
                C.check(C.cosmos_evolve_host_many(g, p, ins, outs, devs, steps, 0.01, dt, ev.ws_rk4))
                for i, o in enumerate(outs):
                    assert torch.equal(o, want[steps, i if i < 4 else 1]), (steps, nbuf, pinned, i)
    ins = [states[0].cpu().pin_memory(), states[1].cpu().pin_memory()]
    devs = [torch.empty_like(states[0]) for _ in range(2)]
    assert C.cosmos_evolve_host_many(g, p, ins, [ins[1], ins[0]], devs, 1, 0.0, dt, ev.ws_rk4) == C.COSMOS_EINVAL


def test_isocurvature_init_and_evolution_parity(C, O):
    """FLRW + zeta + massless-scalar isocurvature data (id kind 2) and 20 RK4
    steps of the fluid + scalar system against the oracle."""
    from paper_2606_02053_gb300.evolve import Evolution

    n = 24
    h = 1.0 / n
    x0 = (-(n // 2) * h,) * 3
    p = C.make_params(fluid=1, scalar=1, w=1.0 / 3.0, H0=40.0)
    ev = Evolution(C.make_grid(n, h, x0=x0), p)
    kw = dict(A=0.02, mu=0.3, sigma=0.125, q=(1.0, 0.9, 1.1))
    ev.init(C.make_id(2, **kw))
    og = O.OGrid((n, n, n), h, x0=x0)
    op = oracle_params(O, p)
    ref = O.init(og, op, O.id_array(2, **kw))
    assert field_errors(ev.get(), ref).max() <= 1e-12
    hm, _ = ev.constraints(want_fields=True)
    assert np.abs(hm[0]).max() <= 1e-12 * 6.0 * 40.0 ** 2
    assert np.abs(hm[1:]).max() == 0.0
    dt = 0.25 * h
    ev.step(0.0, dt, steps=20)
    O.evolve(og, op, ref, 0.0, dt, 20)
    assert field_errors(ev.get(), ref).max() <= STEP_TOL
    pv = C.make_params(fluid=1, scalar=0, H0=40.0)
    evv = Evolution(C.make_grid(n, h, x0=x0), pv)
    assert C.cosmos_init_grid(evv.g, pv, C.make_id(2, **kw), evv.state, evv.ws_init) == C.COSMOS_EINVAL


def test_single_mode_on_gpu_follows_linear_theory(C, O):
    """The single-mode FLRW perturbation of test_oracle_linear_mode on the GPU
    (N = 64 line): mode amplitudes equal the oracle's to 1e-6 of the mode and
    follow linear theory as the oracle does."""
    import test_oracle_linear_mode as LM
    from paper_2606_02053_gb300.evolve import Evolution

    n = 64
    h = 1.0 / n
    p = C.make_params(slicing=1, shift=0, ko_sigma=0.0, fluid=1, w=LM.W, H0=LM.H0)
    ev = Evolution(C.make_grid((n, 1, 1), h), p)
    s = np.zeros((28, 1, 1, n))
    x = h * np.arange(n)
    s[0] = 1.0
    s[1] = s[4] = s[6] = 1.0
    s[7] = -3.0 * LM.H0
    s[17] = 1.0 + LM.EPS * np.cos(2.0 * np.pi * x)
    s[24] = 3.0 * LM.H0 ** 2 / (8.0 * np.pi)
    ev.set_state(s)
    phase = np.exp(-2j * np.pi * x) * (2.0 / n)
    dt = 0.25 * h
    steps = int(round(LM.T_END / dt))
    times, amps = [0.0], [[s[f, 0, 0] @ phase for _, f, _, _ in LM.COMPARED]]
    for m in range(steps):
        ev.step(m * dt, dt)
        if (m + 1) % 8 == 0:
            g = ev.get()
            times.append((m + 1) * dt)
            amps.append([g[f, 0, 0] @ phase for _, f, _, _ in LM.COMPARED])
    t, amps = np.array(times), np.array(amps).T
    t_o, amps_o = LM.oracle_modes(O, n, 8)
    assert np.array_equal(t, t_o)
    for (name, _, _, _), a, b in zip(LM.COMPARED, amps, amps_o):
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), name
    errs = LM.mode_errors(t, amps, 2.0 * np.pi)
    assert max(errs.values()) < 5e-3, errs


def test_invalid_arguments_launch_nothing(C):
    from paper_2606_02053_gb300.evolve import Evolution

    g = C.make_grid((16, 16, 16), 0.0625)
    p = C.make_params()
    ev = Evolution(g, p)
    out = torch.empty_like(ev.state)
    assert C.cosmos_rhs(g, p, ev.state, ev.state, 0.0) == C.COSMOS_EINVAL  # aliasing
    small = torch.empty(16, dtype=torch.float64, device="cuda")
    pf = C.make_params(fluid=1)
    evf = Evolution(g, pf)
    assert C.cosmos_rhs(g, pf, evf.state, torch.empty_like(evf.state), 0.0, small) == C.COSMOS_EWORKSPACE
    assert C.cosmos_rk4_stage(g, p, 5, ev.state, ev.state, out, out, 0.0, 0.1) == C.COSMOS_EINVAL
    assert C.cosmos_init_grid(g, pf, C.make_id(0, A=0.01), evf.state, evf.ws_init) == C.COSMOS_EINVAL


@pytest.mark.parametrize("fluid", [0, 1])
def test_runs_are_deterministic_and_stream_independent(C, fluid):
    """Two runs from the same state give bitwise the same result, on the
    default stream and on a side stream (no atomics, fixed reduction order)."""
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    n = (40, 24, 20)
    h = 1.0 / 40
    p = C.make_params(fluid=fluid, H0=2.0 * fluid)
    ev = Evolution(C.make_grid(n, h), p)
    s0 = inputs.smooth_state(n, seed=123 + fluid, fluid=fluid, scale=0.5)
    outs, norms = [], []
    side = torch.cuda.Stream()
    for stream in (None, side, None):
        ev.set_state(s0)
        torch.cuda.synchronize()  # the state copy (default stream) lands before the side stream starts
        with torch.cuda.stream(side if stream is side else torch.cuda.current_stream()):
            for m in range(3):
                C.check(C.cosmos_rk4_step(ev.g, p, ev.state, m * 0.25 * h, 0.25 * h, ev.ws_rk4,
                                          torch.cuda.current_stream()))
            norms.append(ev.constraints()[1])
        torch.cuda.synchronize()
        outs.append(ev.state.clone())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    assert np.array_equal(norms[0], norms[1]) and np.array_equal(norms[0], norms[2])


def test_rk4_steps_capture_into_a_cuda_graph(C):
    """cosmos_rk4_step launches only kernels on the given stream (no
    allocation, no synchronisation), so a sequence of steps can be captured
    into a CUDA graph; replaying it equals calling the steps directly."""
    from paper_2606_02053_gb300.evolve import Evolution

    n, h = 32, 1.0 / 32
    p = C.make_params(slicing=0, shift=1)
    ev = Evolution(C.make_grid(n, h), p)
    ev.init(C.make_id(0, A=0.01))
    U0 = ev.state.clone()
    dt = 0.25 * h
    ev.step(0.0, dt, steps=5)
    direct = ev.state.clone()
    ev.state.copy_(U0)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=s):
        for m in range(5):
            C.check(C.cosmos_rk4_step(ev.g, p, ev.state, m * dt, dt, ev.ws_rk4, s))
    ev.state.copy_(U0)
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(ev.state, direct)


@pytest.mark.parametrize("ko", [0.0, 0.2])
def test_fluid_totals_are_conserved_on_a_flat_background(C, ko):
    """On a flat, static background the fluid right-hand side is the
    divergence of the face fluxes (each face computed once) plus the KO term,
    so its grid sums vanish to rounding for any physical fluid state."""
    from paper_2606_02053_gb300.evolve import Evolution

    n = (37, 13, 11)
    p = C.make_params(slicing=0, shift=1, ko_sigma=ko, w=1.0 / 3.0, fluid=1)
    s = np.zeros((28, n[2], n[1], n[0]))
    s[0] = 1.0
    s[1] = s[4] = s[6] = 1.0
    s[17] = 1.0
    rng = np.random.default_rng(79)
    E = 1.0 + 0.5 * rng.random((n[2], n[1], n[0]))
    s[24] = E
    s[25:28] = 0.4 * (rng.random((3, n[2], n[1], n[0])) - 0.5) * E
    ev = Evolution(C.make_grid(n, 1.0 / n[0], pitch=40), p)
    ev.set_state(s)
    r = ev.get(ev.rhs(0.0))
    for f in range(24, 28):
        total, scale = r[f].sum(), np.abs(r[f]).sum()
        assert scale > 1.0 and abs(total) <= 1e-13 * scale, (f, total, scale)

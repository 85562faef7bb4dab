"""Reverse mode on the GPU against the oracle's tape and against finite differences."""

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


def rel_err(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    den = np.maximum(np.abs(b).max(axis=1), 1e-12 * np.abs(b).max())
    return (np.abs(a - b).max(axis=1) / den).max()


def ws(C, g, p, op):
    nb = C.cosmos_adjoint_workspace_bytes(g, p, op)
    return torch.empty((nb + 7) // 8, dtype=torch.float64, device="cuda")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda().reshape(-1)


MATTER = [(0, 0), (1, 0), (0, 1), (1, 1)]  # (fluid, scalar)


@pytest.mark.parametrize("fluid,scalar", MATTER)
def test_rhs_vjp_matches_oracle_tape(C, O, fluid, scalar):
    from paper_2606_02053_gb300 import inputs

    n = (9, 8, 7)
    h = 1.0 / 9
    kw = dict(slicing=0, shift=1, eta=1.3, ko_sigma=0.2, fluid=fluid, scalar=scalar, H0=2.0 * fluid)
    p = C.make_params(**kw)
    g = C.make_grid(n, h)
    U = inputs.smooth_state(n, seed=60 + fluid + 2 * scalar, fluid=fluid, scalar=scalar, scale=0.5)
    w = np.random.default_rng(7).standard_normal(U.shape)
    v = torch.empty_like(dev(U))
    C.check(C.cosmos_rhs_vjp(g, p, dev(U), dev(w), v, 0.1, ws(C, g, p, C.COSMOS_OP_VJP)))
    ref = O.rhs_vjp(O.OGrid(n, h), O.params_array(**kw), U, w, 0.1)
    assert rel_err(v.cpu().numpy().reshape(U.shape), ref) <= 1e-10


@pytest.mark.parametrize("fluid,scalar", MATTER)
def test_adjoint_step_matches_oracle(C, O, fluid, scalar):
    from paper_2606_02053_gb300 import inputs

    n = (8, 7, 7)
    h = 1.0 / 8
    kw = dict(slicing=0, shift=1, eta=1.0, ko_sigma=0.1, fluid=fluid, scalar=scalar, H0=2.0 * fluid)
    p = C.make_params(**kw)
    g = C.make_grid(n, h)
    U = inputs.smooth_state(n, seed=70 + fluid + 2 * scalar, fluid=fluid, scalar=scalar, scale=0.5)
    lam = np.random.default_rng(8).standard_normal(U.shape)
    out = torch.empty_like(dev(U))
    dt = 0.25 * h
    C.check(C.cosmos_adjoint_step(g, p, dev(U), dev(lam), out, 0.05, dt, ws(C, g, p, C.COSMOS_OP_ADJOINT)))
    op = O.params_array(**kw)
    ref = O.adjoint_step(O.OGrid(n, h), op, U, lam, 0.05, dt)
    assert rel_err(out.cpu().numpy().reshape(U.shape), ref) <= 1e-10
    # in place (lam_n = lam_np1) gives the same result
    lam_d = dev(lam)
    C.check(C.cosmos_adjoint_step(g, p, dev(U), lam_d, lam_d, 0.05, dt, ws(C, g, p, C.COSMOS_OP_ADJOINT)))
    assert torch.equal(lam_d, out)


@pytest.mark.parametrize("case", ["smooth_fluid_24", "gauge_wave_32"])
def test_adjoint_step_dot_product(C, case):
    """<lam, dPhi v> by central differences of the GPU step vs <Phi'^T lam, v>
    at sizes beyond the oracle's reach.  States are generic: a fluid near rest
    puts minmod slopes and the pair of sound speeds on kinks of the discrete
    map, where no derivative exists (the FLRW scan data start exactly there)."""
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    if case == "smooth_fluid_24":
        n = 24
        h = 1.0 / n
        p = C.make_params(fluid=1, w=1.0 / 3.0, H0=2.0)
        ev = Evolution(C.make_grid(n, h), p)
        ev.set_state(inputs.smooth_state(n, seed=90, fluid=1, scale=0.5))
    else:
        n = 32
        h = 1.0 / n
        p = C.make_params(slicing=0, shift=1)
        ev = Evolution(C.make_grid(n, h), p)
        ev.init(C.make_id(0, A=0.01))
    U = ev.state.clone()
    rng = np.random.default_rng(9)
    v = torch.from_numpy(rng.standard_normal(U.numel())).cuda() * U.abs().clamp(min=1e-2)
    lam = torch.from_numpy(rng.standard_normal(U.numel())).cuda()
    dt = 0.25 * h
    adj = torch.empty_like(U)
    C.check(C.cosmos_adjoint_step(ev.g, p, U, lam, adj, 0.0, dt, ws(C, ev.g, p, C.COSMOS_OP_ADJOINT)))
    rhs = float(torch.dot(adj, v))
    best = None
    for e in (1e-7, 5e-8, 2.5e-8):
        outs = []
        for sgn in (1, -1):
            ev.state.copy_(U + sgn * e * v)
            ev.step(0.0, dt)
            outs.append(ev.state.clone())
        lhs = float(torch.dot(lam, (outs[0] - outs[1]) / (2 * e)))
        best = lhs if best is None or abs(lhs - rhs) < abs(best - rhs) else best
    assert abs(best - rhs) <= 1e-7 * abs(rhs), (best, rhs)


def test_init_zeta_matches_gaussian_init_and_its_vjp(C):
    n = 20
    h = 1.0 / n
    x0 = -(n // 2) * h
    p = C.make_params(fluid=1, w=1.0 / 3.0, H0=20.0)
    g = C.make_grid(n, h, x0=(x0,) * 3)
    x = x0 + h * torch.arange(n, dtype=torch.float64, device="cuda")
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    zeta = (0.5 * torch.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * 0.14 ** 2))).reshape(-1).contiguous()
    nf = 28
    a = torch.empty(nf * n ** 3, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    wsi = torch.empty((C.cosmos_workspace_bytes(g, p, C.COSMOS_OP_INIT) + 7) // 8, dtype=torch.float64,
                      device="cuda")
    C.check(C.cosmos_init_zeta(g, p, zeta, 1.0, a, wsi))
    C.check(C.cosmos_init_grid(g, p, C.make_id(1, mu=0.5, sigma=0.14), b, wsi))
    assert float((a - b).abs().max() / b.abs().max()) <= 1e-13
    # reverse of the initial-data map vs central differences
    rng = np.random.default_rng(10)
    lam = torch.from_numpy(rng.standard_normal(a.numel())).cuda()
    dz = torch.from_numpy(rng.standard_normal(zeta.numel())).cuda()
    zbar = torch.empty_like(zeta)
    C.check(C.cosmos_init_zeta_vjp(g, p, a, lam, zbar, ws(C, g, p, C.COSMOS_OP_INIT_VJP)))
    e = 1e-6
    C.check(C.cosmos_init_zeta(g, p, (zeta + e * dz).contiguous(), 1.0, a, wsi))
    C.check(C.cosmos_init_zeta(g, p, (zeta - e * dz).contiguous(), 1.0, b, wsi))
    lhs = float(torch.dot(lam, (a - b) / (2 * e)))
    rhs = float(torch.dot(zbar, dz))
    assert abs(lhs - rhs) <= 1e-7 * abs(rhs), (lhs, rhs)


def test_compaction_definition_and_vjp(C, O):
    from paper_2606_02053_gb300.evolve import Evolution

    n = 24
    h = 1.0 / n
    p = C.make_params(fluid=1, w=1.0 / 3.0, H0=20.0)
    ev = Evolution(C.make_grid(n, h, x0=(-(n // 2) * h,) * 3), p)
    ev.init(C.make_id(1, mu=0.7, sigma=0.12, q=(1.0, 0.9, 1.1)))
    ev.step(0.0, 0.25 * h, steps=4)
    kmax = n // 2 - 1
    wsd = ws(C, ev.g, p, C.COSMOS_OP_DIAG)
    code, Ck, aux = C.cosmos_compaction(ev.g, p, ev.state, kmax, wsd)
    C.check(code)
    og = O.OGrid((n, n, n), h, x0=(-(n // 2) * h,) * 3)
    op = O.params_array(fluid=1, w=1.0 / 3.0, H0=20.0)
    ref = O.compaction(og, op, ev.get(), kmax)
    np.testing.assert_allclose(Ck, ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())
    kstar = int(np.argmax(Ck)) + 1
    lam = torch.empty_like(ev.state)
    C.check(C.cosmos_compaction_vjp(ev.g, p, ev.state, kstar, kmax, aux, 1.0, lam))
    U = ev.state.clone()
    dv = torch.from_numpy(np.random.default_rng(11).standard_normal(U.numel())).cuda() * U.abs()
    e = 1e-7
    vals = []
    for sgn in (1, -1):
        code, Cs, _ = C.cosmos_compaction(ev.g, p, (U + sgn * e * dv).contiguous(), kmax, wsd)
        vals.append(Cs[kstar - 1])
    lhs = (vals[0] - vals[1]) / (2 * e)
    rhs = float(torch.dot(lam, dv))
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs), (lhs, rhs)
    # the reverse mode equals the oracle's tape of the same function
    ref_lam = O.compaction_vjp(og, op, ev.get(), kmax, kstar, 1.0)
    assert rel_err(ev.get(lam), ref_lam) <= 1e-10


def test_checkpointed_gradient_matches_finite_differences_in_mu(C):
    from paper_2606_02053_gb300.adjoint import CollapseRun, CosmosAdjoint

    n = 20
    h = 1.0 / n
    p = C.make_params(fluid=1, w=1.0 / 3.0, H0=20.0)
    run = CollapseRun(n, p, dt=0.25 * h, steps=12, checkpoint_every=5)
    x = (-(n // 2) + torch.arange(n, dtype=torch.float64, device="cuda")) * h
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    shape = torch.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * 0.14 ** 2)).reshape(-1)
    mu = torch.tensor(0.6, dtype=torch.float64, device="cuda", requires_grad=True)
    out = CosmosAdjoint.apply((mu * shape).contiguous(), run)
    gmin, = torch.autograd.grad(out[0], mu, retain_graph=True)
    gcomp, = torch.autograd.grad(out[1], mu)
    hmu = 1e-6
    plus = run.forward((0.6 + hmu) * shape)[:2]
    minus = run.forward((0.6 - hmu) * shape)[:2]
    fd_min = (plus[0] - minus[0]) / (2 * hmu)
    fd_comp = (plus[1] - minus[1]) / (2 * hmu)
    assert abs(float(gmin) - fd_min) <= 1e-6 * abs(fd_min), (float(gmin), fd_min)
    assert abs(float(gcomp) - fd_comp) <= 1e-6 * abs(fd_comp), (float(gcomp), fd_comp)


@pytest.mark.parametrize("fluid,scalar", [(0, 0), (1, 1)])
def test_saved_stage_states_give_the_same_step_and_adjoint(C, fluid, scalar):
    """cosmos_rk4_step_stages = cosmos_rk4_step (bitwise), its stage states are
    those of the fused stages, and cosmos_adjoint_step_stages on them =
    cosmos_adjoint_step (bitwise)."""
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    n = (20, 14, 12)
    h = 1.0 / n[0]
    p = C.make_params(fluid=fluid, scalar=scalar, H0=2.0 * fluid)
    ev = Evolution(C.make_grid(n, h, pitch=24), p)
    ev.set_state(inputs.smooth_state(n, seed=5 + fluid, fluid=fluid, scalar=scalar, scale=0.5))
    U0 = ev.state.clone()
    t, dt = 0.03, 0.25 * h
    ev.step(t, dt)
    ref = ev.state.clone()
    st = U0.clone()
    U2, U3, U4 = (torch.empty_like(st) for _ in range(3))
    C.check(C.cosmos_rk4_step_stages(ev.g, p, st, t, dt, U2, U3, U4, ev.ws_rk4))
    assert torch.equal(st, ref)
    # stage 1 of the fused stages writes U2 from U_n
    A, acc = torch.empty_like(st), torch.empty_like(st)
    C.check(C.cosmos_rk4_stage(ev.g, p, 1, U0, U0.clone(), A, acc, t, dt, ev.ws_rhs))
    nx = ev.g.nx  # rows are padded to a pitch of 24; the padding is never written
    assert torch.equal(ev.view(A)[..., :nx], ev.view(U2)[..., :nx])
    lam = torch.from_numpy(np.random.default_rng(3).standard_normal(U0.numel())).cuda()
    a = torch.empty_like(lam)
    b = torch.empty_like(lam)
    wsa = ws(C, ev.g, p, C.COSMOS_OP_ADJOINT)
    C.check(C.cosmos_adjoint_step(ev.g, p, U0, lam, a, t, dt, wsa))
    C.check(C.cosmos_adjoint_step_stages(ev.g, p, U0, U2, U3, U4, lam, b, t, dt, wsa))
    assert torch.equal(a, b)
    assert C.cosmos_adjoint_step_stages(ev.g, p, U0, U2, U3, U4, lam, U2, t, dt, wsa) == C.COSMOS_EINVAL
    assert C.cosmos_rk4_step_stages(ev.g, p, st, t, dt, U2, U2, U4, ev.ws_rk4) == C.COSMOS_EINVAL


def test_series_argmin_takes_the_first_minimum(C):
    res = torch.empty(2, dtype=torch.float64, device="cuda")
    cases = [
        [3.0],
        [2.0, 1.0, 1.0, 5.0],
        [float("nan"), 4.0, 2.0, float("nan"), 2.0],
        [float("nan"), float("nan")],
        list(np.cos(np.arange(100) * 0.37)) + [-1.0] * 3,
        [1.0] * 70 + [0.5] + [0.5] * 40,
    ]
    for v in cases:
        a = torch.tensor(v, dtype=torch.float64, device="cuda")
        C.check(C.cosmos_series_argmin(a, len(v), res))
        m, i = res.cpu().tolist()
        finite = [x for x in v if x == x]
        if finite:
            assert m == min(finite) and int(i) == v.index(min(finite)), (v, m, i)
        else:
            assert m != m and int(i) == 0
    assert C.cosmos_series_argmin(a, 0, res) == C.COSMOS_EINVAL


def collapse_case(C, O, n, steps, every, zeta_np, H0=20.0):
    """GPU CollapseRun + CosmosAdjoint against the oracle's pipeline on the same zeta:
    forward values, the selected level / radius, and both zeta gradients point by point."""
    from paper_2606_02053_gb300.adjoint import CollapseRun, CosmosAdjoint

    h = 1.0 / n
    p = C.make_params(fluid=1, w=1.0 / 3.0, H0=H0)
    run = CollapseRun(n, p, dt=0.25 * h, steps=steps, checkpoint_every=every)
    zeta = torch.from_numpy(zeta_np.reshape(-1).copy()).cuda().requires_grad_(True)
    out = CosmosAdjoint.apply(zeta, run)
    g_lapse, = torch.autograd.grad(out[0], zeta, retain_graph=True)
    g_comp, = torch.autograd.grad(out[1], zeta)
    og = O.OGrid((n, n, n), h, x0=(-(n // 2) * h,) * 3)
    op = O.params_array(fluid=1, w=1.0 / 3.0, H0=H0)
    ra, rc, r = O.collapse_gradient(og, op, zeta_np, 0.25 * h, steps, n // 2 - 1)
    out = out.detach()
    assert abs(float(out[0]) - r["min_lapse"]) <= 1e-12 * abs(r["min_lapse"])
    assert abs(float(out[1]) - r["peak"]) <= 1e-10 * abs(r["peak"])
    for got, ref in ((g_lapse, ra), (g_comp, rc)):
        got = got.cpu().numpy().reshape(n, n, n)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= 1e-10, err
    return r


def test_collapse_gradients_match_the_oracle_tape_end_to_end(C, O):
    """init(zeta) -> 8 RK4 steps with checkpoints every 3 -> (min central lapse, peak
    compaction), reversed by the library, against the oracle's own tape of the same
    pipeline at every grid point (generic data: an off-centre anisotropic bump plus
    seeded noise, so the discrete map is differentiable there)."""
    n = 10
    h = 1.0 / n
    x = (-(n // 2) + np.arange(n)) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r2 = ((X - 0.013) / 1.0) ** 2 + ((Y + 0.021) / 0.9) ** 2 + ((Z - 0.007) / 1.1) ** 2
    zeta = 0.6 * np.exp(-r2 / (2 * 0.16 ** 2)) + 0.01 * np.random.default_rng(12).standard_normal((n, n, n))
    r = collapse_case(C, O, n, 8, 3, zeta)
    assert 0 < r["nstar"] <= 8  # the minimum lies after the initial level


def test_collapse_gradients_from_a_fluid_at_rest_match_the_oracle_tape(C, O):
    """The configurations' data: a centred Gaussian zeta, the fluid exactly at rest.
    h = 1/8 keeps the mirror symmetry bitwise on both sides, so the velocity vanishes
    exactly on the symmetry planes; there the discrete map has kinks along single-point
    zeta directions (tests/test_oracle_diagnostics.py shows the one-sided differences
    disagree).  The library's reverse mode takes the same branch as the oracle's tape
    at every tie, so the two gradients agree point by point."""
    n = 8
    h = 1.0 / n
    x = (-(n // 2) + np.arange(n)) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    zeta = 0.6 * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * 0.15 ** 2))
    collapse_case(C, O, n, 4, 2, zeta)


def test_one_sweep_for_both_diagnostics_equals_two(C):
    """backward_many replays each checkpoint segment once for several cotangent pairs;
    each zeta_bar is bitwise the one a separate sweep gives."""
    from paper_2606_02053_gb300.adjoint import CollapseRun

    n = 12
    h = 1.0 / n
    run = CollapseRun(n, C.make_params(fluid=1, w=1.0 / 3.0, H0=20.0), dt=0.25 * h, steps=7, checkpoint_every=3)
    x = (-(n // 2) + torch.arange(n, dtype=torch.float64, device="cuda")) * h
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    zeta = (0.6 * torch.exp(-((X - 0.01) ** 2 + Y ** 2 + Z ** 2) / (2 * 0.15 ** 2))).reshape(-1).contiguous()
    _, _, rec = run.forward(zeta)
    pairs = [(1.0, 0.0), (0.0, 1.0), (0.3, -2.0)]
    many = run.backward_many(rec, pairs)
    for (ga, gc), zb in zip(pairs, many):
        assert torch.equal(zb, run.backward(rec, ga, gc))

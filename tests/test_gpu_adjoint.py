"""Reverse mode on the GPU against the oracle's tape and against finite differences."""
import ctypes

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


def compaction_numpy(U, n, h, kmax):
    """The compaction function as defined in include/cosmos.h, in plain numpy."""
    chi = U[0]
    tau = U[24]
    sg = chi ** -1.5
    c = n // 2
    idx = np.arange(n) - c
    m = idx[:, None, None] ** 2 + idx[None, :, None] ** 2 + idx[None, None, :] ** 2
    Ebar = tau.sum() / sg.sum()
    out = []
    for k in range(1, kmax + 1):
        inside = m < k * k
        dM = h ** 3 * (tau[inside].sum() - Ebar * sg[inside].sum())
        axis = [chi[c, c, c + k], chi[c, c, c - k], chi[c, c + k, c], chi[c, c - k, c], chi[c + k, c, c],
                chi[c - k, c, c]]
        R = k * h * np.mean([a ** -0.5 for a in axis])
        out.append(2 * dM / R)
    return np.array(out)


def test_compaction_definition_and_vjp(C):
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
    ref = compaction_numpy(ev.get(), n, h, kmax)
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

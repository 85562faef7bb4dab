"""Pins of the CPU oracle against what the mathematics fixes (no GPU).

Each test names the property it pins and the mistake it would catch.
"""

import numpy as np
import pytest

from paper_2606_02053_gb300 import inputs

CHI, GT, TRK, AT, GAM, ALP, BET, BB = 0, 1, 7, 8, 14, 17, 18, 21
SYM = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def flat_state(O, n, params, chi=1.0, alpha=1.0, beta=(0.0, 0.0, 0.0)):
    nf = O.nfields(params)
    s = np.zeros((nf, n[2], n[1], n[0]))
    s[CHI] = chi
    s[GT + 0] = s[GT + 3] = s[GT + 5] = 1.0
    s[ALP] = alpha
    for d in range(3):
        s[BET + d] = beta[d]
    return s


# ---------------------------------------------------------------------------
# P1: flat space has an identically zero right-hand side (bitwise)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("slicing,shift", [(0, 1), (1, 0), (0, 0), (1, 1)])
def test_flat_space_rhs_is_exactly_zero(O, slicing, shift):
    n = (8, 7, 6)
    g = O.OGrid(n, (0.125, 0.11, 0.09))
    P = O.params_array(slicing=slicing, shift=shift, ko_sigma=0.1)
    for chi, alpha, beta in [(1.0, 1.0, (0, 0, 0)), (0.7, 1.3, (0.2, -0.1, 0.05)), (2.5, 0.4, (0, 0.3, 0))]:
        s = flat_state(O, n, P, chi, alpha, beta)
        r = O.rhs(g, P, s)
        assert np.all(r == 0.0), np.abs(r).max()


def test_flat_space_with_scalar_at_rest_is_zero(O):
    n = (6, 6, 6)
    g = O.OGrid(n, 1 / 6)
    P = O.params_array(scalar=1)
    s = flat_state(O, n, P, 0.9, 1.1)
    s[24] = 0.37  # constant phi, Pi = 0
    assert np.all(O.rhs(g, P, s) == 0.0)


# ---------------------------------------------------------------------------
# P2: Fourier symbols of the 4th-order first/second derivative, the mixed
# derivative and the 6th-derivative Kreiss-Oliger operator.
#   state: flat, frozen shift, beta^x = eps sin(tx i + ty j)
#   d_t chi    = -2/3 D_x beta^x
#   d_t Gt^x   = (D_xx + D_yy) beta^x + 1/3 D_xx beta^x
#   d_t Gt^y   = 1/3 D_y D_x beta^x
#   d_t beta^x = KO beta^x
# ---------------------------------------------------------------------------
def test_fourier_symbols(O):
    n = (16, 16, 8)
    h = 1.0 / 16
    g = O.OGrid(n, h)
    sig = 0.1
    P = O.params_array(slicing=1, shift=0, ko_sigma=sig)
    s = flat_state(O, n, P)
    tx, ty = 2 * np.pi * 3 / 16, 2 * np.pi * 2 / 16
    eps = 1e-3
    i = np.arange(16)[None, None, :]
    j = np.arange(16)[None, :, None]
    ph = tx * i + ty * j + 0 * np.arange(8)[:, None, None]
    s[BET] = eps * np.sin(ph)
    r = O.rhs(g, P, s)

    def s1(t):
        return (8 * np.sin(t) - np.sin(2 * t)) / (6 * h)

    def s2(t):
        return -(15 - 16 * np.cos(t) + np.cos(2 * t)) / (6 * h * h)

    def ko(t):
        return -(sig / h) * np.sin(t / 2) ** 6

    Dx = eps * s1(tx) * np.cos(ph)
    Dxx = eps * s2(tx) * np.sin(ph)
    Dyy = eps * s2(ty) * np.sin(ph)
    Dxy = -eps * s1(tx) * s1(ty) * np.sin(ph)
    KOb = eps * (ko(tx) + ko(ty)) * np.sin(ph)
    tol = 1e-13
    np.testing.assert_allclose(r[CHI], -2.0 / 3.0 * Dx, rtol=0, atol=tol * np.abs(Dx).max())
    np.testing.assert_allclose(r[GT + 0], 4.0 / 3.0 * Dx, rtol=0, atol=tol * np.abs(Dx).max())
    np.testing.assert_allclose(r[GAM], Dxx + Dyy + Dxx / 3.0, rtol=0, atol=tol * np.abs(Dxx).max())
    np.testing.assert_allclose(r[GAM + 1], Dxy / 3.0, rtol=0, atol=tol * np.abs(Dxy).max())
    np.testing.assert_allclose(r[BET], KOb, rtol=0, atol=1e-11 * np.abs(KOb).max())
    assert np.all(r[GAM + 2] == 0.0)


# ---------------------------------------------------------------------------
# P3: translation invariance (bitwise) and x<->y axis permutation symmetry.
# A wrong index in any contraction breaks the permutation check.
# ---------------------------------------------------------------------------
def _perm_xy(s, fluid, scalar):
    """Swap the x and y axes of a state: grid axes and tensor components."""
    t = s.transpose(0, 1, 3, 2).copy()
    out = t.copy()
    # symmetric tensors: xx<->yy, xz<->yz, xy, zz fixed
    for base in (GT, AT):
        out[base + 0], out[base + 3] = t[base + 3], t[base + 0]
        out[base + 2], out[base + 4] = t[base + 4], t[base + 2]
    for base in (GAM, BET, BB):
        out[base + 0], out[base + 1] = t[base + 1], t[base + 0]
    if fluid:
        out[25], out[26] = t[26], t[25]
    return out


@pytest.mark.parametrize("fluid,scalar", [(0, 0), (1, 1)])
def test_translation_and_axis_permutation(O, fluid, scalar):
    n = (12, 12, 10)
    g = O.OGrid(n, 1.0 / 12)
    P = O.params_array(slicing=0, shift=1, fluid=fluid, scalar=scalar)
    s = inputs.smooth_state(n, seed=11, fluid=fluid, scalar=scalar)
    r = O.rhs(g, P, s)
    r_roll = O.rhs(g, P, np.ascontiguousarray(np.roll(s, 1, axis=3)))
    assert np.array_equal(r_roll, np.roll(r, 1, axis=3))
    r_roll = O.rhs(g, P, np.ascontiguousarray(np.roll(s, -2, axis=1)))
    assert np.array_equal(r_roll, np.roll(r, -2, axis=1))
    sp = _perm_xy(s, fluid, scalar)
    rp = O.rhs(g, P, sp)
    expect = _perm_xy(r, fluid, scalar)
    scale = np.abs(expect).max(axis=(1, 2, 3), keepdims=True) + 1e-300
    assert (np.abs(rp - expect) / scale).max() < 1e-12


# ---------------------------------------------------------------------------
# P4: gauge wave.  ds^2 = -H dt^2 + H dx^2 + dy^2 + dz^2, H = 1 - A sin(2pi(x-t)/L)
# is flat spacetime; with harmonic slicing and zero shift it is an exact
# solution.  Its BSSN variables are written out here from the metric.
# ---------------------------------------------------------------------------
def gauge_wave_exact(n, h, t, A):
    L = n * h
    x = np.arange(n) * h
    ph = 2 * np.pi * (x - t) / L
    H = 1 - A * np.sin(ph)
    dtH = A * 2 * np.pi / L * np.cos(ph)
    dxH = -dtH
    Kxx = -dtH / (2 * np.sqrt(H))  # K_ij = -d_t gamma_ij / (2 alpha), alpha = sqrt(H)
    trK = Kxx / H
    chi = H ** (-1.0 / 3.0)  # det gamma = H
    v = np.zeros((24, n))
    v[CHI] = chi
    v[GT + 0] = chi * H
    v[GT + 3] = v[GT + 5] = chi
    v[TRK] = trK
    v[AT + 0] = chi * (Kxx - H * trK / 3)
    v[AT + 3] = v[AT + 5] = chi * (-trK / 3)
    v[GAM + 0] = (2.0 / 3.0) * H ** (-5.0 / 3.0) * dxH  # = -d_x gt^xx with gt^xx = H^(-2/3)
    v[ALP] = np.sqrt(H)
    return v


def test_gauge_wave_initial_data_matches_closed_form(O):
    n = 32
    g = O.OGrid((n, 3, 2), 1.0 / n)
    P = O.params_array(slicing=1, shift=0)
    s = O.init(g, P, O.id_array(0, A=0.01))
    ex = gauge_wave_exact(n, 1.0 / n, 0.0, 0.01)
    np.testing.assert_allclose(s[:, 1, 2, :], ex, rtol=0, atol=1e-15)


def test_thin_grid_reproduces_3d_gauge_wave_bitwise(O):
    n = 16
    P = O.params_array(slicing=0, shift=1)
    g3 = O.OGrid((n, n, n), 1.0 / n)
    g1 = O.OGrid((n, 1, 1), 1.0 / n)
    s3 = O.init(g3, P, O.id_array(0, A=0.01))
    s1 = O.init(g1, P, O.id_array(0, A=0.01))
    O.rk4_step(g3, P, s3, 0.0, 0.25 / n)
    O.rk4_step(g1, P, s1, 0.0, 0.25 / n)
    assert np.array_equal(s3[:, 5, 9, :], s1[:, 0, 0, :])


def test_gauge_wave_closed_form_4th_order(O):
    A, T = 0.01, 0.25
    errs = []
    for n in (16, 32, 64):
        g = O.OGrid((n, 1, 1), 1.0 / n)
        P = O.params_array(slicing=1, shift=0, ko_sigma=0.1)
        s = O.init(g, P, O.id_array(0, A=A))
        dt = 0.25 / n
        steps = int(round(T / dt))
        O.evolve(g, P, s, 0.0, dt, steps)
        ex = gauge_wave_exact(n, 1.0 / n, steps * dt, A)
        errs.append(np.abs(s[:, 0, 0, :] - ex).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13 < r1 < 19 and 14 < r2 < 18, (errs, r1, r2)
    assert errs[2] < 1e-6


def test_gauge_wave_constraints_converge_any_gauge(O):
    """Pure gauge: H and M vanish in the continuum for any slicing/shift;
    with 1+log + Gamma-driver they converge to zero at 4th order."""
    A, T = 0.01, 0.25
    norms = []
    for n in (16, 32, 64):
        g = O.OGrid((n, 1, 1), 1.0 / n)
        P = O.params_array(slicing=0, shift=1, eta=2.0, ko_sigma=0.1)
        s = O.init(g, P, O.id_array(0, A=A))
        dt = 0.25 / n
        O.evolve(g, P, s, 0.0, dt, int(round(T / dt)))
        _, nm = O.constraints(g, P, s)
        norms.append(nm)
    norms = np.array(norms)
    for m in (0, 1, 4, 5):  # H and M^x (L2, Linf); M^y, M^z vanish by symmetry
        r1, r2 = norms[0, m] / norms[1, m], norms[1, m] / norms[2, m]
        assert 12 < r1 < 20 and 13 < r2 < 19, (m, norms[:, m])
    assert np.all(norms[:, [2, 3, 6, 7]] == 0.0)


# ---------------------------------------------------------------------------
# P6: homogeneous radiation-dominated FLRW background.  On a 1x1x1 grid every
# stencil sees the same value, so the oracle integrates the Friedmann system:
#   a = (1 + 2 H0 t)^(1/2),  H_b = H0 / (1 + 2 H0 t),  rho = 3 H_b^2 / (8 pi)
# (w = 1/3).  RK4 error must be 4th order in dt.
# ---------------------------------------------------------------------------
def test_flrw_homogeneous_expansion_law(O):
    H0, w, T = 1.0, 1.0 / 3.0, 2.0
    errs = []
    for nsteps in (100, 200):
        g = O.OGrid((1, 1, 1), 1.0)
        P = O.params_array(slicing=0, shift=1, fluid=1, w=w, H0=H0, ko_sigma=0.1)
        s = O.init(g, P, O.id_array(1, mu=0.0))
        Hb0 = H0
        np.testing.assert_allclose(s[24, 0, 0, 0], 3 * Hb0 ** 2 / (8 * np.pi), rtol=1e-15)
        dt = T / nsteps
        O.evolve(g, P, s, 0.0, dt, nsteps)
        a_ex = np.sqrt(1 + 2 * H0 * T)
        Hb = H0 / (1 + 2 * H0 * T)
        chi = s[CHI, 0, 0, 0]
        a_num = chi ** -0.5
        E_num = s[24, 0, 0, 0] * chi ** 1.5
        e = max(abs(a_num / a_ex - 1), abs(s[TRK, 0, 0, 0] / (-3 * Hb) - 1), abs(E_num / (3 * Hb ** 2 / (8 * np.pi)) - 1),
                abs(s[ALP, 0, 0, 0] - 1))
        errs.append(e)
        assert np.all(s[GT:GT + 6, 0, 0, 0] == np.array([1, 0, 0, 1, 0, 1.0]))
    assert errs[1] < 1e-8
    assert 12 < errs[0] / errs[1] < 20, errs


def test_flrw_homogeneous_all_points_identical(O):
    n = (6, 5, 4)
    g = O.OGrid(n, 0.1, x0=(-0.3, -0.25, -0.2))
    P = O.params_array(fluid=1, H0=3.0)
    s = O.init(g, P, O.id_array(1, mu=0.0))
    O.rk4_step(g, P, s, 0.0, 0.01)
    assert np.all(s == s[:, :1, :1, :1])


# ---------------------------------------------------------------------------
# P7: FLRW + zeta initial data satisfy the discrete constraints.
# ---------------------------------------------------------------------------
def test_flrw_zeta_initial_data_satisfies_constraints(O):
    n = 24
    h = 1.0 / n
    g = O.OGrid((n, n, n), h, x0=(-(n // 2) * h,) * 3)
    H0 = 40.0
    P = O.params_array(slicing=0, shift=1, fluid=1, w=1 / 3, H0=H0)
    s = O.init(g, P, O.id_array(1, mu=0.5, sigma=0.125, q=(1.0, 0.9, 1.1)))
    hm, nm = O.constraints(g, P, s)
    scale = 2.0 / 3.0 * (3 * H0) ** 2
    assert np.abs(hm[0]).max() < 1e-13 * scale
    assert np.all(hm[1:] == 0.0)
    # the perturbation is real: chi varies and E is not uniform
    assert s[CHI].max() - s[CHI].min() > 0.5
    assert s[24].std() > 0


def test_flop_count_is_deterministic_and_positive(O):
    n = 16
    g = O.OGrid((n, n, n), 1.0 / n)
    P = O.params_array()
    s = inputs.smooth_state(n, seed=3)
    c1 = O.flop_count(g, P, s)
    c2 = O.flop_count(g, P, inputs.smooth_state(n, seed=4))
    assert c1 == c2
    assert c1["add"] > 1000 and c1["mul"] > 1000


# ---------------------------------------------------------------------------
# Kurganov-Tadmor at a density step (flat slice).  Across a single jump the
# minmod slopes vanish, so the face states are the two cell states and the
# flux difference at the cell left of the jump is, by hand,
#   RHS = -[ (F_R - F_L)/2 - a (U_R - U_L)/2 ] / h
# with a the largest characteristic speed:  a = alpha sqrt(w gamma^xx) + |beta^x|
# for a fluid at rest, a = (v + c)/(1 + v c) for a uniform boost v > 0
# (relativistic velocity addition, c^2 = w).
# ---------------------------------------------------------------------------
def _fluid_line(O, n, P, chi, alpha, betax, rho, vx):
    s = flat_state(O, (n, 1, 1), P, chi=chi, alpha=alpha, beta=(betax, 0.0, 0.0))
    w = P[4]
    gxx = chi  # gamma^xx = chi gt^xx, gt = identity
    v2 = gxx * vx * vx
    W2 = 1.0 / (1.0 - v2)
    E = (rho + w * rho) * W2 - w * rho
    J = (rho + w * rho) * W2 * vx
    sqrtg = chi ** -1.5
    s[24, 0, 0, :] = sqrtg * E
    s[25, 0, 0, :] = sqrtg * J
    return s, E, J


@pytest.mark.parametrize("betax", [0.3, -0.2, 0.0])
def test_kt_step_fluid_at_rest_with_shift(O, betax):
    n, m, w = 16, 8, 1.0 / 3.0
    h = 1.0 / n
    g = O.OGrid((n, 1, 1), h)
    P = O.params_array(slicing=1, shift=0, ko_sigma=0.0, w=w, fluid=1)
    chi, alpha = 0.8, 1.2
    rho = np.where(np.arange(n) < m, 1.0, 1.5)
    s, E, J = _fluid_line(O, n, P, chi, alpha, betax, rho, 0.0)
    r = O.rhs(g, P, s)
    sqrtg = chi ** -1.5
    a = alpha * np.sqrt(w * chi) + abs(betax)
    EL, ER = E[m - 1], E[m]
    F = lambda Ev: sqrtg * (-betax * Ev)
    expect = -(0.5 * (F(ER) - F(EL)) - 0.5 * a * sqrtg * (ER - EL)) / h
    assert abs(r[24, 0, 0, m - 1] - expect) <= 1e-12 * abs(expect)
    # momentum: flux sqrtg * alpha * P, no jump in U_x
    expect_S = -(0.5 * sqrtg * alpha * w * (rho[m] - rho[m - 1])) / h
    assert abs(r[25, 0, 0, m - 1] - expect_S) <= 1e-12 * abs(expect_S)
    # cell right of the jump: its own slope is limited to zero (minmod of a
    # jump and a flat difference), so its right face carries F(E_R) exactly
    H_jump = 0.5 * (F(ER) + F(EL)) - 0.5 * a * sqrtg * (ER - EL)
    expect_m = -(F(ER) - H_jump) / h
    assert abs(r[24, 0, 0, m] - expect_m) <= 1e-12 * abs(expect_m)


@pytest.mark.parametrize("v", [0.4, 0.7])
def test_kt_step_boosted_fluid_speed_is_velocity_addition(O, v):
    n, m, w = 16, 8, 1.0 / 3.0
    h = 1.0 / n
    g = O.OGrid((n, 1, 1), h)
    P = O.params_array(slicing=1, shift=0, ko_sigma=0.0, w=w, fluid=1)
    rho = np.where(np.arange(n) < m, 1.0, 2.0)
    s, E, J = _fluid_line(O, n, P, 1.0, 1.0, 0.0, rho, v)
    r = O.rhs(g, P, s)
    c = np.sqrt(w)
    a = (v + c) / (1 + v * c)
    W2 = 1.0 / (1 - v * v)
    FE = J
    FJ = (rho + w * rho) * W2 * v * v + w * rho
    for f, (Fv, Uv) in enumerate([(FE, E), (FJ, J)]):
        expect = -(0.5 * (Fv[m] - Fv[m - 1]) - 0.5 * a * (Uv[m] - Uv[m - 1])) / h
        assert abs(r[24 + f, 0, 0, m - 1] - expect) <= 1e-12 * abs(expect), (f, r[24 + f, 0, 0, m - 1], expect)


# ---------------------------------------------------------------------------
# Scalar field pins (section "Physical system settings": box phi = 0).
# ---------------------------------------------------------------------------
def test_scalar_plane_wave_on_flat_space_4th_order(O):
    """phi = eps sin(k (x - t)) solves box phi = 0 on flat space; with Pi =
    -n.d phi = eps k cos(k (x - t)) and eps = 1e-6 the metric response is
    O(eps^2).  The oracle's phi after one crossing time converges to it at 4th
    order (centred stencils, RK4 with dt = h/4)."""
    eps = 1e-6
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        g = O.OGrid((n, 1, 1), h)
        P = O.params_array(slicing=1, shift=0, scalar=1, ko_sigma=0.0)
        s = np.zeros((26, 1, 1, n))
        x = h * np.arange(n)
        k = 2 * np.pi
        s[CHI] = 1.0
        s[GT] = s[GT + 3] = s[GT + 5] = 1.0
        s[ALP] = 1.0
        s[24] = eps * np.sin(k * x)
        s[25] = eps * k * np.cos(k * x)
        T = 0.5
        steps = int(round(T / (0.25 * h)))
        O.evolve(g, P, s, 0.0, T / steps, steps)
        errs.append(np.abs(s[24, 0, 0] - eps * np.sin(k * (x - T))).max() / eps)
    assert errs[2] < 1e-5, errs
    assert 13 < errs[0] / errs[1] < 19 and 14 < errs[1] / errs[2] < 18, errs


def test_homogeneous_scalar_momentum_redshifts_as_a_minus_3(O):
    """A homogeneous Pi in radiation FLRW obeys d_t Pi = alpha K Pi = -3 H Pi,
    so Pi a^3 stays constant (a = chi^{-1/2}), and d_t phi = -alpha Pi
    integrates to phi(T) = -Pi0 (1 - (1 + 2 H0 T)^{-1/2}) / H0; RK4 error O(dt^4)."""
    H0, T = 1.0, 2.0
    errs = []
    for nsteps in (100, 200):
        g = O.OGrid((1, 1, 1), 1.0)
        P = O.params_array(slicing=0, shift=1, fluid=1, scalar=1, w=1.0 / 3.0, H0=H0)
        s = O.init(g, P, O.id_array(1, mu=0.0))
        s[29] = 1e-7  # Pi (its energy 1/2 Pi^2 would otherwise move K, and the lapse, off K_ref)
        O.evolve(g, P, s, 0.0, T / nsteps, nsteps)
        a = s[CHI, 0, 0, 0] ** -0.5
        phi_exact = -1e-7 * (1.0 - (1.0 + 2.0 * H0 * T) ** -0.5) / H0
        errs.append(max(abs(s[29, 0, 0, 0] * a ** 3 / 1e-7 - 1.0), abs(s[28, 0, 0, 0] / phi_exact - 1.0)))
    assert errs[1] < 1e-7, errs
    assert 12 < errs[0] / errs[1] < 20, errs


# ---------------------------------------------------------------------------
# P8: primitive recovery round trip.
# ---------------------------------------------------------------------------
def test_fluid_primitive_recovery_round_trip(O):
    """For P = w rho: E = (rho + P) W^2 - P, J = (rho + P) W^2 v with W^2 = 1/(1 - v^2);
    the oracle's recovery from (E, J^2) returns rho to rounding (times the
    problem's condition number), for slow and fast flows and several equations
    of state."""
    rng = np.random.default_rng(8)
    for w in (1.0 / 3.0, 0.1, 1.0):
        rho = 10.0 ** rng.uniform(-3, 3, 2000)
        v = np.concatenate([rng.uniform(0, 0.1, 1000), rng.uniform(0.1, 0.99, 1000)])
        W2 = 1.0 / (1.0 - v * v)
        P = w * rho
        E = (rho + P) * W2 - P
        J = (rho + P) * W2 * v
        got = O.fluid_rho(E, J * J, w)
        # E^2 - J^2 = (rho + P)^2 W^2 - ... cancels as v -> 1: the recovery's condition
        # number grows like W^4, so the bound does too (a wrong formula is off by O(1))
        assert np.all(np.abs(got - rho) <= 4e-15 * W2 * W2 * rho), (w, np.max(np.abs(got / rho - 1)))


# ---------------------------------------------------------------------------
# Conservation: on a flat, static background (chi = 1, gt = delta, K = 0,
# alpha = 1, beta = 0) the fluid's geometric sources vanish, so the fluid
# right-hand side is minus the divergence of the Kurganov-Tadmor face fluxes
# plus the Kreiss-Oliger term; on a periodic grid both telescope, and the grid
# sums of the tau~ and S~_i right-hand sides vanish for any fluid state.  A flux
# that is not the same on both sides of a face (a non-conservative form, an
# upwinding on one side only, a wrong face index) breaks the sum.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ko", [0.0, 0.2])
def test_kt_fluid_totals_are_conserved_on_a_flat_background(O, ko):
    n = (12, 10, 9)
    P = O.params_array(slicing=0, shift=1, ko_sigma=ko, w=1.0 / 3.0, fluid=1)
    s = flat_state(O, n, P)
    rng = np.random.default_rng(77)
    E = 1.0 + 0.5 * rng.random((n[2], n[1], n[0]))
    J = 0.4 * (rng.random((3, n[2], n[1], n[0])) - 0.5) * E  # |J| <= 0.35 E: a physical state
    s[24] = E
    s[25:28] = J
    r = O.rhs(O.OGrid(n, 1.0 / n[0]), P, s)
    for f in range(24, 28):
        total, scale = r[f].sum(), np.abs(r[f]).sum()
        assert scale > 1.0
        assert abs(total) <= 1e-13 * scale, (f, total, scale)


def test_kt_conservation_pin_catches_a_one_sided_flux(O):
    """The same sum with a planted non-conservative term (the first face of
    every cell weighted 1 + 1e-6) is far from zero: the pin can fail."""
    n = 12
    rng = np.random.default_rng(78)
    E = 1.0 + 0.5 * rng.random(n)
    H = E + 0.1 * np.roll(E, -1)  # any face flux H_{i+1/2}
    good = -(H - np.roll(H, 1))
    bad = -(H - (1 + 1e-6) * np.roll(H, 1))
    assert abs(good.sum()) <= 1e-13 * np.abs(good).sum()
    assert abs(bad.sum()) > 1e-8 * np.abs(bad).sum()

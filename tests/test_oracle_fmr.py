"""Pins of the oracle's fixed mesh refinement (section "Statement of need":
nested refinement levels around the collapsing region; the scheme's readings
are listed in the oracle's FMR section).

What pins it, independently of its own formulas:
* space: the ghost values of a child equal a tensor-product polynomial of
  degree <= 5 per axis sampled on the parent, to rounding, for a child of the
  periodic box and for a child of a refined box; a degree-6 term is not
  reproduced (the interpolation is exactly 6-point Lagrange); interior points
  are left alone;
* injection copies exactly the child's interior points that lie on parent
  points and nothing else;
* time: the continuous extension of RK4 reproduces the exact solution of a
  quadrature problem y' = f(t) with f of degree <= 2, and for y' = lambda y it
  equals 1 + z theta + (z theta)^2/2 + (z theta)^3/6 + O(z^4) with the z^4
  remainder a pure z^4 term (the order-3 conditions, including the one through
  a_ij); at theta = 0 and 1 it gives U_n and the RK4 step;
* the whole scheme: the gauge wave (harmonic slicing, zero shift: its closed
  form is exact) on three levels converges at 4th order on every level (error
  ratio > 12 per doubling), and the error at the finest resolution is below
  that of the uniform grid; ghost values taken at the stage times instead of
  the stage-consistent ones break this (the convergence stalls), which the
  last test plants in a copy of the scheme written here with the oracle's
  operators; the same copy with stage-consistent values, its Taylor data
  taken by difference formulas, agrees with the oracle's scheme.
"""
import numpy as np
import pytest

from paper_2606_02053_gb300.inputs import nested_boxes


def coords(level):
    n, h, x0 = level["n"], level["h"], level["x0"]
    x = x0[0] + h[0] * np.arange(n[0])
    y = x0[1] + h[1] * np.arange(n[1])
    z = x0[2] + h[2] * np.arange(n[2])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def poly(X, Y, Z, coef):
    """sum_{a,b,c} coef[a,b,c] X^a Y^b Z^c."""
    out = np.zeros_like(X)
    for a in range(coef.shape[0]):
        for b in range(coef.shape[1]):
            for c in range(coef.shape[2]):
                if coef[a, b, c] != 0.0:
                    out += coef[a, b, c] * X ** a * Y ** b * Z ** c
    return out


@pytest.fixture(scope="module")
def levels3():
    return nested_boxes(24, 1.0 / 24, (-0.5, -0.5, -0.5), 3, [20, 20])


def test_prolongation_reproduces_degree_five_polynomials(O, levels3):
    rng = np.random.default_rng(5)
    coef = rng.uniform(-1, 1, size=(6, 6, 6)) * (rng.uniform(size=(6, 6, 6)) < 0.3)
    coef[5, 5, 5] = 1.0
    coef[5, 0, 0] = coef[0, 5, 0] = coef[0, 0, 5] = 2.0
    for l in (1, 2):
        par = poly(*coords(levels3[l - 1]), coef)[None].repeat(2, axis=0).copy()
        par[1] *= -3.0
        exact = poly(*coords(levels3[l]), coef)[None].repeat(2, axis=0)
        exact[1] *= -3.0
        child = np.full_like(exact, 7.0)
        O.fmr_prolong(levels3, l, par, child)
        inner = O.fmr_interior(levels3[l])
        assert np.all(child[:, inner] == 7.0)
        err = np.abs(child - exact)[:, ~inner].max() / np.abs(exact).max()
        assert err < 1e-13, (l, err)


def test_prolongation_is_not_exact_for_degree_six(O, levels3):
    coef = np.zeros((7, 1, 1))
    coef[6, 0, 0] = 1.0
    par = poly(*coords(levels3[0]), coef)[None].copy()
    exact = poly(*coords(levels3[1]), coef)[None]
    child = exact.copy()
    O.fmr_prolong(levels3, 1, par, child)
    err = np.abs(child - exact).max() / np.abs(exact).max()
    assert err > 1e-6, err


def test_restriction_injects_coincident_interior_points(O, levels3):
    rng = np.random.default_rng(3)
    for l in (1, 2):
        child = rng.standard_normal((3,) + tuple(levels3[l]["n"][::-1]))
        par0 = rng.standard_normal((3,) + tuple(levels3[l - 1]["n"][::-1]))
        par = par0.copy()
        O.fmr_restrict(levels3, l, child, par)
        lv = levels3[l]
        expect = par0.copy()
        for k in range(lv["lo"][2], lv["hi"][2]):
            for j in range(lv["lo"][1], lv["hi"][1]):
                for i in range(lv["lo"][0], lv["hi"][0]):
                    X2 = (lv["origin"][0] + i, lv["origin"][1] + j, lv["origin"][2] + k)
                    if all(v % 2 == 0 for v in X2):
                        expect[:, X2[2] // 2, X2[1] // 2, X2[0] // 2] = child[:, k, j, i]
        assert np.array_equal(par, expect)
        assert not np.array_equal(par, par0)


def rk4_stages_quadrature(f, t, dt):
    return [f(t), f(t + 0.5 * dt), f(t + 0.5 * dt), f(t + dt)]


def test_dense_output_exact_for_quadrature_of_degree_two(O):
    a, b, c = 0.7, -1.3, 2.1
    f = lambda t: a + b * t + c * t * t
    F = lambda t: a * t + b * t * t / 2 + c * t ** 3 / 3
    t, dt, y0 = 0.4, 0.3, 1.25
    k = [np.array([v]) for v in rk4_stages_quadrature(f, t, dt)]
    for theta in (0.0, 0.25, 0.5, 0.75, 1.0, 0.1234):
        y = O.rk4_dense(np.array([y0]), k, dt, theta)[0]
        assert abs(y - (y0 + F(t + theta * dt) - F(t))) < 1e-14, theta
    # a cubic f (quartic solution) is not reproduced: order 3 exactly
    f3 = lambda t: t ** 3
    k = [np.array([v]) for v in rk4_stages_quadrature(f3, t, dt)]
    y = O.rk4_dense(np.array([y0]), k, dt, 0.5)[0]
    exact = y0 + ((t + 0.5 * dt) ** 4 - t ** 4) / 4
    assert abs(y - exact) > 1e-6


def test_dense_output_order_three_on_linear_ode(O):
    y0 = 1.0
    for theta in (0.25, 0.5, 0.75):
        rem = []
        for z in (0.05, 0.1, 0.2):
            lam, dt = z, 1.0
            k1 = lam * y0
            k2 = lam * (y0 + 0.5 * dt * k1)
            k3 = lam * (y0 + 0.5 * dt * k2)
            k4 = lam * (y0 + dt * k3)
            y = O.rk4_dense(np.array([y0]), [np.array([v]) for v in (k1, k2, k3, k4)], dt, theta)[0]
            zt = z * theta
            rem.append((y - (1 + zt + zt ** 2 / 2 + zt ** 3 / 6)) / z ** 4)
        # rounding of y ~ 1e-16 divided by z^4 >= 6e-6: remainders equal to ~1e-10
        assert max(rem) - min(rem) < 1e-6 * max(abs(r) for r in rem) + 1e-9, (theta, rem)
    # end points: U_n and the RK4 step
    z = 0.3
    k1 = z
    k2 = z * (1 + 0.5 * k1)
    k3 = z * (1 + 0.5 * k2)
    k4 = z * (1 + k3)
    ks = [np.array([v]) for v in (k1, k2, k3, k4)]
    assert O.rk4_dense(np.array([1.0]), ks, 1.0, 0.0)[0] == 1.0
    step = 1 + (k1 + 2 * k2 + 2 * k3 + k4) / 6
    assert abs(O.rk4_dense(np.array([1.0]), ks, 1.0, 1.0)[0] - step) < 1e-15


A_GW = 0.01


def gauge_wave_exact(level, t):
    x = level["x0"][0] + level["h"][0] * np.arange(level["n"][0])
    H = 1.0 - A_GW * np.sin(2.0 * np.pi * (x - t))
    return {17: np.sqrt(H), 0: H ** (-1.0 / 3.0), 1: H ** (2.0 / 3.0)}  # alpha, chi, gt_xx


def gauge_wave_errors(O, n0, nlev, T=0.25):
    P = O.params_array(slicing=1, shift=0, ko_sigma=0.1)
    nc = n0 + 8
    lv = nested_boxes((n0, 1, 1), 1.0 / n0, (0.0, 0.0, 0.0), nlev, [(nc, 2, 2), (nc, 4, 4)][: nlev - 1])
    st = O.fmr_init(lv, P, O.id_array(0, A=A_GW))
    dt = 0.25 / n0
    steps = int(round(T / dt))
    for s in range(steps):
        O.fmr_step(lv, P, st, s * dt, dt)
    errs = []
    for l, L in enumerate(lv):
        ex = gauge_wave_exact(L, steps * dt)
        errs.append(max(np.abs(st[l][f] - v[None, None, :]).max() for f, v in ex.items()))
    return errs


def test_gauge_wave_on_three_levels_converges_at_fourth_order(O):
    e = [gauge_wave_errors(O, n, 3) for n in (16, 32, 64)]
    print("\nFMR gauge wave errors per level:", e)
    for l in range(3):
        r1, r2 = e[0][l] / e[1][l], e[1][l] / e[2][l]
        assert r1 > 12.0 and r2 > 12.0, (l, r1, r2)
    uni = gauge_wave_errors(O, 64, 1)[0]
    assert e[2][0] < uni, (e[2][0], uni)


def test_stage_time_ghost_values_lose_an_order(O):
    """Planted mistake: a two-level scheme written here with the oracle's own
    operators, whose child stages take the parent's continuous extension at
    the stage times (not the stage-consistent values), stalls where the
    oracle's scheme keeps converging."""
    P = O.params_array(slicing=1, shift=0, ko_sigma=0.1)

    def run(n0, consistent):
        nc = n0 + 8
        lv = nested_boxes((n0, 1, 1), 1.0 / n0, (0.0, 0.0, 0.0), 2, [(nc, 2, 2)])
        U = O.fmr_init(lv, P, O.id_array(0, A=A_GW))
        g0, g1 = O.level_grid(lv[0]), O.level_grid(lv[1])
        inner = O.fmr_interior(lv[1])
        dt = 0.25 / n0
        steps = int(round(0.25 / dt))

        def rhs1(Y, t):
            r = O.rhs(g1, P, Y, t)
            r[:, ~inner] = 0.0
            return r

        for s in range(steps):
            t = s * dt
            Un = U[0].copy()
            k = []
            Y = Un
            for c, w in ((0.0, 0.5), (0.5, 0.5), (0.5, 1.0), (1.0, None)):
                k.append(O.rhs(g0, P, Y, t + c * dt))
                if w is not None:
                    Y = Un + w * dt * k[-1]
            U[0] = Un + dt / 6 * (k[0] + 2 * k[1] + 2 * k[2] + k[3])
            for m in (0, 1):
                tc, h = t + m * 0.5 * dt, 0.5 * dt
                th0 = 0.5 * m

                def ghosts(Yc, stage):
                    if consistent:
                        # theta-derivatives of the (cubic) extension by difference
                        # formulas exact for cubics, times powers of the step ratio 1/2
                        e = 0.25
                        d = [O.rk4_dense(Un, k, dt, th0 + j * e) for j in (-2, -1, 0, 1, 2)]
                        u = d[2]
                        u1 = (8 * (d[3] - d[1]) - (d[4] - d[0])) / (12 * e) * 0.5
                        u2 = (d[3] - 2 * d[2] + d[1]) / e ** 2 * 0.25
                        u3 = (d[4] - 2 * d[3] + 2 * d[1] - d[0]) / (2 * e ** 3) * 0.125
                        e1, e2, e3 = [(0, 0, 0), (0.5, 0, 0), (0.5, 0.25, 0), (1.0, 0.5, 0.25)][stage - 1]
                        par = u + e1 * u1 + e2 * u2 + e3 * u3
                    else:
                        par = O.rk4_dense(Un, k, dt, th0 + 0.5 * [0.0, 0.5, 0.5, 1.0][stage - 1])
                    O.fmr_prolong(lv, 1, np.ascontiguousarray(par), Yc)

                ghosts(U[1], 1)
                V = U[1].copy()
                kc = []
                Y = V
                for st, (c, w) in enumerate(((0.0, 0.5), (0.5, 0.5), (0.5, 1.0), (1.0, None))):
                    kc.append(rhs1(Y, tc + c * h))
                    if w is not None:
                        Y = V + w * h * kc[-1]
                        ghosts(Y, st + 2)
                U[1] = V + h / 6 * (kc[0] + 2 * kc[1] + 2 * kc[2] + kc[3])
            O.fmr_restrict(lv, 1, U[1], U[0])
        ex = gauge_wave_exact(lv[0], steps * dt)
        err = max(np.abs(U[0][f] - v[None, None, :]).max() for f, v in ex.items())
        return err, U, lv

    plain = [run(n, False)[0] for n in (32, 64)]
    assert plain[0] / plain[1] < 8.0, plain
    ref = [run(n, True) for n in (32, 64)]
    assert ref[0][0] / ref[1][0] > 12.0, [r[0] for r in ref]
    # the stage-consistent copy written here and the oracle's scheme agree
    _, U, lv = ref[0]
    st = O.fmr_init(lv, P, O.id_array(0, A=A_GW))
    dt = 0.25 / 32
    for s in range(int(round(0.25 / dt))):
        O.fmr_step(lv, P, st, s * dt, dt)
    for l in range(2):
        inner = O.fmr_interior(lv[l])
        assert np.abs(st[l][:, inner] - U[l][:, inner]).max() < 1e-12

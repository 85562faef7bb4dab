"""Pins of the oracle's collapse diagnostics, its per-point zeta map and their
reverse modes (the quantities a primordial-black-hole threshold search
differentiates; the paper's examples follow the central lapse and the
compaction of the overdensity, section "Examples").

* the zeta map is the leading-order initial data of the paper's initial-data
  paragraph: given the Gaussian's values it reproduces the Gaussian data, and
  the Hamiltonian and momentum constraints vanish on it;
* compaction C(r_k) = 2 dM / R: zero for a homogeneous state, and for a top-hat
  overdensity on a uniform conformal factor the closed form
  2 h^2 dE [n(min(b, k)) - n(b) n(k) / N] / (k chi), with the lattice-point
  counts n(.) taken by brute force; the areal radius R sees exactly the six
  axis points at distance r_k;
* the tapes against central differences (dot-product tests), and the whole
  pipeline zeta -> RK4 steps -> (min central lapse, peak compaction) against
  differences along the amplitude mu;
* from a fluid exactly at rest (the configurations' data) the discrete map is
  not differentiable along single-point perturbations of zeta: the forward and
  backward differences disagree (a kink of the minmod limiter on a symmetry
  plane), so no gradient exists there; along mu both agree with the tape.
"""
import itertools

import numpy as np
import pytest


def flrw(O, n, H0=20.0):
    h = 1.0 / n
    x0 = (-(n // 2) * h,) * 3
    g = O.OGrid((n, n, n), h, x0=x0)
    P = O.params_array(slicing=0, shift=1, eta=2.0, ko_sigma=0.1, fluid=1, w=1.0 / 3.0, H0=H0)
    return g, P, h, x0


def gaussian(n, h, x0, mu, sigma, centre=(0.0, 0.0, 0.0), q=(1.0, 1.0, 1.0)):
    x = x0[0] + h * np.arange(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r2 = ((X - centre[0]) / q[0]) ** 2 + ((Y - centre[1]) / q[1]) ** 2 + ((Z - centre[2]) / q[2]) ** 2
    return mu * np.exp(-r2 / (2 * sigma ** 2))


def test_zeta_map_is_the_leading_order_data_and_satisfies_the_constraints(O):
    n = 12
    g, P, h, x0 = flrw(O, n, H0=40.0)
    zeta = gaussian(n, h, x0, 0.5, 0.15, q=(1.0, 0.9, 1.1))
    s = O.init_zeta(g, P, zeta)
    ref = O.init(g, P, O.id_array(1, mu=0.5, sigma=0.15, q=(1.0, 0.9, 1.1)))
    scale = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    assert (np.abs(s - ref).reshape(s.shape[0], -1).max(axis=1) <= 1e-15 * scale).all()
    _, norms = O.constraints(g, P, s)
    assert norms[4] <= 1e-12 * 6.0 * 40.0 ** 2 and norms[5:].max() == 0.0
    assert O.central_lapse(g, s) == 1.0


def uniform_state(O, g, P, chi, E):
    s = np.zeros((O.nfields(P), g.n[2], g.n[1], g.n[0]))
    s[0] = chi
    s[1] = s[4] = s[6] = 1.0
    s[17] = 1.0
    s[24] = E * chi ** -1.5
    return s


def lattice_count(r2):
    """Points (di, dj, dk) of the integer lattice with di^2 + dj^2 + dk^2 < r2."""
    m = int(np.ceil(np.sqrt(r2))) + 1
    return sum(1 for p in itertools.product(range(-m, m + 1), repeat=3) if p[0] ** 2 + p[1] ** 2 + p[2] ** 2 < r2)


def test_compaction_of_a_homogeneous_state_is_zero(O):
    n = 14
    g, P, h, _ = flrw(O, n)
    E, chi = 3.0 * 20.0 ** 2 / (8 * np.pi), 0.7
    kmax = n // 2 - 1
    C = O.compaction(g, P, uniform_state(O, g, P, chi, E), kmax)
    # scale: 2 M / R of the whole mass inside r_k; dM cancels it to the rounding of the box means
    for k in range(1, kmax + 1):
        total = 2.0 * h * h * lattice_count(k * k) * E / (k * chi)
        assert abs(C[k - 1]) <= 1e-13 * total, (k, C[k - 1], total)


@pytest.mark.parametrize("chi", [1.0, 0.6])
def test_compaction_of_a_top_hat_overdensity(O, chi):
    n = 16
    g, P, h, _ = flrw(O, n)
    E0, dE, b = 2.0, 0.3, 3  # E = E0 + dE on the points with di^2 + dj^2 + dk^2 < b^2
    s = uniform_state(O, g, P, chi, E0)
    c = n // 2
    idx = np.arange(n) - c
    m = idx[:, None, None] ** 2 + idx[None, :, None] ** 2 + idx[None, None, :] ** 2
    s[24][m < b * b] = (E0 + dE) * chi ** -1.5
    kmax = n // 2 - 1
    C = O.compaction(g, P, s, kmax)
    N = n ** 3
    nb = lattice_count(b * b)
    for k in range(1, kmax + 1):
        nk = lattice_count(k * k)
        expect = 2.0 * h * h * dE * (lattice_count(min(b, k) ** 2) - nb * nk / N) / (k * chi)
        total = 2.0 * h * h * nk * (E0 + dE) / (k * chi)  # dM is a difference of sums of this size
        assert abs(C[k - 1] - expect) <= 1e-13 * total, (k, C[k - 1], expect)


def test_areal_radius_uses_the_six_axis_points(O):
    """Changing chi (at fixed E) on the six axis points at distance k changes R(r_k) to
    k h times their mean chi^{-1/2}; the same change on six other points at the same
    distance (off the axes) leaves R(r_k) alone.  Both change the box mean Ebar
    the same way, and neither set lies inside r_k."""
    n, k, b = 16, 5, 2
    g, P, h, _ = flrw(O, n)
    E0, dE, c0, c1 = 2.0, 0.3, 0.8, 0.5
    base = uniform_state(O, g, P, c0, E0)
    c = n // 2
    idx = np.arange(n) - c
    m = idx[:, None, None] ** 2 + idx[None, :, None] ** 2 + idx[None, None, :] ** 2
    base[24][m < b * b] = (E0 + dE) * c0 ** -1.5
    axis = [(c, c, c + k), (c, c, c - k), (c, c + k, c), (c, c - k, c), (c + k, c, c), (c - k, c, c)]
    off = [(c + 3, c + 4, c), (c - 3, c + 4, c), (c, c + 3, c - 4), (c, c - 3, c - 4), (c + 4, c, c + 3),
           (c - 4, c, c + 3)]  # 3^2 + 4^2 = 5^2
    Cs = []
    for pts in (axis, off):
        s = base.copy()
        for p in pts:
            s[0][p] = c1
            s[24][p] = E0 * c1 ** -1.5
        Cs.append(O.compaction(g, P, s, k)[k - 1])
    # dM is the same in both (same weights, same E, none inside r_k): the ratio is R_off / R_axis
    assert abs(Cs[0] / Cs[1] - c0 ** -0.5 / c1 ** -0.5) <= 1e-13


def dot_check(f, vjp_dir, x, v, eps=(1e-6, 5e-7)):
    best = None
    for e in eps:
        lhs = (f(x + e * v) - f(x - e * v)) / (2 * e)
        best = lhs if best is None or abs(lhs - vjp_dir) < abs(best - vjp_dir) else best
    return best


def test_compaction_tape_dot_product(O):
    from paper_2606_02053_gb300 import inputs

    n = 10
    g, P, h, _ = flrw(O, n)
    U = inputs.smooth_state(n, seed=81, fluid=1, scale=0.5)
    kmax, kstar = 4, 3
    lam = O.compaction_vjp(g, P, U, kmax, kstar, 1.0)
    v = np.random.default_rng(5).standard_normal(U.shape)
    lhs = dot_check(lambda X: O.compaction(g, P, np.ascontiguousarray(X), kmax)[kstar - 1], float(np.sum(lam * v)),
                    U, v)
    assert abs(lhs - np.sum(lam * v)) <= 1e-8 * abs(np.sum(lam * v))


def test_zeta_map_tape_dot_product(O):
    n = 9
    g, P, h, x0 = flrw(O, n)
    zeta = gaussian(n, h, x0, 0.4, 0.2, centre=(0.03, -0.02, 0.01)) + 0.02 * np.random.default_rng(3).standard_normal(
        (n, n, n))
    rng = np.random.default_rng(4)
    lam = rng.standard_normal((O.nfields(P), n, n, n))
    v = rng.standard_normal((n, n, n))
    zbar = O.init_zeta_vjp(g, P, zeta, lam)
    lhs = dot_check(lambda Z: float(np.sum(lam * O.init_zeta(g, P, Z))), float(np.sum(zbar * v)), zeta, v)
    assert abs(lhs - np.sum(zbar * v)) <= 1e-8 * abs(np.sum(zbar * v))


def test_collapse_gradient_matches_differences_along_mu(O):
    n, steps = 8, 4
    g, P, h, x0 = flrw(O, n)
    shape = gaussian(n, h, x0, 1.0, 0.15)
    mu, dt, kmax = 0.6, 0.25 * h, n // 2 - 1
    ga, gc, r = O.collapse_gradient(g, P, mu * shape, dt, steps, kmax)
    dmu = 1e-6
    rp = O.collapse_run(g, P, (mu + dmu) * shape, dt, steps, kmax)
    rm = O.collapse_run(g, P, (mu - dmu) * shape, dt, steps, kmax)
    assert rp["nstar"] == rm["nstar"] == r["nstar"] and rp["kstar"] == rm["kstar"] == r["kstar"]
    fd_a = (rp["min_lapse"] - rm["min_lapse"]) / (2 * dmu)
    fd_c = (rp["peak"] - rm["peak"]) / (2 * dmu)
    assert abs(np.sum(ga * shape) - fd_a) <= 1e-6 * abs(fd_a), (np.sum(ga * shape), fd_a)
    assert abs(np.sum(gc * shape) - fd_c) <= 1e-6 * abs(fd_c), (np.sum(gc * shape), fd_c)


def test_single_point_zeta_perturbations_meet_a_kink_from_a_fluid_at_rest(O):
    """Mirror-symmetric data (h = 1/8 keeps every coordinate exact, so the symmetry is
    bitwise): the velocity vanishes exactly on the symmetry planes, and a perturbation of
    zeta at one point off those planes moves minmod's two equal slopes there apart.  The
    forward and backward differences of the peak compaction then differ by percents, and
    each is stable as the step shrinks tenfold: the map has a kink along those
    directions and no gradient exists.  The tape returns the derivative of the branches
    taken at the ties (its value lies between the two one-sided ones here); along mu the
    data stay symmetric and the tape agrees with the differences."""
    n, steps = 8, 3
    g, P, h, x0 = flrw(O, n)
    shape = gaussian(n, h, x0, 1.0, 0.15)
    mu, dt, kmax = 0.6, 0.25 * h, n // 2 - 1
    _, gc, r = O.collapse_gradient(g, P, mu * shape, dt, steps, kmax)
    base = r["peak"]

    def one_sided(p, eps):
        e = np.zeros_like(shape)
        e[p] = 1.0
        fwd = (O.collapse_run(g, P, mu * shape + eps * e, dt, steps, kmax)["peak"] - base) / eps
        bwd = (base - O.collapse_run(g, P, mu * shape - eps * e, dt, steps, kmax)["peak"]) / eps
        return fwd, bwd

    for p in [(5, 4, 3), (4, 5, 6), (3, 4, 4), (6, 5, 4)]:  # (k, j, i), off the symmetry planes
        f1, b1 = one_sided(p, 1e-5)
        f2, b2 = one_sided(p, 1e-6)
        scale = max(abs(f1), abs(b1))
        assert abs(f1 - f2) <= 1e-3 * scale and abs(b1 - b2) <= 1e-3 * scale  # each side converged
        assert abs(f1 - b1) >= 5e-3 * scale, (p, f1, b1)  # but the two sides disagree: a kink
        assert min(f1, b1) <= gc[p] <= max(f1, b1)

"""Pins of the oracle's isocurvature initial data (id kind 2).

Reading of the paper (section "Examples", spherically symmetric iso-curvature;
section "Physical system settings", initial data): a massless scalar carries
the isocurvature mode Upsilon(x) and is not part of the background metric; at
leading gradient order phi = Upsilon, Pi = 0, the metric is the FLRW + zeta
data of kind 1, and the fluid energy E takes what the discrete Hamiltonian
constraint leaves: E = (R + 2/3 K^2 - At.At)/(16 pi) - 1/2 chi gt^ij d_i phi d_j phi.

What pins it, independently of its own formula:
* the full constraint evaluation (scalar + fluid sources) gives H = 0 to
  rounding and M = 0 exactly;
* with zeta = 0 the metric is homogeneous, R = 0 exactly, and E must approach
  3 H0^2/(8 pi) - 1/2 chi |grad Upsilon|^2 with the ANALYTIC gradient of the
  Gaussian at 4th order in h (interior points, away from the periodic seam);
* with Upsilon = 0 the data are bitwise those of kind 1.
"""
import numpy as np

H0 = 40.0
W = 1.0 / 3.0


def params(O):
    return O.params_array(slicing=0, shift=1, fluid=1, scalar=1, w=W, H0=H0)


def grid(O, n):
    h = 1.0 / n
    return O.OGrid((n, n, n), h, x0=(-(n // 2) * h,) * 3)


def test_isocurvature_data_satisfy_the_discrete_constraints(O):
    n = 24
    g, P = grid(O, n), params(O)
    s = O.init(g, P, O.id_array(2, A=0.02, mu=0.3, sigma=0.125, q=(1.0, 0.9, 1.1)))
    phi, Pi = s[28], s[29]
    assert np.all(Pi == 0.0) and np.abs(phi).max() > 0.019
    hm, norms = O.constraints(g, P, s)
    scale = 6.0 * H0 ** 2  # background size of each term of H
    assert np.abs(hm[0]).max() <= 1e-12 * scale
    assert np.all(hm[1:] == 0.0)


def test_isocurvature_energy_converges_to_the_analytic_gradient_energy(O):
    A, sigma = 0.05, 0.125
    errs = []
    for n in (16, 32, 64):
        g, P = grid(O, n), params(O)
        s = O.init(g, P, O.id_array(2, A=A, mu=0.0, sigma=sigma))
        h = 1.0 / n
        x = -(n // 2) * h + h * np.arange(n)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        ups = A * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * sigma ** 2))
        grad2 = ups ** 2 * (X ** 2 + Y ** 2 + Z ** 2) / sigma ** 4
        chi = s[0]
        assert np.all(chi == 1.0)
        E_exact = 3.0 * H0 ** 2 / (8.0 * np.pi) - 0.5 * chi * grad2
        E = s[24] * chi ** 1.5  # tau~ = sqrt(gamma) E
        inner = (np.abs(X) < 0.25) & (np.abs(Y) < 0.25) & (np.abs(Z) < 0.25)
        errs.append(np.abs(E - E_exact)[inner].max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12.0 < r1 < 20.0 and 13.0 < r2 < 19.0, errs


def test_isocurvature_without_upsilon_equals_the_adiabatic_data(O):
    n = 12
    g, P = grid(O, n), params(O)
    a = O.init(g, P, O.id_array(2, A=0.0, mu=0.4, sigma=0.2))
    b = O.init(g, P, O.id_array(1, mu=0.4, sigma=0.2))
    assert np.array_equal(a, b)

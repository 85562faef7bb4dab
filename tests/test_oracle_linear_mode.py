"""Single-mode perturbation of the radiation FLRW universe against linear theory.

The paper's first example (section "Examples", evolution of a single-mode
perturbation) compares the trace of the extrinsic curvature of a small
sinusoidal fluctuation with the solution of the linear perturbation equations.
Here the same comparison pins the oracle's coupled BSSN + fluid system.

Background: w = 1/3, a(t) = (1 + 2 H0 t)^(1/2), H = H0/(1 + 2 H0 t), chi_b = a^-2,
K_b = -3 H, E_b = 3 H^2/(8 pi), tau_b = a^3 E_b; harmonic slicing with the
background trace, d_t alpha = -alpha^2 (K - K_ref), and a frozen shift.
Perturbation: alpha = 1 + eps cos(k x) at t = 0, every other field at its
background value.  To first order in eps, every field is a multiple of e^{ikx};
with chi = chi_b (1 + c), gt_xx = 1 + g1, gt_yy = gt_zz = 1 + g2, K = K_b + kap,
At_xx = A1, At_yy = At_zz = A2, Gt^x = G, alpha = 1 + a, tau~ = tau_b + y,
S~_x = z, the BSSN and fluid equations linearise to (derived here from the
equations of motion, X_ij = -D_iD_j alpha + alpha (R_ij - 8 pi S_ij)):

  c'   = 2/3 (kap + a K_b)
  g1'  = -2 A1,   g2' = -2 A2
  kap' = chi_b k^2 a + a (K_b^2/3 + 4 pi (1+3w) E_b) + 2/3 K_b kap + 4 pi (1+3w) dE,
         dE = chi_b^(3/2) (y + 3/2 tau_b c)
  a'   = -kap
  X_xx - X_yy = k^2 a + k^2 (g1 - g2)/2 + i k G - k^2 c/2
  A1'  = 2/3 chi_b (X_xx - X_yy) + K_b A1,   A2' = -1/3 chi_b (X_xx - X_yy) + K_b A2
  G'   = -4/3 i k kap - 16 pi chi_b^(3/2) z
  y'   = -i k chi_b z + w (tau_b (a K_b + kap) + y K_b)
  z'   = -i k w (tau_b a + y) - i k tau_b a + i k w tau_b (g1 + 2 g2 - 3 c)/2

(S_ij = P gamma_ij at this order, so its trace-free part vanishes and
K_ij S^ij = P K; the momentum source is (P/2) d_x ln det gamma.)

The oracle runs the full nonlinear discrete system on an N x 1 x 1 grid
(eps = 1e-7, no Kreiss-Oliger); the complex amplitude of the mode in K, At_xx,
Gt^x, alpha, chi, tau~ and S~_x (discrete Fourier projection) is compared with
the linear solution (trK is the paper's observable; the others pin the
trace-free and fluid sectors, which trK alone does not see at this order).
Differences: 4th order for the finite differences and 2nd order for the
Kurganov-Tadmor fluid, so each error must fall by > 3 per doubling of N and
be small at N = 64.
"""
import math

import numpy as np
import pytest

scipy_integrate = pytest.importorskip("scipy.integrate")

W = 1.0 / 3.0
H0 = 2.0
EPS = 1e-7
T_END = 0.5


def background(t):
    s = 1.0 + 2.0 * H0 * t
    a_s = math.sqrt(s)
    H = H0 / s
    E = 3.0 * H * H / (8.0 * math.pi)
    return a_s ** -2, -3.0 * H, E, a_s ** 3 * E


def linear_rhs(t, u, k):
    c, g1, g2, kap, a, A1, A2, G, y, z = u
    chi, K, E, tau = background(t)
    dE = chi ** 1.5 * (y + 1.5 * tau * c)
    X = k * k * a + 0.5 * k * k * (g1 - g2) + 1j * k * G - 0.5 * k * k * c
    return np.array([
        2.0 / 3.0 * (kap + a * K),
        -2.0 * A1,
        -2.0 * A2,
        chi * k * k * a + a * (K * K / 3.0 + 4.0 * math.pi * (1.0 + 3.0 * W) * E) + 2.0 / 3.0 * K * kap
        + 4.0 * math.pi * (1.0 + 3.0 * W) * dE,
        -kap,
        2.0 / 3.0 * chi * X + K * A1,
        -1.0 / 3.0 * chi * X + K * A2,
        -4.0 / 3.0 * 1j * k * kap - 16.0 * math.pi * chi ** 1.5 * z,
        -1j * k * chi * z + W * (tau * (a * K + kap) + y * K),
        -1j * k * W * (tau * a + y) - 1j * k * tau * a + 1j * k * W * tau * 0.5 * (g1 + 2.0 * g2 - 3.0 * c),
    ], dtype=complex)


# fields compared: (name, state index, linear variable, scale by chi_b)
COMPARED = [("K", 7, 3, False), ("At_xx", 8, 5, False), ("Gt^x", 14, 7, False), ("alpha", 17, 4, False),
            ("chi", 0, 0, True), ("tau", 24, 8, False), ("S_x", 25, 9, False)]


def linear_solution(times, k):
    u0 = np.zeros(10, dtype=complex)
    u0[4] = EPS
    sol = scipy_integrate.solve_ivp(linear_rhs, (0.0, times[-1]), u0, method="DOP853", t_eval=times, args=(k,),
                                    rtol=1e-12, atol=1e-24)
    assert sol.success
    return sol.y


def oracle_modes(O, n, record_every):
    """Complex amplitude F of each compared field, f(x) = f_mean + Re(F e^{ikx}) + ...,
    by the discrete Fourier projection over the grid."""
    h = 1.0 / n
    g = O.OGrid((n, 1, 1), h)
    P = O.params_array(slicing=1, shift=0, ko_sigma=0.0, fluid=1, w=W, H0=H0)
    s = np.zeros((28, 1, 1, n))
    x = h * np.arange(n)
    s[0] = 1.0
    s[1] = s[4] = s[6] = 1.0
    s[7] = -3.0 * H0
    s[17] = 1.0 + EPS * np.cos(2.0 * np.pi * x)
    s[24] = 3.0 * H0 * H0 / (8.0 * np.pi)
    phase = np.exp(-2j * np.pi * x) * (2.0 / n)
    dt = 0.25 * h
    steps = int(round(T_END / dt))
    times, amps = [0.0], [[s[f, 0, 0] @ phase for _, f, _, _ in COMPARED]]
    for m in range(steps):
        O.rk4_step(g, P, s, m * dt, dt)
        if (m + 1) % record_every == 0:
            times.append((m + 1) * dt)
            amps.append([s[f, 0, 0] @ phase for _, f, _, _ in COMPARED])
    return np.array(times), np.array(amps).T


def mode_errors(t, amps, k):
    lin = linear_solution(t, k)
    chi_b = np.array([background(tt)[0] for tt in t])
    errs = {}
    for (name, _, v, by_chi), amp in zip(COMPARED, amps):
        ref = lin[v] * (chi_b if by_chi else 1.0)
        errs[name] = np.abs(amp - ref).max() / np.abs(ref).max()
    return errs


def test_single_mode_follows_linear_theory(O):
    k = 2.0 * np.pi
    runs = [mode_errors(*oracle_modes(O, n, every), k) for n, every in ((16, 2), (32, 4), (64, 8))]
    for name in runs[0]:
        e = [r[name] for r in runs]
        assert e[2] < 5e-3, (name, e)
        assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, (name, e)

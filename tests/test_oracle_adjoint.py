"""The oracle's reverse mode against its own (pinned) forward map.

For random directions v and cotangents w,  <w, (F(U + e v) - F(U - e v)) / 2e>
must equal <(dF/dU)^T w, v> to the accuracy of the central difference (the
tape is exact; the difference has O(e^2) truncation and O(eps/e) rounding).
The same holds for one RK4 step.  A wrong partial anywhere on the tape, a
dropped dependency (e.g. a neighbour's derivative or face flux treated as a
constant) or a wrong reverse of the RK4 combine breaks the equality.
"""
import numpy as np
import pytest

from paper_2606_02053_gb300 import inputs


def dot_test(fwd, vjp, U, seed, eps=(1e-7, 5e-8, 2.5e-8)):
    """The fluid's minmod limiter and max |speed| make the discrete map only
    piecewise smooth; a difference step that crosses a kink is not a
    derivative, so the closest of a few small steps is compared."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(U.shape)
    w = rng.standard_normal(U.shape)
    rhs = float(np.sum(vjp(w) * v))
    best = None
    for e in eps:
        jv = (fwd(U + e * v) - fwd(U - e * v)) / (2 * e)
        lhs = float(np.sum(w * jv))
        if best is None or abs(lhs - rhs) < abs(best - rhs):
            best = lhs
    return best, rhs


@pytest.mark.parametrize("fluid", [0, 1])
def test_rhs_vjp_matches_directional_derivative(O, fluid):
    n = (7, 6, 6)
    h = 1.0 / 7
    g = O.OGrid(n, h)
    P = O.params_array(slicing=0, shift=1, eta=1.3, ko_sigma=0.2, fluid=fluid, H0=2.0 * fluid)
    U = inputs.smooth_state(n, seed=40 + fluid, fluid=fluid, scale=0.5)
    lhs, rhs = dot_test(lambda X: O.rhs(g, P, np.ascontiguousarray(X), 0.1),
                        lambda w: O.rhs_vjp(g, P, U, w, 0.1), U, seed=1)
    assert abs(lhs - rhs) <= 1e-8 * abs(rhs), (lhs, rhs)


def test_rhs_vjp_is_linear_and_exact_for_kreiss_oliger(O):
    """On flat space with frozen shift only KO and the linearised algebra act;
    the KO part is symmetric: the VJP of a KO-only map equals the map itself."""
    n = (8, 6, 7)
    g = O.OGrid(n, 0.1)
    P = O.params_array(slicing=1, shift=0, ko_sigma=0.3)
    U = np.zeros((24, n[2], n[1], n[0]))
    U[0] = 1.0
    U[1] = U[4] = U[6] = 1.0
    U[17] = 1.0
    rng = np.random.default_rng(3)
    w = np.zeros_like(U)
    w[21] = rng.standard_normal(w[21].shape)  # B^x: d_t B = KO(B) only (frozen shift)
    v = O.rhs_vjp(g, P, U, w)
    Bp = U.copy()
    Bp[21] = w[21]
    ko = O.rhs(g, P, Bp)[21]
    np.testing.assert_allclose(v[21], ko, rtol=0, atol=1e-12 * np.abs(ko).max())


@pytest.mark.parametrize("fluid", [0, 1])
def test_rk4_adjoint_matches_directional_derivative(O, fluid):
    n = (6, 7, 6)
    h = 1.0 / 7
    g = O.OGrid(n, h)
    P = O.params_array(slicing=0, shift=1, eta=1.0, ko_sigma=0.1, fluid=fluid, H0=2.0 * fluid)
    U = inputs.smooth_state(n, seed=50 + fluid, fluid=fluid, scale=0.5)
    dt = 0.25 * h

    def step(X):
        Y = np.ascontiguousarray(X).copy()
        O.rk4_step(g, P, Y, 0.05, dt)
        return Y

    lhs, rhs = dot_test(step, lambda lam: O.adjoint_step(g, P, U, lam, 0.05, dt), U, seed=2)
    assert abs(lhs - rhs) <= 1e-8 * abs(rhs), (lhs, rhs)

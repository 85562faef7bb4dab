"""Edge cases of the derivative pass's exact integer arithmetic (every field's
values as 64-bit fixed point relative to the field's largest exponent, stencil
sums formed exactly, each result rounded once), through cosmos_rhs against the
oracle's FP64 right-hand side:

* fields scaled to extreme binary exponents (2^-600, 2^+600): the fixed-point
  scale follows each field, so the derivatives keep full relative accuracy;
* a field with a wide dynamic range inside the grid (an O(1) part and a 1e-30
  part elsewhere): the small values are held to 2^-62 of the field's largest
  value, far below the tolerance;
* a field of denormal values only;
* a non-finite value in one field: it must show in the output (NaN), never be
  replaced by a finite number.

Tolerance as in test_gpu_parity: per field, 1e-12 of the field's largest
right-hand side (floor 1e-12 of the largest over all fields).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-12


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


def rhs_both(C, O, state, p, n, pitch=None):
    from paper_2606_02053_gb300.evolve import Evolution

    h = 1.0 / n[0]
    ev = Evolution(C.make_grid(n, h, pitch=pitch), p)
    ev.set_state(state)
    r = ev.get(ev.rhs(0.0))
    ref = O.rhs(O.OGrid(n, h), O.params_array(slicing=p.slicing, shift=p.shift, eta=p.eta, ko_sigma=p.ko_sigma,
                                              w=p.w, fluid=p.fluid, scalar=p.scalar, H0=p.H0, t0=p.t0), state, 0.0)
    return r, ref


def test_extreme_binary_exponents(C, O):
    """Shift-type fields at 2^-600 and the driver fields at 2^+600: linear in the
    RHS where they appear alone, so the oracle's values are exact references."""
    from paper_2606_02053_gb300 import inputs

    n = (20, 14, 12)
    s = inputs.smooth_state(n, seed=901)
    s[18:21] *= 2.0 ** -600  # beta^i
    s[21:24] *= 2.0 ** 600   # B^i
    p = C.make_params(slicing=0, shift=1, eta=1.3, ko_sigma=0.1)
    r, ref = rhs_both(C, O, s, p, n, pitch=24)
    assert np.all(np.isfinite(r))
    scale = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    err = np.abs(r - ref).reshape(r.shape[0], -1).max(axis=1) / np.maximum(scale, 1e-300)
    assert err.max() <= RHS_TOL, (err.argmax(), err.max())


def test_wide_dynamic_range_inside_a_field(C, O):
    from paper_2606_02053_gb300 import inputs

    n = (24, 10, 9)
    s = inputs.smooth_state(n, seed=902)
    # K: O(1) in the lower half of x, 1e-30 times itself in the upper half (a step in scale)
    s[7, :, :, n[0] // 2:] *= 1e-30
    p = C.make_params(slicing=1, shift=0, ko_sigma=0.2)
    r, ref = rhs_both(C, O, s, p, n)
    assert field_errors(r, ref).max() <= RHS_TOL


def test_denormal_field(C, O):
    from paper_2606_02053_gb300 import inputs

    n = (16, 8, 8)
    s = inputs.smooth_state(n, seed=903)
    s[14] = 1e-310 * np.sign(s[14])  # Gt^x: denormals of both signs
    p = C.make_params(slicing=0, shift=1)
    r, ref = rhs_both(C, O, s, p, n)
    assert field_errors(r, ref).max() <= RHS_TOL


def test_non_finite_value_is_not_hidden(C, O):
    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300.evolve import Evolution

    n = (16, 8, 8)
    s = inputs.smooth_state(n, seed=904)
    s[8, 3, 4, 5] = np.nan  # At_xx
    p = C.make_params(slicing=0, shift=1)
    ev = Evolution(C.make_grid(n, 1.0 / 16), p)
    ev.set_state(s)
    r = ev.get(ev.rhs(0.0))
    # the field's derivatives (its advection and KO terms) are NaN at every point, not finite numbers
    assert np.isnan(r[8]).all()


@pytest.mark.parametrize("n", [(35, 11, 3), (34, 11, 3), (35, 10, 3), (35, 11, 2), (70, 19, 5)])
def test_periodic_wrap_on_both_sides_of_the_division_free_threshold(C, O, n):
    """The pass wraps its periodic neighbour indices with one compare and
    select when every index of a tile lies in [-n, 2n) (nx >= 35, ny >= 11,
    nz >= 3), else by integer division; grids on both sides of that line,
    with tiles that overhang the grid's end, against the oracle."""
    from paper_2606_02053_gb300 import inputs

    s = inputs.smooth_state(n, seed=905 + sum(n))
    p = C.make_params(slicing=0, shift=1, eta=1.1, ko_sigma=0.15)
    r, ref = rhs_both(C, O, s, p, n)
    assert field_errors(r, ref).max() <= RHS_TOL

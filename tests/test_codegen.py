"""Host-side checks of the generated pointwise algebra (no GPU).

* the committed generated header matches what the generator writes now;
* the generated algebra, interpreted on the CPU with derivatives from the
  same finite-difference stencils, reproduces the oracle right-hand side
  (Kreiss-Oliger off) at sample points, for every matter variant.
"""
import numpy as np
import pytest

from paper_2606_02053_gb300 import inputs
from paper_2606_02053_gb300.codegen import bssn, generate
from paper_2606_02053_gb300.codegen import fluid as fluid_dsl
from paper_2606_02053_gb300.codegen.expr import evaluate


def test_generated_header_is_up_to_date():
    assert generate.main(["--check"]) == 0


def _fd_inputs(s, p, h, L, fluid, w):
    """Inputs of the algebra at point p = (i, j, k) from 4th-order FD."""
    nz, ny, nx = s.shape[1:]
    i, j, k = p

    def at(f, di=0, dj=0, dk=0):
        return s[f, (k + dk) % nz, (j + dj) % ny, (i + di) % nx]

    def off(d, o):
        return [(o, 0, 0), (0, o, 0), (0, 0, o)][d]

    def D1(f, d, base=(0, 0, 0)):
        a = [base[m] + off(d, 1)[m] for m in range(3)]
        b = [base[m] + off(d, -1)[m] for m in range(3)]
        c = [base[m] + off(d, 2)[m] for m in range(3)]
        e = [base[m] + off(d, -2)[m] for m in range(3)]
        return (8 * (at(f, *a) - at(f, *b)) - (at(f, *c) - at(f, *e))) / (12 * h)

    def D2(f, d):
        f0 = at(f)
        s1 = (at(f, *off(d, 1)) - f0) + (at(f, *off(d, -1)) - f0)
        s2 = (at(f, *off(d, 2)) - f0) + (at(f, *off(d, -2)) - f0)
        return (16 * s1 - s2) / (12 * h * h)

    def Dm(f, a, b):
        m1 = D1(f, b, off(a, 1)) - D1(f, b, off(a, -1))
        m2 = D1(f, b, off(a, 2)) - D1(f, b, off(a, -2))
        return (8 * m1 - m2) / (12 * h)

    vals = {}
    for f in range(L["nf"]):
        vals[f"u{f}"] = at(f)
    for f in L["d1"]:
        for d in range(3):
            vals[f"d{f}_{d}"] = D1(f, d)
    for f in L["d2"]:
        for m, (a, b) in enumerate(bssn.PAIRS):
            vals[f"dd{f}_{m}"] = D2(f, a) if a == b else Dm(f, a, b)
    if fluid:
        # fluid rest-frame density from (tau, S_i) and the metric at the point
        chi = at(0)
        gt = np.zeros((3, 3))
        for m, (a, b) in enumerate(bssn.PAIRS):
            gt[a, b] = gt[b, a] = at(1 + m)
        gu = np.linalg.inv(gt) * chi
        c32 = chi * np.sqrt(chi)
        E = at(24) * c32
        J = np.array([at(25 + q) for q in range(3)]) * c32
        J2 = J @ gu @ J
        a_ = (1 - w) * E
        vals["rho"] = (np.sqrt(a_ * a_ + 4 * w * (E * E - J2)) - a_) / (2 * w)
    return vals


def _flux_divergence(s, p, h, w):
    """sum_d (H_d(p) - H_d(p - e_d)) / h from the generated prim / face-flux graphs."""
    nz, ny, nx = s.shape[1:]
    gp, pn, po = fluid_dsl.prim()
    fp = dict(w=w, sqrt_w=np.sqrt(w))

    def cell(c):
        i, j, k = c[0] % nx, c[1] % ny, c[2] % nz
        return s[:, k, j, i]

    def prim_at(c):
        v = cell(c)
        vals = dict(chi=v[0], tau=v[24], S0=v[25], S1=v[26], S2=v[27])
        vals.update({f"gt{m}": v[1 + m] for m in range(6)})
        return evaluate(gp, po, vals, fp)

    def face(c, d):
        gf, fn, fo = fluid_dsl.face_flux(d)
        vals = {}
        for o in range(4):
            cc = list(c)
            cc[d] += o - 1
            q = prim_at(cc)
            for mm in range(4):
                vals[f"q{o}_{mm}"] = q[mm]
        for sd in range(2):
            cc = list(c)
            cc[d] += sd
            v = cell(cc)
            vals[f"chi{sd}"], vals[f"alpha{sd}"], vals[f"beta{sd}"] = v[0], v[17], v[18 + d]
            for mm in range(6):
                vals[f"gt{sd}_{mm}"] = v[1 + mm]
        return np.array(evaluate(gf, fo, vals, fp), dtype=float)

    div = np.zeros(4)
    for d in range(3):
        cm = list(p)
        cm[d] -= 1
        div += (face(list(p), d) - face(cm, d)) / h
    return div


@pytest.mark.parametrize("fluid,scalar", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_generated_algebra_matches_oracle(O, fluid, scalar):
    n = 12
    h = 1.0 / n
    g = O.OGrid((n, n, n), h)
    w = 1.0 / 3.0
    Kref = -0.7
    P = O.params_array(slicing=0, shift=1, eta=1.5, ko_sigma=0.0, w=w, fluid=fluid, scalar=scalar, H0=0.0)
    s = inputs.smooth_state(n, seed=21, fluid=fluid, scalar=scalar)
    pts = [(3, 5, 7), (0, 11, 2), (9, 1, 10)]
    ref = O.rhs_points(g, P, s, pts)
    gr, L, out = bssn.algebra(bool(fluid), bool(scalar))
    params = dict(eta=1.5, Kref=0.0, lapse_c1=2.0, lapse_c2=0.0, shift_on=1.0, w=w)
    for m, p in enumerate(pts):
        vals = _fd_inputs(s, p, h, L, fluid, w)
        got = np.array(evaluate(gr, out, vals, params), dtype=float)
        r = ref[m]
        if fluid:
            got[24:28] -= _flux_divergence(s, p, h, w)
        idx = list(range(L["nf"]))
        scale = np.abs(r[idx]).max()
        err = np.abs(got[idx] - r[idx]).max() / scale
        assert err < 1e-12, (p, err, np.argmax(np.abs(got[idx] - r[idx])))
    # K_ref enters the lapse equation only, linearly
    vals = _fd_inputs(s, pts[0], h, L, fluid, w)
    a = evaluate(gr, out, vals, params)[17]
    b = evaluate(gr, out, vals, dict(params, Kref=Kref))[17]
    np.testing.assert_allclose(b - a, 2.0 * vals["u17"] * Kref, rtol=1e-12)

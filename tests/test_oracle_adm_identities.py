"""Oracle right-hand side and constraints against exact 3+1 identities.

A generic smooth spacetime with fluid and scalar matter is written in closed
form (``spacetime_ad.Spacetime``); torch autodiff supplies the exact time
derivative of every evolved variable and the 4D Einstein tensor, div T and
box phi at a few sample points.  The oracle, run on grids of spacing 1/16,
1/32 and 1/64 that contain those points, must converge to the identities at
the order of its discretisation:

* BSSN variables and scalar field: 4th order (ratio ~16 per halving);
* fluid (Kurganov-Tadmor, minmod): 2nd order for monotone primitives, and
  at least 1st order (limiter clipping at extrema) in general.

A dropped term, a wrong sign or index, or a transposed operand anywhere in
the algebra leaves an O(1) residual that does not converge.
Only the grid points within reach of the stencils around each sample point
are filled from the closed form; the rest of the grid holds flat filler.
"""
import numpy as np
import pytest
import torch

from spacetime_ad import ALP, BB, BET, CHI, GAM, Spacetime, implied_adm_rates, sample_state

PHYS = [(0.25, 0.5, 0.75), (0.5, 0.125, 0.375), (0.8125, 0.6875, 0.0625)]
NS = (16, 32, 64)
REACH = 4


def local_state(st, n, centers, nf):
    h = 1.0 / n
    s = np.zeros((nf, n, n, n))
    s[CHI] = 1.0
    s[1] = s[4] = s[6] = 1.0
    s[ALP] = 1.0
    if st.fluid:
        s[24] = 1.0
    idx = set()
    for c in centers:
        for dk in range(-REACH, REACH + 1):
            for dj in range(-REACH, REACH + 1):
                for di in range(-REACH, REACH + 1):
                    idx.add(((c[0] + di) % n, (c[1] + dj) % n, (c[2] + dk) % n))
    idx = np.array(sorted(idx))
    X = torch.tensor(np.c_[np.zeros(len(idx)), idx * h], dtype=torch.float64)
    vals = sample_state(st, X).numpy()
    s[:, idx[:, 2], idx[:, 1], idx[:, 0]] = vals.T
    return s


def run_identities(O, st, params, eta):
    nf = O.nfields(params)
    exp = [st.expected(torch.tensor([0.0, *p], dtype=torch.float64), eta=eta) for p in PHYS]
    errs = {}
    for n in NS:
        centers = [tuple(int(round(c * n)) for c in p) for p in PHYS]
        s = local_state(st, n, centers, nf)
        g = O.OGrid((n, n, n), 1.0 / n)
        r = O.rhs_points(g, params, s, centers)
        hm, _ = O.constraints(g, params, s)
        e = {}
        for m, c in enumerate(centers):
            ex = exp[m]
            stv = s[:, c[2], c[1], c[0]]
            gdot, Kdot = implied_adm_rates(stv, r[m])
            er = np.abs(r[m] - ex["rhs"].numpy())
            cur = dict(gdot=np.abs(gdot - ex["gdot"].numpy()).max(), Kdot=np.abs(Kdot - ex["Kdot"].numpy()).max(),
                       chi=er[CHI], Gam=er[GAM:GAM + 3].max(), alp=er[ALP], beta=er[BET:BET + 3].max(),
                       B=er[BB:BB + 3].max(),
                       ham=abs(hm[0, c[2], c[1], c[0]] - ex["ham"].item()),
                       mom=np.abs(hm[1:, c[2], c[1], c[0]] - ex["mom"].numpy()).max())
            off = 24
            if st.fluid:
                cur["tau"] = er[off]
                cur["S"] = er[off + 1:off + 4].max()
                off += 4
            if st.scalar:
                cur["phi"] = er[off]
                cur["Pi"] = er[off + 1]
            for k, v in cur.items():
                e[k] = max(e.get(k, 0.0), v)
        errs[n] = e
    return errs


def ratios(errs, key):
    return errs[16][key] / errs[32][key], errs[32][key] / errs[64][key]


BSSN_KEYS = ["gdot", "Kdot", "chi", "Gam", "alp", "beta", "B", "ham", "mom"]


def assert_4th(errs, keys):
    for k in keys:
        r1, r2 = ratios(errs, k)
        assert r2 > 13.0 and r1 > 8.0, (k, [errs[n][k] for n in NS], r1, r2)


def test_g4inv_closed_form_matches_generic_inverse():
    st = Spacetime(seed=5)
    X = torch.tensor([0.1, 0.3, 0.6, 0.9], dtype=torch.float64)
    assert torch.allclose(st.g4inv(X), torch.linalg.inv(st.g4(X)), rtol=1e-13, atol=1e-13)


def test_vacuum_bssn_identities_4th_order(O):
    st = Spacetime(seed=1, fluid=False, scalar=False)
    P = O.params_array(slicing=0, shift=1, eta=2.0, ko_sigma=0.0, fluid=0, scalar=0)
    errs = run_identities(O, st, P, eta=2.0)
    assert_4th(errs, BSSN_KEYS)


def test_matter_bssn_scalar_identities_4th_order_fluid_converges(O):
    st = Spacetime(seed=2, fluid=True, scalar=True)
    P = O.params_array(slicing=0, shift=1, eta=2.0, ko_sigma=0.0, w=1.0 / 3.0, fluid=1, scalar=1)
    errs = run_identities(O, st, P, eta=2.0)
    assert_4th(errs, BSSN_KEYS + ["phi", "Pi"])
    for k in ("tau", "S"):
        r1, r2 = ratios(errs, k)
        assert r1 > 1.4 and r2 > 1.4, (k, [errs[n][k] for n in NS])


def test_monotone_fluid_kt_2nd_order(O):
    st = Spacetime(seed=1, fluid=True, scalar=False, monotone_fluid=True)
    P = O.params_array(slicing=0, shift=1, eta=2.0, ko_sigma=0.0, w=1.0 / 3.0, fluid=1, scalar=0)
    errs = run_identities(O, st, P, eta=2.0)
    assert_4th(errs, BSSN_KEYS)
    for k in ("tau", "S"):
        r1, r2 = ratios(errs, k)
        assert r2 > 3.3, (k, [errs[n][k] for n in NS], r1, r2)


@pytest.mark.parametrize("w", [0.2, 0.6])
def test_fluid_identities_other_eos(O, w):
    """The equation-of-state parameter enters recovery, pressure and speeds."""
    st = Spacetime(seed=3, fluid=True, scalar=False, monotone_fluid=True, w=w)
    P = O.params_array(slicing=1, shift=1, eta=1.0, ko_sigma=0.0, w=w, fluid=1, scalar=0)
    errs = run_identities(O, st, P, eta=1.0)
    for k in ("Kdot", "Gam", "tau", "S"):
        r1, r2 = ratios(errs, k)
        assert r2 > 3.3, (k, [errs[n][k] for n in NS], r1, r2)

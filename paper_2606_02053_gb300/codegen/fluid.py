"""Fluid pieces of the right-hand side in the expression DSL.

Perfect fluid with P = w rho (section "Physical system settings"), evolved in
conservative 3+1 form (tau~ = sqrt(gamma) E, S~_i = sqrt(gamma) J_i) with the
Kurganov-Tadmor central scheme (the paper's fluid method):

* ``prim``: cell-centred recovery of (rho, v_i) from (tau~, S~_i).  With
  h W^2 = (1 + w) rho W^2:  E = h W^2 - w rho,  J_i = h W^2 v_i, hence
  w rho^2 + (1 - w) E rho + (J^2 - E^2) = 0 and rho is its positive root.
* ``face_flux(d)``: numerical flux through the face between cells c and
  c + e_d: minmod-limited linear reconstruction of (rho, v_i) from cells
  c-1 .. c+2, face metric = mean of the two adjacent cells, and
  H = (F(q_L) + F(q_R))/2 - a (U(q_R) - U(q_L))/2 with a the largest
  |characteristic speed| of both states, speeds
  lambda_pm = alpha/(1 - v^2 w) [v^d (1 - w) pm sqrt(w (1 - v^2)(gamma^dd (1 - v^2 w) - v^d v^d (1 - w)))] - beta^d.
"""
from __future__ import annotations

from .expr import Graph, fabs, fmax, minmod, sqrt

PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
PIDX = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 0): 1, (1, 1): 3, (1, 2): 4, (2, 0): 2, (2, 1): 4, (2, 2): 5}


def _inv_sym(gt):
    c00 = gt[3] * gt[5] - gt[4] * gt[4]
    c01 = gt[2] * gt[4] - gt[1] * gt[5]
    c02 = gt[1] * gt[4] - gt[2] * gt[3]
    c11 = gt[0] * gt[5] - gt[2] * gt[2]
    c12 = gt[1] * gt[2] - gt[0] * gt[4]
    c22 = gt[0] * gt[3] - gt[1] * gt[1]
    idet = (gt[0] * c00 + gt[1] * c01 + gt[2] * c02).rcp()
    return [c00 * idet, c01 * idet, c02 * idet, c11 * idet, c12 * idet, c22 * idet]


def prim():
    """Inputs: chi, gt[6], tau, S[3]  ->  outputs rho, v_0, v_1, v_2."""
    g = Graph()
    names = ["chi"] + [f"gt{m}" for m in range(6)] + ["tau", "S0", "S1", "S2"]
    x = {n: g.input(n) for n in names}
    w = g.param("w")
    chi = x["chi"]
    gu = _inv_sym([x[f"gt{m}"] for m in range(6)])
    chi32 = chi * sqrt(chi)
    E = x["tau"] * chi32
    J = [x[f"S{i}"] * chi32 for i in range(3)]
    wJ = [gu[PIDX[(i, 0)]] * J[0] + gu[PIDX[(i, 1)]] * J[1] + gu[PIDX[(i, 2)]] * J[2] for i in range(3)]
    J2 = chi * (wJ[0] * J[0] + wJ[1] * J[1] + wJ[2] * J[2])
    a = (1.0 - w) * E
    # positive root, rationalised to avoid cancellation: 2 (E^2 - J^2) / (a + sqrt(a^2 + 4 w (E^2 - J^2)))
    D = E * E - J2
    rho = 2.0 * D * (a + sqrt(a * a + 4.0 * w * D)).rcp()
    iEP = (E + w * rho).rcp()
    out = [rho] + [J[i] * iEP for i in range(3)]
    return g, names, out


def face_flux(d: int):
    """Inputs: rho/v at cells c-1..c+2 (q{o}_{m}, o = 0..3, m = rho, v0..2) and
    metric at cells c, c+1 (chi{s}, alpha{s}, beta{s} (component d), gt{s}_{m}).
    Outputs: H_tau, H_S0, H_S1, H_S2."""
    g = Graph()
    names = [f"q{o}_{m}" for o in range(4) for m in range(4)]
    for s in range(2):
        names += [f"chi{s}", f"alpha{s}", f"beta{s}"] + [f"gt{s}_{m}" for m in range(6)]
    x = {n: g.input(n) for n in names}
    w = g.param("w")
    sqw = g.param("sqrt_w")
    q = [[x[f"q{o}_{m}"] for m in range(4)] for o in range(4)]
    qL = [q[1][m] + 0.5 * minmod(q[1][m] - q[0][m], q[2][m] - q[1][m]) for m in range(4)]
    qR = [q[2][m] - 0.5 * minmod(q[2][m] - q[1][m], q[3][m] - q[2][m]) for m in range(4)]
    chi = 0.5 * (x["chi0"] + x["chi1"])
    alpha = 0.5 * (x["alpha0"] + x["alpha1"])
    betad = 0.5 * (x["beta0"] + x["beta1"])
    gt = [0.5 * (x[f"gt0_{m}"] + x[f"gt1_{m}"]) for m in range(6)]
    gtu = _inv_sym(gt)
    gu = [chi * c for c in gtu]
    sqrtg = (chi * sqrt(chi)).rcp()
    one_m_w = 1.0 - w
    U, F, lam = [], [], []
    for side in (qL, qR):
        rho, v = side[0], side[1:]
        vu = [gu[PIDX[(i, 0)]] * v[0] + gu[PIDX[(i, 1)]] * v[1] + gu[PIDX[(i, 2)]] * v[2] for i in range(3)]
        v2 = vu[0] * v[0] + vu[1] * v[1] + vu[2] * v[2]
        W2 = (1.0 - v2).rcp()
        P = w * rho
        hW2 = (rho + P) * W2
        E = hW2 - P
        J = [hW2 * v[i] for i in range(3)]
        # densitised by sqrt(gamma) once per face, below, instead of per component
        Ui = [E] + [J[i] for i in range(3)]
        Fi = [alpha * hW2 * vu[d] - betad * E]
        for i in range(3):
            Sdi = hW2 * vu[d] * v[i] + (P if i == d else 0.0)
            Fi.append(alpha * Sdi - betad * J[i])
        disc = (1.0 - v2) * (gu[PIDX[(d, d)]] * (1.0 - v2 * w) - vu[d] * vu[d] * one_m_w)
        root = sqw * sqrt(disc)
        pre = alpha * (1.0 - v2 * w).rcp()
        lp = pre * (vu[d] * one_m_w + root) - betad
        lm = pre * (vu[d] * one_m_w - root) - betad
        U.append(Ui)
        F.append(Fi)
        lam.append((lp, lm))
    a = fmax(fmax(fabs(lam[0][0]), fabs(lam[0][1])), fmax(fabs(lam[1][0]), fabs(lam[1][1])))
    hs = 0.5 * sqrtg
    out = [hs * ((F[0][m] + F[1][m]) - a * (U[1][m] - U[0][m])) for m in range(4)]
    return g, names, out

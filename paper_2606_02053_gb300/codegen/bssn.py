"""Pointwise BSSN + matter algebra, stated in the expression DSL.

This is the GPU path's own statement of the evolution equations of the paper
(section "Physical system settings": Einstein equations with T = T^SC + T^FL,
P = w rho, box phi = 0, div T^FL = 0), rewritten in the standard BSSN
(chi-variant) form that the paper defers to numerical-relativity textbooks.
It is turned into straight-line CUDA by ``generate.py``.

Inputs at one grid point (layout shared with the stencil kernels):
  in[0 .. NF)                        field values (state order)
  in[NF + 3 m + k]                   d_k of the m-th first-derivative field
  in[NF + 3 ND1 + 6 m + p]           second derivative p = xx,xy,xz,yy,yz,zz
                                     of the m-th second-derivative field
  in[NF + 3 ND1 + 6 ND2]             fluid rest-frame density rho (fluid only)
First-derivative fields: the 24 BSSN fields, then phi, Pi (scalar on).
Second-derivative fields: chi, gt_xx..gt_zz, alpha, beta^x..z, then phi.

Outputs: out[f] = d_t of field f WITHOUT the Kreiss-Oliger term and, for the
fluid fields, without the flux divergence (geometric sources only).

Runtime parameters (struct AlgebraParams): eta (Gamma-driver damping),
Kref (background trace K_ref(t) of the stage time), lapse_c1, lapse_c2
(d_t alpha = beta.d alpha - alpha (c1 + c2 alpha)(K - Kref): 1+log is
c1=2, c2=0; harmonic is c1=0, c2=1), shift_on (1 Gamma-driver, 0 frozen),
w (equation of state).
"""
from __future__ import annotations

import math

from .expr import Graph, sqrt

PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
PIDX = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 0): 1, (1, 1): 3, (1, 2): 4, (2, 0): 2, (2, 1): 4, (2, 2): 5}

CHI, GT, TRK, AT, GAM, ALP, BET, BB = 0, 1, 7, 8, 14, 17, 18, 21
D2_FIELDS_BSSN = [CHI, 1, 2, 3, 4, 5, 6, ALP, BET, BET + 1, BET + 2]


def layout(fluid: bool, scalar: bool):
    nf = 24 + 4 * fluid + 2 * scalar
    d1 = list(range(24))
    d2 = list(D2_FIELDS_BSSN)
    if scalar:
        s = 24 + 4 * fluid
        d1 += [s, s + 1]
        d2 += [s]
    names = [f"u{f}" for f in range(nf)]
    names += [f"d{f}_{k}" for f in d1 for k in range(3)]
    names += [f"dd{f}_{p}" for f in d2 for p in range(6)]
    if fluid:
        names += ["rho"]
    return dict(nf=nf, d1=d1, d2=d2, names=names, nin=len(names))


class Sym:
    """Symmetric 3x3 tensor of expressions stored as 6 components."""

    def __init__(self, c):
        self.c = list(c)

    def __getitem__(self, ij):
        return self.c[PIDX[ij]]


def contract_sym(Mu, N):
    """sum_ij M^ij N_ij for symmetric M, N (M given with doubled off-diagonals)."""
    s = None
    for m, (i, j) in enumerate(PAIRS):
        t = Mu[m] * N[(i, j)]
        s = t if s is None else s + t
    return s


def algebra(fluid: bool, scalar: bool):
    g = Graph()
    L = layout(fluid, scalar)
    nf = L["nf"]
    u = [g.input(f"u{f}") for f in range(nf)]

    def d(f, k):
        return g.input(f"d{f}_{k}")

    def dd(f, i, j):
        return g.input(f"dd{f}_{PIDX[(i, j)]}")

    eta, Kref = g.param("eta"), g.param("Kref")
    c1, c2, shift_on, w = g.param("lapse_c1"), g.param("lapse_c2"), g.param("shift_on"), g.param("w")
    pi = math.pi

    chi, K, alpha = u[CHI], u[TRK], u[ALP]
    gt = Sym(u[GT:GT + 6])
    At = Sym(u[AT:AT + 6])
    Gt = u[GAM:GAM + 3]
    beta = u[BET:BET + 3]
    B = u[BB:BB + 3]
    dchi = [d(CHI, k) for k in range(3)]
    dK = [d(TRK, k) for k in range(3)]
    dal = [d(ALP, k) for k in range(3)]

    def dgt(k, i, j):
        return d(GT + PIDX[(i, j)], k)

    def dAt(k, i, j):
        return d(AT + PIDX[(i, j)], k)

    def dGt(k, i):
        return d(GAM + i, k)

    def dbeta(k, i):
        return d(BET + i, k)

    def dB(k, i):
        return d(BB + i, k)

    def ddgt(l, m, i, j):
        return dd(GT + PIDX[(i, j)], l, m)

    # ---- inverse conformal metric (cofactors / det) ----
    c00 = gt[1, 1] * gt[2, 2] - gt[1, 2] * gt[1, 2]
    c01 = gt[0, 2] * gt[1, 2] - gt[0, 1] * gt[2, 2]
    c02 = gt[0, 1] * gt[1, 2] - gt[0, 2] * gt[1, 1]
    c11 = gt[0, 0] * gt[2, 2] - gt[0, 2] * gt[0, 2]
    c12 = gt[0, 1] * gt[0, 2] - gt[0, 0] * gt[1, 2]
    c22 = gt[0, 0] * gt[1, 1] - gt[0, 1] * gt[0, 1]
    idet = (gt[0, 0] * c00 + gt[0, 1] * c01 + gt[0, 2] * c02).rcp()
    gu = Sym([c00 * idet, c01 * idet, c02 * idet, c11 * idet, c12 * idet, c22 * idet])
    gu2 = [gu[i, j] * (1.0 if i == j else 2.0) for (i, j) in PAIRS]  # doubled off-diagonals
    ichi = chi.rcp()

    # ---- Christoffels: first-kind Gl[k][(i,j)] = Gamma_kij ----
    Gl = []
    for k in range(3):
        row = []
        for (i, j) in PAIRS:
            if i == k:
                row.append(0.5 * dgt(j, k, k))
            elif j == k:
                row.append(0.5 * dgt(i, k, k))
            else:
                row.append(0.5 * (dgt(i, k, j) + dgt(j, k, i) - dgt(k, i, j)))
        Gl.append(Sym(row))
    # second kind Gu[k][(i,j)] = gt^kl Gamma_lij
    Gu = []
    for k in range(3):
        Gu.append(Sym([gu[k, 0] * Gl[0][i, j] + gu[k, 1] * Gl[1][i, j] + gu[k, 2] * Gl[2][i, j] for (i, j) in PAIRS]))

    # ---- conformal Ricci tensor ----
    # R_ij = -1/2 gt^lm d_l d_m gt_ij + gt_k(i d_j) Gt^k + Gd^k Gamma_(ij)k
    #        + (T_ij + T_ji) + U_ij,
    # T_ij = sum_km C[k][m][i] Gamma_jkm, U_ij = sum_kl C[k][l][i] Gamma_klj,
    # C[k][m][i] = gt^ml Gamma^k_li.  The Christoffel products are accumulated
    # into the six components index i by index i, so that only the nine
    # C[.][.][i] of one i exist at a time (fewer values live at once).
    acc = [None] * 6

    def add_to(m, t):
        acc[m] = t if acc[m] is None else acc[m] + t

    for i in range(3):
        Ci = [[gu[m, 0] * Gu[k][0, i] + gu[m, 1] * Gu[k][1, i] + gu[m, 2] * Gu[k][2, i] for m in range(3)]
              for k in range(3)]
        # Gamma_jkm is symmetric in k, m: T_ij sums (C[k][m][i] + C[m][k][i]) Gamma_jkm over k <= m
        Cs = {(k, m): (Ci[k][m] if k == m else Ci[k][m] + Ci[m][k]) for (k, m) in PAIRS}
        for j in range(3):
            s = None
            for (k, m) in PAIRS:
                t = Cs[(k, m)] * Gl[j][k, m]
                s = t if s is None else s + t
            add_to(PIDX[(i, j)], 2.0 * s if i == j else s)  # T_ij into R_ij (T_ii counted twice)
            if j >= i:
                u_ = None
                for k in range(3):
                    for l in range(3):
                        t = Ci[k][l] * Gl[k][l, j]
                        u_ = t if u_ is None else u_ + t
                add_to(PIDX[(i, j)], u_)  # U_ij
    Gd = [contract_sym(gu2, Gu[k]) for k in range(3)]
    # R_ij as one flat sum, the constant factors folded into factors formed once:
    #   -1/2 gt^lm d_l d_m gt_ij          -> (-1/2 gt^lm) d_l d_m gt_ij
    #   gt_k(i d_j) Gt^k                   -> (1/2 gt_ki) d_j Gt^k + (1/2 gt_kj) d_i Gt^k (i != j)
    #   Gd^k Gamma_(ij)k = 1/2 Gd^k d_k gt_ij   (Gamma_ijk + Gamma_jik = d_k gt_ij)
    ngu2 = [-0.5 * x for x in gu2]
    hGd = [0.5 * x for x in Gd]
    hgt = Sym([0.5 * x for x in gt.c])
    Ric = []
    for m, (i, j) in enumerate(PAIRS):
        r = None
        for q, (l, n) in enumerate(PAIRS):
            t = ngu2[q] * ddgt(l, n, i, j)
            r = t if r is None else r + t
        for k in range(3):
            if i == j:
                r = r + gt[k, i] * dGt(i, k)
            else:
                r = r + hgt[k, i] * dGt(j, k) + hgt[k, j] * dGt(i, k)
        for k in range(3):
            r = r + hGd[k] * dgt(k, i, j)
        Ric.append(r + acc[m])
    # the remaining uses of the second-kind Christoffels, formed here so that
    # those 18 values die early
    Gu_dchi = [Gu[0][i, j] * dchi[0] + Gu[1][i, j] * dchi[1] + Gu[2][i, j] * dchi[2] for (i, j) in PAIRS]
    Gu_dal = [Gu[0][i, j] * dal[0] + Gu[1][i, j] * dal[1] + Gu[2][i, j] * dal[2] for (i, j) in PAIRS]
    Aud = [[gu[i, 0] * At[0, j] + gu[i, 1] * At[1, j] + gu[i, 2] * At[2, j] for j in range(3)] for i in range(3)]
    Atu = Sym([Aud[i][0] * gu[0, j] + Aud[i][1] * gu[1, j] + Aud[i][2] * gu[2, j] for (i, j) in PAIRS])
    Atu2 = [Atu[a, b] * (1.0 if a == b else 2.0) for (a, b) in PAIRS]
    GA = [contract_sym(Atu2, Gu[i]) for i in range(3)]

    # chi part: Rchi_ij = (DDchi_ij + gt_ij trDD)/(2chi) - d_i chi d_j chi/(4chi^2) - 3 gt_ij |dchi|^2/(4chi^2)
    wchi = [gu[l, 0] * dchi[0] + gu[l, 1] * dchi[1] + gu[l, 2] * dchi[2] for l in range(3)]  # gt^lm d_m chi
    dchi2 = wchi[0] * dchi[0] + wchi[1] * dchi[1] + wchi[2] * dchi[2]
    DDchi = [dd(CHI, i, j) - Gu_dchi[m] for m, (i, j) in enumerate(PAIRS)]
    trDD = contract_sym(gu2, Sym(DDchi))
    half_ichi = 0.5 * ichi
    q_ichi2 = 0.25 * ichi * ichi
    diag_coef = half_ichi * trDD - 3.0 * q_ichi2 * dchi2
    for m, (i, j) in enumerate(PAIRS):
        Ric[m] = Ric[m] + half_ichi * DDchi[m] + gt[i, j] * diag_coef - q_ichi2 * (dchi[i] * dchi[j])
    Ric = Sym(Ric)

    # ---- lapse derivatives ----
    dchi_dal = wchi[0] * dal[0] + wchi[1] * dal[1] + wchi[2] * dal[2]
    DDa = []
    for m, (i, j) in enumerate(PAIRS):
        s = dd(ALP, i, j) - Gu_dal[m]
        s = s + half_ichi * (dchi[i] * dal[j] + dchi[j] * dal[i] - gt[i, j] * dchi_dal)
        DDa.append(s)
    lap_a = chi * (contract_sym(gu2, Sym([dd(ALP, i, j) for (i, j) in PAIRS]))
                   - (Gd[0] * dal[0] + Gd[1] * dal[1] + Gd[2] * dal[2])) - 0.5 * dchi_dal

    # ---- raised At (Aud, Atu formed above) ----
    AA = contract_sym(Atu2, At)

    # ---- matter ----
    rhoH = None
    Jl = [None, None, None]
    Sl = [None] * 6
    Str = None
    fl = {}
    if fluid:
        q = 24
        tau, St = u[q], u[q + 1:q + 4]
        sq = sqrt(chi)
        chi32 = chi * sq  # 1/sqrt(gamma)
        isg = chi32.rcp()  # sqrt(gamma)
        E = tau * chi32
        J = [St[i] * chi32 for i in range(3)]
        wJ = [gu[i, 0] * J[0] + gu[i, 1] * J[1] + gu[i, 2] * J[2] for i in range(3)]  # gt^ij J_j
        J2 = chi * (wJ[0] * J[0] + wJ[1] * J[1] + wJ[2] * J[2])
        rho = g.input("rho")
        P = w * rho
        iEP = (E + P).rcp()
        Pi_chi = P * ichi  # P gamma_ij = P gt_ij / chi
        Sf = [J[i] * J[j] * iEP + Pi_chi * gt[i, j] for (i, j) in PAIRS]
        rhoH = E
        Jl = list(J)
        Sl = list(Sf)
        Str = J2 * iEP + 3.0 * P
        fl = dict(E=E, J=J, wJ=wJ, Sf=Sf, isg=isg, P=P)
    if scalar:
        s = 24 + 4 * fluid
        Pi_ = u[s + 1]
        dphi = [d(s, k) for k in range(3)]
        wphi = [gu[i, 0] * dphi[0] + gu[i, 1] * dphi[1] + gu[i, 2] * dphi[2] for i in range(3)]
        dphi2 = chi * (wphi[0] * dphi[0] + wphi[1] * dphi[1] + wphi[2] * dphi[2])
        Pi2 = Pi_ * Pi_
        r_sc = 0.5 * (Pi2 + dphi2)
        rhoH = r_sc if rhoH is None else rhoH + r_sc
        for i in range(3):
            Jl[i] = Pi_ * dphi[i] if Jl[i] is None else Jl[i] + Pi_ * dphi[i]
        half_diff_ichi = 0.5 * (dphi2 - Pi2) * ichi
        for m, (i, j) in enumerate(PAIRS):
            t = dphi[i] * dphi[j] - half_diff_ichi * gt[i, j]
            Sl[m] = t if Sl[m] is None else Sl[m] + t
        t = 1.5 * Pi2 - 0.5 * dphi2
        Str = t if Str is None else Str + t
    have_matter = fluid or scalar

    # ---- right-hand sides ----
    out = [None] * nf
    divb = dbeta(0, 0) + dbeta(1, 1) + dbeta(2, 2)

    def adv(f):
        return beta[0] * d(f, 0) + beta[1] * d(f, 1) + beta[2] * d(f, 2)

    out[CHI] = adv(CHI) + (2.0 / 3.0) * chi * (alpha * K - divb)
    for m, (i, j) in enumerate(PAIRS):
        s = adv(GT + m)
        for k in range(3):
            s = s + gt[i, k] * dbeta(j, k) + gt[j, k] * dbeta(i, k)
        out[GT + m] = s - (2.0 / 3.0) * gt[i, j] * divb - 2.0 * alpha * At[i, j]
    kk = alpha * (AA + (1.0 / 3.0) * K * K)
    if have_matter:
        kk = kk + (4.0 * pi) * alpha * (rhoH + Str)
    out[TRK] = adv(TRK) - lap_a + kk
    X = []
    for m, (i, j) in enumerate(PAIRS):
        r = Ric[i, j] - (8.0 * pi) * Sl[m] if have_matter else Ric[i, j]
        X.append(alpha * r - DDa[m])
    trX = contract_sym(gu2, Sym(X))
    third_trX = (1.0 / 3.0) * trX
    for m, (i, j) in enumerate(PAIRS):
        s = adv(AT + m)
        for k in range(3):
            s = s + At[i, k] * dbeta(j, k) + At[j, k] * dbeta(i, k)
        s = s - (2.0 / 3.0) * At[i, j] * divb
        s = s + chi * (X[m] - gt[i, j] * third_trX)
        AA_ij = At[i, 0] * Aud[0][j] + At[i, 1] * Aud[1][j] + At[i, 2] * Aud[2][j]
        s = s + alpha * (K * At[i, j] - 2.0 * AA_ij)
        out[AT + m] = s
    ddivb = [dd(BET + 0, j, 0) + dd(BET + 1, j, 1) + dd(BET + 2, j, 2) for j in range(3)]  # d_j d_k beta^k
    gu_dK = [gu[i, 0] * dK[0] + gu[i, 1] * dK[1] + gu[i, 2] * dK[2] for i in range(3)]
    Gt_rhs = []
    for i in range(3):
        s = contract_sym(gu2, Sym([dd(BET + i, a, b) for (a, b) in PAIRS]))
        s = s + (1.0 / 3.0) * (gu[i, 0] * ddivb[0] + gu[i, 1] * ddivb[1] + gu[i, 2] * ddivb[2])
        s = s + adv(GAM + i)
        s = s - (Gd[0] * dbeta(0, i) + Gd[1] * dbeta(1, i) + Gd[2] * dbeta(2, i))
        s = s + (2.0 / 3.0) * Gd[i] * divb
        s = s - 2.0 * (Atu[i, 0] * dal[0] + Atu[i, 1] * dal[1] + Atu[i, 2] * dal[2])
        Adchi = Atu[i, 0] * dchi[0] + Atu[i, 1] * dchi[1] + Atu[i, 2] * dchi[2]
        s = s + 2.0 * alpha * (GA[i] - 1.5 * ichi * Adchi - (2.0 / 3.0) * gu_dK[i])
        if have_matter:
            s = s - (16.0 * pi) * alpha * (gu[i, 0] * Jl[0] + gu[i, 1] * Jl[1] + gu[i, 2] * Jl[2])
        Gt_rhs.append(s)
        out[GAM + i] = s
    out[ALP] = adv(ALP) - alpha * (c1 + c2 * alpha) * (K - Kref)
    for i in range(3):
        out[BET + i] = shift_on * (adv(BET + i) + 0.75 * B[i])
        out[BB + i] = shift_on * (adv(BB + i) + (Gt_rhs[i] - adv(GAM + i)) - eta * B[i])
    if fluid:
        q = 24
        E, J, wJ, Sf, isg, P = fl["E"], fl["J"], fl["wJ"], fl["Sf"], fl["isg"], fl["P"]
        chi2 = chi * chi
        # S^i_j = gt^ik S_kj, S^ij = chi^2 S^i_k gt^kj
        Smix = [[gu[i, 0] * Sf[PIDX[(0, j)]] + gu[i, 1] * Sf[PIDX[(1, j)]] + gu[i, 2] * Sf[PIDX[(2, j)]]
                 for j in range(3)] for i in range(3)]
        Su = Sym([chi2 * (Smix[i][0] * gu[0, j] + Smix[i][1] * gu[1, j] + Smix[i][2] * gu[2, j]) for (i, j) in PAIRS])
        Su2 = [Su[i, j] * (1.0 if i == j else 2.0) for (i, j) in PAIRS]
        # K_ij S^ij with K_ij = (At_ij + gt_ij K / 3)/chi
        KS = ichi * (contract_sym(Su2, At) + (1.0 / 3.0) * K * contract_sym(Su2, gt))
        Jda = chi * (wJ[0] * dal[0] + wJ[1] * dal[1] + wJ[2] * dal[2])  # J^j d_j alpha
        out[q] = isg * (alpha * KS - Jda)
        Sgt = contract_sym(Su2, gt)  # S^jk gt_jk
        for i in range(3):
            s = -E * dal[i] + (J[0] * dbeta(i, 0) + J[1] * dbeta(i, 1) + J[2] * dbeta(i, 2))
            Sdg = ichi * contract_sym(Su2, Sym([dgt(i, a, b) for (a, b) in PAIRS])) - ichi * ichi * dchi[i] * Sgt
            s = s + 0.5 * alpha * Sdg
            out[q + 1 + i] = isg * s
    if scalar:
        s = 24 + 4 * fluid
        Pi_ = u[s + 1]
        dPi = [d(s + 1, k) for k in range(3)]
        ddphi = contract_sym(gu2, Sym([dd(s, a, b) for (a, b) in PAIRS]))
        Gd_dphi = Gd[0] * dphi[0] + Gd[1] * dphi[1] + Gd[2] * dphi[2]
        wchi_dphi = wchi[0] * dphi[0] + wchi[1] * dphi[1] + wchi[2] * dphi[2]
        lap_phi = chi * (ddphi - Gd_dphi) - 0.5 * wchi_dphi
        da_dphi = chi * (wphi[0] * dal[0] + wphi[1] * dal[1] + wphi[2] * dal[2])
        out[s] = adv(s) - alpha * Pi_
        out[s + 1] = (beta[0] * dPi[0] + beta[1] * dPi[1] + beta[2] * dPi[2]) + alpha * (K * Pi_ - lap_phi) - da_dphi
    # ---- constraints (diagnostic outputs, same graph) ----
    #  H   = R + 2/3 K^2 - At_ij At^ij - 16 pi rho_H,   R = chi gt^ij R_ij
    #  M^i = gt^ik gt^jl Dt_j At_kl - 3/(2 chi) At^ij d_j chi - 2/3 gt^ij d_j K - 8 pi gt^ij J_j
    Rs = chi * contract_sym(gu2, Ric)
    H = Rs + (2.0 / 3.0) * K * K - AA
    if have_matter:
        H = H - (16.0 * pi) * rhoH
    Y = []
    for k in range(3):
        s = None
        for j in range(3):
            for l in range(3):
                DA = dAt(j, k, l)
                for m in range(3):
                    DA = DA - Gu[m][j, k] * At[m, l] - Gu[m][j, l] * At[k, m]
                t = gu[j, l] * DA
                s = t if s is None else s + t
        Y.append(s)
    M = []
    for i in range(3):
        Adchi = Atu[i, 0] * dchi[0] + Atu[i, 1] * dchi[1] + Atu[i, 2] * dchi[2]
        m_i = (gu[i, 0] * Y[0] + gu[i, 1] * Y[1] + gu[i, 2] * Y[2]) - 1.5 * ichi * Adchi - (2.0 / 3.0) * gu_dK[i]
        if have_matter:
            m_i = m_i - (8.0 * pi) * (gu[i, 0] * Jl[0] + gu[i, 1] * Jl[1] + gu[i, 2] * Jl[2])
        M.append(m_i)
    g.constraints = [H] + M
    return g, L, out

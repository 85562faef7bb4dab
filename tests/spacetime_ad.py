"""Analytic 4D spacetimes + matter, differentiated exactly with torch autodiff.

Test-side machinery that pins the oracle against the mathematics rather than
against a retyped copy of its own formulas.  A smooth 4-metric g_{mu nu}(t, x)
(built from a lapse, a shift and a spatial metric), a perfect fluid (rho, v_i)
and a massless scalar phi are given in closed form.  From them autodiff gives,
at any point:

* the 3+1 data the oracle evolves (BSSN variables, fluid conserved variables,
  scalar field and its momentum) -- these fill the oracle's grid;
* the exact time derivative of every such variable;
* the 4D Ricci / Einstein tensors, div T and box phi.

The identities checked in the tests hold for ANY smooth metric and matter
(they are the 3+1 decomposition itself, with the Einstein and matter equations
appearing only as the residual terms):

  d_t K_ij  = [ADM vacuum RHS]_ij - alpha gamma^mu_i gamma^nu_j 4R_{mu nu}
  H         = R + K^2 - K_ij K^ij - 16 pi rho  = 2 G_{nn} - 16 pi rho      (Gauss)
  M_i(phys) = D_j(K^j_i - delta^j_i K) - 8 pi J_i = -G_{i n} - 8 pi J_i     (Codazzi)
  d_t(sqrt(g) E)   = [conservative RHS] - alpha sqrt(g) n^nu div_mu T^mu_nu
  d_t(sqrt(g) J_i) = [conservative RHS] + alpha sqrt(g) div_mu T^mu_i
  d_t Pi           = [3+1 wave RHS] + alpha box phi

so the oracle's RHS is compared against  exact d_t(variable) + residuals.
Coordinates: t and x in [0, 1)^3; all fields periodic in x with period 1.
"""
from __future__ import annotations

import math

import numpy as np
import torch
from torch.func import jacfwd, vmap

DT = torch.float64
TWO_PI = 2.0 * math.pi
PI = math.pi

# oracle field order
CHI, GT, TRK, AT, GAM, ALP, BET, BB = 0, 1, 7, 8, 14, 17, 18, 21
SYM = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def _modes(rng, n, kmax=2, omega=1.0):
    k = rng.integers(-kmax, kmax + 1, size=(n, 3))
    k[np.all(k == 0, axis=1), 0] = 1
    w = rng.uniform(-omega, omega, size=n)
    ph = rng.uniform(0, 2 * math.pi, size=n)
    return (torch.tensor(k, dtype=DT), torch.tensor(w, dtype=DT), torch.tensor(ph, dtype=DT))


def _wave(modes, amp, X):
    """sum_m amp[m, ...] * sin(2 pi k_m.x + w_m t + ph_m), amp[m] any shape."""
    k, w, ph = modes
    arg = TWO_PI * (k @ X[1:]) + w * X[0] + ph  # (m,)
    s = torch.sin(arg)
    return torch.tensordot(s, amp, dims=([0], [0]))


def det3(m):
    return (m[0, 0] * (m[1, 1] * m[2, 2] - m[1, 2] * m[2, 1]) - m[0, 1] * (m[1, 0] * m[2, 2] - m[1, 2] * m[2, 0])
            + m[0, 2] * (m[1, 0] * m[2, 1] - m[1, 1] * m[2, 0]))


def inv3(m):
    """Inverse by cofactors (elementwise ops only: safe under vmap + jacfwd)."""
    c = torch.stack([
        torch.stack([m[1, 1] * m[2, 2] - m[1, 2] * m[2, 1], m[0, 2] * m[2, 1] - m[0, 1] * m[2, 2],
                     m[0, 1] * m[1, 2] - m[0, 2] * m[1, 1]]),
        torch.stack([m[1, 2] * m[2, 0] - m[1, 0] * m[2, 2], m[0, 0] * m[2, 2] - m[0, 2] * m[2, 0],
                     m[0, 2] * m[1, 0] - m[0, 0] * m[1, 2]]),
        torch.stack([m[1, 0] * m[2, 1] - m[1, 1] * m[2, 0], m[0, 1] * m[2, 0] - m[0, 0] * m[2, 1],
                     m[0, 0] * m[1, 1] - m[0, 1] * m[1, 0]]),
    ])
    return c / det3(m)


class Spacetime:
    """A generic smooth spacetime with fluid and scalar matter (seeded)."""

    def __init__(self, seed=0, eps_g=0.1, eps_k=1.0, eps_a=0.1, eps_b=0.05, rho0=1.0, eps_rho=0.3, eps_v=0.15,
                 eps_phi=0.2, w=1.0 / 3.0, fluid=True, scalar=True, nm=3, monotone_fluid=False):
        rng = np.random.default_rng(seed)
        # monotone fluid: rho = rho0 exp(g.x + c t), v_i = a_i + b_i.x (+ e_i t); no extremum of any
        # primitive anywhere, so the minmod limiter never clips and Kurganov-Tadmor is 2nd order.
        self.monotone_fluid = monotone_fluid
        self.mono_g = torch.tensor(rng.choice([-1, 1], size=3) * rng.uniform(0.3, 0.6, size=3), dtype=DT)
        self.mono_a = torch.tensor(rng.uniform(-0.1, 0.1, size=3), dtype=DT)
        self.mono_b = torch.tensor(rng.choice([-1, 1], size=(3, 3)) * rng.uniform(0.05, 0.1, size=(3, 3)), dtype=DT)
        self.w = w
        self.fluid = fluid
        self.scalar = scalar
        self.mg = _modes(rng, nm, omega=eps_k * 2.0)
        A = rng.uniform(-1, 1, size=(nm, 3, 3))
        self.Ag = torch.tensor(eps_g * 0.5 * (A + A.transpose(0, 2, 1)), dtype=DT)
        self.ma = _modes(rng, 2, omega=1.5)
        self.Aa = torch.tensor(eps_a * rng.uniform(-1, 1, size=2), dtype=DT)
        self.mb = _modes(rng, 3, omega=1.5)
        self.Ab = torch.tensor(eps_b * rng.uniform(-1, 1, size=(3, 3)), dtype=DT)
        self.mB = _modes(rng, 2)
        self.AB = torch.tensor(eps_b * rng.uniform(-1, 1, size=(2, 3)), dtype=DT)
        self.mr = _modes(rng, 2, omega=1.5)
        self.rho0 = rho0
        self.Ar = torch.tensor(eps_rho * rng.uniform(-0.5, 0.5, size=2), dtype=DT)
        self.mv = _modes(rng, 3, omega=1.5)
        self.Av = torch.tensor(eps_v * rng.uniform(-1, 1, size=(3, 3)), dtype=DT)
        self.mp = _modes(rng, 2, omega=2.0)
        self.Ap = torch.tensor(eps_phi * rng.uniform(-1, 1, size=2), dtype=DT)

    # ---- primitive closed forms -------------------------------------------
    def lapse(self, X):
        return 1.0 + _wave(self.ma, self.Aa, X)

    def shift_up(self, X):
        return _wave(self.mb, self.Ab, X)

    def gamma(self, X):
        return torch.eye(3, dtype=DT) + _wave(self.mg, self.Ag, X)

    def Bvec(self, X):
        return _wave(self.mB, self.AB, X)

    def rho(self, X):
        if self.monotone_fluid:
            return self.rho0 * torch.exp(self.mono_g @ X[1:] + 0.2 * X[0])
        return self.rho0 * (1.0 + _wave(self.mr, self.Ar, X))

    def v_low(self, X):
        if self.monotone_fluid:
            return self.mono_a + self.mono_b @ X[1:] + 0.05 * X[0]
        return _wave(self.mv, self.Av, X)

    def phi(self, X):
        return _wave(self.mp, self.Ap, X)

    # ---- 4-metric ------------------------------------------------------------
    def g4(self, X):
        a = self.lapse(X)
        b = self.shift_up(X)
        g = self.gamma(X)
        bl = g @ b
        top = torch.cat([(-a * a + bl @ b).reshape(1), bl])
        rest = torch.cat([bl.reshape(3, 1), g], dim=1)
        return torch.cat([top.reshape(1, 4), rest], dim=0)

    def g4inv(self, X):
        """Inverse 4-metric in 3+1 form: g^tt = -1/a^2, g^ti = b^i/a^2,
        g^ij = gamma^ij - b^i b^j/a^2 (checked against a generic inverse in
        the tests)."""
        a = self.lapse(X)
        b = self.shift_up(X)
        gi = inv3(self.gamma(X))
        a2 = a * a
        top = torch.cat([(-1.0 / a2).reshape(1), b / a2])
        rest = torch.cat([(b / a2).reshape(3, 1), gi - torch.outer(b, b) / a2], dim=1)
        return torch.cat([top.reshape(1, 4), rest], dim=0)

    def chris4(self, X):
        """Gamma^l_{mn}."""
        gi = self.g4inv(X)
        dg = jacfwd(self.g4)(X)  # dg[a, b, c] = d_c g_ab
        # Gamma_{k m n} = 1/2 (d_m g_kn + d_n g_km - d_k g_mn)
        d_m_gkn = dg.permute(0, 2, 1)   # [k, m, n] = d_m g_kn
        d_n_gkm = dg                    # [k, m, n] = d_n g_km
        d_k_gmn = dg.permute(2, 0, 1)   # [k, m, n] = d_k g_mn
        low = 0.5 * (d_m_gkn + d_n_gkm - d_k_gmn)
        return torch.einsum("lk,kmn->lmn", gi, low)

    def ricci4(self, X):
        G = self.chris4(X)
        dG = jacfwd(self.chris4)(X)  # [l, m, n, c] = d_c Gamma^l_mn
        t1 = torch.einsum("lmnl->mn", dG)
        t2 = torch.einsum("lmln->mn", dG)
        t3 = torch.einsum("llk,kmn->mn", G, G)
        t4 = torch.einsum("lnk,kml->mn", G, G)
        return t1 - t2 + t3 - t4

    def einstein4(self, X):
        Rmn = self.ricci4(X)
        gi = self.g4inv(X)
        Rs = torch.einsum("mn,mn->", gi, Rmn)
        return Rmn - 0.5 * self.g4(X) * Rs

    def normal_up(self, X):
        a = self.lapse(X)
        b = self.shift_up(X)
        return torch.cat([(1.0 / a).reshape(1), -b / a])

    def normal_low(self, X):
        a = self.lapse(X)
        return torch.cat([(-a).reshape(1), torch.zeros(3, dtype=DT)])

    # ---- matter ----------------------------------------------------------------
    def T_up(self, X, part="all"):
        T = torch.zeros(4, 4, dtype=DT)
        gi = self.g4inv(X)
        if self.fluid and part in ("all", "fluid"):
            g = self.gamma(X)
            v_l = self.v_low(X)
            v_u = inv3(g) @ v_l
            W = 1.0 / torch.sqrt(1.0 - v_u @ v_l)
            n = self.normal_up(X)
            u = W * (n + torch.cat([torch.zeros(1, dtype=DT), v_u]))
            rho = self.rho(X)
            P = self.w * rho
            T = T + (rho + P) * torch.outer(u, u) + P * gi
        if self.scalar and part in ("all", "scalar"):
            dphi = jacfwd(self.phi)(X)
            dphi_u = gi @ dphi
            T = T + torch.outer(dphi_u, dphi_u) - 0.5 * gi * (dphi @ dphi_u)
        return T

    def T_mixed(self, X, part="all"):
        return self.T_up(X, part) @ self.g4(X)  # T^mu_nu

    def divT(self, X, part="fluid"):
        """(div T)_nu = nabla_mu T^mu_nu."""
        Tm = self.T_mixed(X, part)
        dT = jacfwd(lambda Y: self.T_mixed(Y, part))(X)  # [mu, nu, c]
        G = self.chris4(X)
        return (torch.einsum("mnm->n", dT) + torch.einsum("mml,ln->n", G, Tm) - torch.einsum("lmn,ml->n", G, Tm))

    def box_phi(self, X):
        gi = self.g4inv(X)
        H = jacfwd(jacfwd(self.phi))(X)
        d = jacfwd(self.phi)(X)
        G = self.chris4(X)
        return torch.einsum("mn,mn->", gi, H - torch.einsum("lmn,l->mn", G, d))

    # ---- 3+1 projections -------------------------------------------------------
    def E(self, X, part="all"):
        nl = self.normal_low(X)
        return torch.einsum("m,n,mn->", nl, nl, self.T_up(X, part))

    def J_low(self, X, part="all"):
        a = self.lapse(X)
        return a * self.T_mixed(X, part)[0, 1:]

    def S_low(self, X, part="all"):
        g4 = self.g4(X)
        Tl = g4 @ self.T_up(X, part) @ g4
        return Tl[1:, 1:]

    def sqrtg(self, X):
        return torch.sqrt(det3(self.gamma(X)))

    def K_low(self, X):
        """K_ij = -(d_t gamma_ij - D_i beta_j - D_j beta_i) / (2 alpha)."""
        g = self.gamma(X)
        dg = jacfwd(self.gamma)(X)  # [i, j, c]
        gi = inv3(g)
        b_low = lambda Y: self.gamma(Y) @ self.shift_up(Y)
        bl = b_low(X)
        dbl = jacfwd(b_low)(X)  # [j, c] = d_c beta_j
        ds = dg[:, :, 1:]  # spatial derivatives [i, j, k] = d_k g_ij
        low = 0.5 * (ds.permute(0, 2, 1) + ds - ds.permute(2, 0, 1))  # Gamma_{k i j}
        chr3 = torch.einsum("lk,kij->lij", gi, low)
        Db = dbl[:, 1:].T - torch.einsum("kij,k->ij", chr3, bl)  # D_i beta_j
        return -(dg[:, :, 0] - Db - Db.T) / (2.0 * self.lapse(X))

    def chi(self, X):
        return det3(self.gamma(X)) ** (-1.0 / 3.0)

    def gt_low(self, X):
        return self.chi(X) * self.gamma(X)

    def gt_up(self, X):
        return inv3(self.gt_low(X))

    def Gt_up(self, X):
        d = jacfwd(self.gt_up)(X)  # [i, j, c]
        return -(d[:, 0, 1] + d[:, 1, 2] + d[:, 2, 3])

    def Pi(self, X):
        d = jacfwd(self.phi)(X)
        return -(d[0] - self.shift_up(X) @ d[1:]) / self.lapse(X)

    def state(self, X):
        """All evolved variables in oracle order (fluid, scalar as configured)."""
        chi = self.chi(X)
        g = self.gamma(X)
        gt = chi * g
        K = self.K_low(X)
        trK = torch.einsum("ij,ij->", inv3(g), K)
        At = chi * (K - g * trK / 3.0)
        vals = [chi.reshape(1), torch.stack([gt[i, j] for i, j in SYM]), trK.reshape(1),
                torch.stack([At[i, j] for i, j in SYM]), self.Gt_up(X), self.lapse(X).reshape(1),
                self.shift_up(X), self.Bvec(X)]
        if self.fluid:
            sg = self.sqrtg(X)
            vals += [(sg * self.E(X, "fluid")).reshape(1), sg * self.J_low(X, "fluid")]
        if self.scalar:
            vals += [self.phi(X).reshape(1), self.Pi(X).reshape(1)]
        return torch.cat(vals)

    # ---- exact right-hand sides ---------------------------------------------------
    def expected(self, X, eta, Kref=0.0):
        """Expected RHS of every evolved variable at X (continuum), plus the
        constraints.  Returns dict with 'rhs' (tensor nf) and 'ham', 'mom'."""
        st = self.state(X)
        dst = jacfwd(self.state)(X)  # [f, c]
        d_t = dst[:, 0]
        a = self.lapse(X)
        b = self.shift_up(X)
        g = self.gamma(X)
        gi = inv3(g)
        chi = st[CHI]
        nu = self.normal_up(X)
        G4 = self.einstein4(X)
        R4 = self.ricci4(X)
        Gnn = torch.einsum("m,n,mn->", nu, nu, G4)
        Gin = torch.einsum("mi,m->i", G4[:, 1:], nu)  # gamma^mu_i n^nu G_mu nu (gamma^mu_i = delta for lower i)
        rhoH = self.E(X)
        J = self.J_low(X)
        S = self.S_low(X)
        Str = torch.einsum("ij,ij->", gi, S)
        ham = 2.0 * Gnn - 16.0 * PI * rhoH
        M_phys_low = -Gin - 8.0 * PI * J
        M_conf = (gi @ M_phys_low) / chi
        rhs = d_t.clone()
        # d_t K_ij = ADM-vacuum - alpha 4R_ij ; ADM-with-matter adds -8 pi alpha (S_ij - 1/2 gamma_ij (S - rho))
        # BSSN adds -alpha H gamma_ij / 3 through its K equation.
        Kl = self.K_low(X)
        dK = jacfwd(self.K_low)(X)[:, :, 0]
        Kdot_expected = dK + a * R4[1:, 1:] - 8.0 * PI * a * (S - 0.5 * g * (Str - rhoH)) - a * ham * g / 3.0
        # Gamma-tilde: exact kinematic rate + 2 alpha M^i_conf
        rhs[GAM:GAM + 3] = d_t[GAM:GAM + 3] + 2.0 * a * M_conf
        # gauge (definitions): 1+log slicing with K_ref, Gamma-driver shift
        dXs = dst[:, 1:]  # spatial derivatives [f, k]
        rhs[ALP] = b @ dXs[ALP] - 2.0 * a * (st[TRK] - Kref)
        rhs[BET:BET + 3] = dXs[BET:BET + 3] @ b + 0.75 * st[BB:BB + 3]
        rhs[BB:BB + 3] = dXs[BB:BB + 3] @ b + (rhs[GAM:GAM + 3] - dXs[GAM:GAM + 3] @ b) - eta * st[BB:BB + 3]
        off = 24
        if self.fluid:
            sg = self.sqrtg(X)
            dv = self.divT(X, "fluid")
            rhs[off] = d_t[off] + a * sg * (nu @ dv)
            rhs[off + 1:off + 4] = d_t[off + 1:off + 4] - a * sg * dv[1:]
            off += 4
        if self.scalar:
            rhs[off + 1] = d_t[off + 1] - a * self.box_phi(X)
        return dict(rhs=rhs, Kdot=Kdot_expected, gdot=jacfwd(self.gamma)(X)[:, :, 0], ham=ham, mom=M_conf,
                    state=st, K=Kl)


def implied_adm_rates(st, rhs):
    """Map BSSN values+rates (numpy, oracle order, one point) to (d_t gamma_ij, d_t K_ij)."""
    chi, dchi = st[CHI], rhs[CHI]
    gt = np.zeros((3, 3))
    dgt = np.zeros((3, 3))
    At = np.zeros((3, 3))
    dAt = np.zeros((3, 3))
    for m, (i, j) in enumerate(SYM):
        gt[i, j] = gt[j, i] = st[GT + m]
        dgt[i, j] = dgt[j, i] = rhs[GT + m]
        At[i, j] = At[j, i] = st[AT + m]
        dAt[i, j] = dAt[j, i] = rhs[AT + m]
    K, dK = st[TRK], rhs[TRK]
    gdot = dgt / chi - gt * dchi / chi ** 2
    Kij = (At + gt * K / 3.0) / chi
    Kdot = (dAt + dgt * K / 3.0 + gt * dK / 3.0) / chi - Kij * dchi / chi
    return gdot, Kdot


def sample_state(st: Spacetime, X: torch.Tensor):
    """Evaluate the oracle state at many points X[m] = (t, x, y, z)."""
    return vmap(st.state)(X)

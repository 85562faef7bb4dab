/*
 * COSMOS evolution oracle — plain, slow, obviously-correct FP64 CPU code.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference leg of bench.py may load this library.  The product
 * library (paper_2606_02053_gb300) never links, loads or calls it, and the two
 * share no source, header, table or constant.
 *
 * What it computes (paper: Yoo et al., "COSMOS: a numerical relativity code
 * specialized for PBH formation", section "Physical system settings"):
 *   - Einstein equations G_{mu nu} = 8 pi T_{mu nu} (G = c = 1), with
 *     T = T^SC + T^FL, T^SC = d phi d phi - 1/2 g (d phi)^2,
 *     T^FL = (rho + P) u u + P g, P = w rho, box phi = 0, div T^FL = 0;
 *   - cast (the paper leaves this to standard numerical-relativity texts)
 *     into the BSSN (chi-variant) 3+1 form, 4th-order centred finite differences,
 *     6th-derivative Kreiss-Oliger dissipation and classic RK4;
 *   - the fluid advanced with the Kurganov-Tadmor central scheme in a
 *     conservative (Shibata-Font lineage) 3+1 form;
 *   - long-wavelength initial data: conformal factor from the curvature
 *     perturbation zeta, the fluid density fixed so that the (discrete)
 *     Hamiltonian constraint holds (section "Physical system settings", last
 *     paragraph).
 * The paper does not print these formulas; each reading taken where it is
 * silent is stated beside the code that takes it.
 *
 * Style: full 3x3 index arrays and explicit loops over the summed indices, in
 * the textbook notation; no blocking, no fusion, no reuse beyond named
 * intermediates.  Compiled with -O2 -ffp-contract=off (no FMA contraction).
 * Arithmetic is templated on the scalar type R only so that the very same
 * code can be run with a counting type to obtain the algorithmic flop count.
 *
 * State layout: state[f][k][j][i], i fastest, no padding, n = nx*ny*nz points
 * per field.  Field order: chi, gt_xx, gt_xy, gt_xz, gt_yy, gt_yz, gt_zz, K,
 * At_xx..At_zz, Gt^x, Gt^y, Gt^z, alpha, beta^x,y,z, B^x,y,z  (24), then, if
 * the fluid is on, tau~ = sqrt(gamma) E and S~_i = sqrt(gamma) J_i (4), then,
 * if the scalar is on, phi and Pi (2).
 */
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>
#include <type_traits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

/* ------------------------------------------------------------------------ */
/* Counting scalar: every +, -, *, / and sqrt is tallied.                    */
/* ------------------------------------------------------------------------ */
struct Tally { double add, mul, div, sqrt, cmp; };
Tally g_tally;  // only touched single-threaded (flop counting runs on one point)

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { g_tally.add += 1; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_tally.add += 1; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_tally.mul += 1; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_tally.div += 1; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt sqrt(Cnt a) { g_tally.sqrt += 1; return Cnt(std::sqrt(a.v)); }
inline Cnt fabs(Cnt a) { return Cnt(std::fabs(a.v)); }
inline bool operator<(Cnt a, Cnt b) { g_tally.cmp += 1; return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { g_tally.cmp += 1; return a.v > b.v; }
inline double val(Cnt a) { return a.v; }
inline double val(double a) { return a; }
using std::sqrt;
using std::fabs;
using std::exp;

/* ------------------------------------------------------------------------ */
/* Taped scalar for reverse mode: every operation appends a node holding its */
/* (at most two) parents and the partial derivatives with respect to them.   */
/* Leaves 0 .. nleaves-1 are the state entries; id -1 marks a constant.      */
/* ------------------------------------------------------------------------ */
struct TapeNode { long a, b; double da, db; };
std::vector<TapeNode> g_tape;  // only touched single-threaded (tiny grids)

struct AD {
  double v;
  long id;
  AD() : v(0), id(-1) {}
  AD(double x) : v(x), id(-1) {}
  AD(double x, long i) : v(x), id(i) {}
};
inline AD node(double v, long a, double da, long b = -1, double db = 0.0) {
  if (a < 0 && b < 0) return AD(v);
  g_tape.push_back(TapeNode{a, b, da, db});
  return AD(v, (long)g_tape.size() - 1);
}
inline AD operator+(AD x, AD y) { return node(x.v + y.v, x.id, 1.0, y.id, 1.0); }
inline AD operator-(AD x, AD y) { return node(x.v - y.v, x.id, 1.0, y.id, -1.0); }
inline AD operator*(AD x, AD y) { return node(x.v * y.v, x.id, y.v, y.id, x.v); }
inline AD operator/(AD x, AD y) { return node(x.v / y.v, x.id, 1.0 / y.v, y.id, -x.v / (y.v * y.v)); }
inline AD operator-(AD x) { return node(-x.v, x.id, -1.0); }
inline AD sqrt(AD x) {
  double r = std::sqrt(x.v);
  return node(r, x.id, 0.5 / r);
}
inline AD fabs(AD x) { return node(std::fabs(x.v), x.id, x.v < 0.0 ? -1.0 : 1.0); }
inline AD exp(AD x) {
  double e = std::exp(x.v);
  return node(e, x.id, e);
}
inline double val(AD a) { return a.v; }
inline long tape_id(double) { return -1; }
inline long tape_id(AD a) { return a.id; }

/* Adjoints of the first nleaves tape entries after one reverse sweep from the
 * given (node id, cotangent) seeds. */
std::vector<double> reverse_sweep(long nleaves, const std::vector<std::pair<long, double>>& seeds) {
  std::vector<double> adj(g_tape.size(), 0.0);
  for (auto& sd : seeds) adj[sd.first] += sd.second;
  for (long q = (long)g_tape.size() - 1; q >= nleaves; --q) {
    const double a = adj[q];
    if (a == 0.0) continue;
    const TapeNode& nd = g_tape[q];
    if (nd.a >= 0) adj[nd.a] += a * nd.da;
    if (nd.b >= 0) adj[nd.b] += a * nd.db;
  }
  adj.resize(nleaves);
  return adj;
}
inline bool operator<(AD x, AD y) { return x.v < y.v; }
inline bool operator>(AD x, AD y) { return x.v > y.v; }

template <class R> struct is_ad { static constexpr bool value = false; };
template <> struct is_ad<AD> { static constexpr bool value = true; };

template <class R> inline R rmax(R a, R b) { return (a < b) ? b : a; }
template <class R> inline R rmin(R a, R b) { return (b < a) ? b : a; }

constexpr double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Field indices                                                             */
/* ------------------------------------------------------------------------ */
enum {
  CHI = 0, GT = 1 /* 6 */, TRK = 7, AT = 8 /* 6 */, GAM = 14 /* 3 */,
  ALP = 17, BET = 18 /* 3 */, BB = 21 /* 3 */, NBSSN = 24
};
constexpr int NFMAX = 30;
// symmetric pair (i,j) -> 0..5 in the order xx, xy, xz, yy, yz, zz
inline int sym(int i, int j) {
  static const int m[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return m[i][j];
}

struct Params {
  int slicing;    // 0 = 1+log, 1 = harmonic
  int shift;      // 0 = frozen, 1 = Gamma-driver
  double eta;     // Gamma-driver damping
  double sigma;   // Kreiss-Oliger strength
  double w;       // P = w rho
  int fluid;      // 1 = perfect fluid on
  int scalar;     // 1 = massless scalar on
  double H0;      // background Hubble rate at t0 (0 = no background)
  double t0;
  int nf() const { return NBSSN + 4 * fluid + 2 * scalar; }
  int ifl() const { return NBSSN; }
  int isc() const { return NBSSN + 4 * fluid; }
};

Params unpack_params(const double* p) {
  Params q;
  q.slicing = (int)p[0];
  q.shift = (int)p[1];
  q.eta = p[2];
  q.sigma = p[3];
  q.w = p[4];
  q.fluid = (int)p[5];
  q.scalar = (int)p[6];
  q.H0 = p[7];
  q.t0 = p[8];
  return q;
}

constexpr long WRAP_PAD = 8;  // largest stencil reach used anywhere is 4

struct Grid {
  long n[3];
  double h[3];
  double x0[3];
  // periodic index tables: wrap[d][i + WRAP_PAD] = i mod n[d]
  std::vector<long> wrap[3];
  long npts() const { return n[0] * n[1] * n[2]; }
};

Grid make_grid(const int* n, const double* h, const double* x0) {
  Grid g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = n[d];
    g.h[d] = h[d];
    g.x0[d] = x0[d];
    g.wrap[d].resize(n[d] + 2 * WRAP_PAD);
    for (long i = 0; i < n[d] + 2 * WRAP_PAD; ++i) {
      long a = (i - WRAP_PAD) % n[d];
      g.wrap[d][i] = a < 0 ? a + n[d] : a;
    }
  }
  return g;
}

/* Background reference trace K_ref(t) = -3 H_b(t), H_b the Hubble rate of a
 * flat FLRW universe filled with the P = w rho fluid (Friedmann equations);
 * zero when no background is set. */
double K_ref(const Params& P, double t) {
  if (P.H0 == 0.0) return 0.0;
  double Hb = P.H0 / (1.0 + 1.5 * (1.0 + P.w) * P.H0 * (t - P.t0));
  return -3.0 * Hb;
}

/* ------------------------------------------------------------------------ */
/* Periodic grid access                                                      */
/* ------------------------------------------------------------------------ */
struct Pt { long i[3]; };

inline long wrapi(long a, long n) {
  a %= n;
  return a < 0 ? a + n : a;
}

struct Field {
  const Grid* g;
  const double* s;
  // reverse mode only: tape id of every entry (-1 = constant); when null the
  // entries themselves are the tape's leaves (id = their index)
  const long* ids = nullptr;
  long wrapped(int d, long a) const {
    long m = a + WRAP_PAD;
    if (m >= 0 && m < (long)g->wrap[d].size()) return g->wrap[d][m];
    return wrapi(a, g->n[d]);
  }
  long index(int f, Pt p) const {
    long i = wrapped(0, p.i[0]), j = wrapped(1, p.i[1]), k = wrapped(2, p.i[2]);
    return (long)f * g->npts() + (k * g->n[1] + j) * g->n[0] + i;
  }
  double at(int f, Pt p) const { return s[index(f, p)]; }
};

/* A state entry as a value of the scalar type (a tape leaf for reverse mode). */
template <class R> inline R load(const Field& F, int f, Pt p) { return R(F.at(f, p)); }
template <> inline AD load<AD>(const Field& F, int f, Pt p) {
  const long q = F.index(f, p);
  return AD(F.s[q], F.ids ? F.ids[q] : q);
}

inline Pt shift(Pt p, int d, long o) {
  p.i[d] += o;
  return p;
}

/* ------------------------------------------------------------------------ */
/* Finite-difference operators (4th-order centred, periodic)                 */
/*   D_d f   = [8 (f+1 - f-1) - (f+2 - f-2)] / (12 h)                       */
/*   D_dd f  = [16 ((f+1 - f0) + (f-1 - f0)) - ((f+2 - f0) + (f-2 - f0))]/(12 h^2)
 *   D_ab f  = D_a (D_b f)      (a != b, the 16-point product stencil)        */
/*   KO f    = sigma/64 sum_d (1/h_d) [ (f+3 - f0) + (f-3 - f0)              */
/*             - 6 ((f+2 - f0) + (f-2 - f0)) + 15 ((f+1 - f0) + (f-1 - f0)) ] */
/* Each stencil is written with neighbour differences first: these are exact */
/* for a smooth field (Sterbenz), so the result carries only the rounding of */
/* the small quantities that follow.  The values are identical, as real     */
/* numbers, to the textbook coefficient sums.                                */
/* ------------------------------------------------------------------------ */
template <class R>
R D1(const Field& F, int f, Pt p, int d) {
  R a = load<R>(F, f, shift(p, d, 1)) - load<R>(F, f, shift(p, d, -1));
  R b = load<R>(F, f, shift(p, d, 2)) - load<R>(F, f, shift(p, d, -2));
  return (R(8.0) * a - b) / R(12.0 * F.g->h[d]);
}

template <class R>
R D2(const Field& F, int f, Pt p, int d) {
  R f0 = load<R>(F, f, p);
  R s1 = (load<R>(F, f, shift(p, d, 1)) - f0) + (load<R>(F, f, shift(p, d, -1)) - f0);
  R s2 = (load<R>(F, f, shift(p, d, 2)) - f0) + (load<R>(F, f, shift(p, d, -2)) - f0);
  return (R(16.0) * s1 - s2) / R(12.0 * F.g->h[d] * F.g->h[d]);
}

/* Mixed derivative D_a(D_b f).  The inner first derivatives at the four
 * neighbours along a are the same numbers that those neighbours compute for
 * themselves, so they are evaluated in plain double and enter R as data: the
 * flop tally then charges one D_a stencil per mixed derivative, which is what
 * a grid-wide evaluation that stores first derivatives costs. */
template <class R>
R Dmix(const Field& F, int f, Pt p, int a, int b) {
  if constexpr (is_ad<R>::value) {  // reverse mode: the neighbours' derivatives are taped too
    R m1 = D1<R>(F, f, shift(p, a, 1), b) - D1<R>(F, f, shift(p, a, -1), b);
    R m2 = D1<R>(F, f, shift(p, a, 2), b) - D1<R>(F, f, shift(p, a, -2), b);
    return (R(8.0) * m1 - m2) / R(12.0 * F.g->h[a]);
  } else {
    R m1 = R(D1<double>(F, f, shift(p, a, 1), b)) - R(D1<double>(F, f, shift(p, a, -1), b));
    R m2 = R(D1<double>(F, f, shift(p, a, 2), b)) - R(D1<double>(F, f, shift(p, a, -2), b));
    return (R(8.0) * m1 - m2) / R(12.0 * F.g->h[a]);
  }
}

template <class R>
R KO(const Field& F, int f, Pt p, double sigma) {
  R f0 = load<R>(F, f, p);
  R sum = R(0.0);
  for (int d = 0; d < 3; ++d) {
    R s1 = (load<R>(F, f, shift(p, d, 1)) - f0) + (load<R>(F, f, shift(p, d, -1)) - f0);
    R s2 = (load<R>(F, f, shift(p, d, 2)) - f0) + (load<R>(F, f, shift(p, d, -2)) - f0);
    R s3 = (load<R>(F, f, shift(p, d, 3)) - f0) + (load<R>(F, f, shift(p, d, -3)) - f0);
    R sd = (s3 - R(6.0) * s2) + R(15.0) * s1;
    sum = sum + sd / R(F.g->h[d]);
  }
  return R(sigma / 64.0) * sum;
}

/* ------------------------------------------------------------------------ */
/* Small tensor helpers                                                      */
/* ------------------------------------------------------------------------ */
/* Inverse of a symmetric 3x3 matrix by cofactors: inv = adj(m) / det(m).
 * Only the six independent cofactors are formed; the result is symmetric. */
template <class R>
void inverse_sym3(const R m[3][3], R inv[3][3], R* det_out) {
  R c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
  R c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
  R c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
  R c11 = m[0][0] * m[2][2] - m[0][2] * m[2][0];
  R c12 = m[0][1] * m[2][0] - m[0][0] * m[2][1];
  R c22 = m[0][0] * m[1][1] - m[0][1] * m[1][0];
  R det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
  inv[0][0] = c00 / det;
  inv[0][1] = inv[1][0] = c01 / det;
  inv[0][2] = inv[2][0] = c02 / det;
  inv[1][1] = c11 / det;
  inv[1][2] = inv[2][1] = c12 / det;
  inv[2][2] = c22 / det;
  if (det_out) *det_out = det;
}

/* ------------------------------------------------------------------------ */
/* Everything the pointwise algebra needs at one grid point                  */
/* ------------------------------------------------------------------------ */
template <class R>
struct Local {
  // values
  R chi, gt[3][3], K, At[3][3], Gt[3], alpha, beta[3], B[3];
  // first derivatives: d?[k] = d_k ?, dgt[k][i][j] = d_k gt_ij, dbeta[k][i] = d_k beta^i
  R dchi[3], dgt[3][3][3], dK[3], dAt[3][3][3], dGt[3][3], dalpha[3], dbeta[3][3], dB[3][3];
  // second derivatives: dd?[k][l] = d_k d_l ?
  R ddchi[3][3], ddgt[3][3][3][3], ddalpha[3][3], ddbeta[3][3][3];
  // scalar field
  R phi, Pi, dphi[3], dPi[3], ddphi[3][3];
  // fluid conserved variables at the point
  R tau, St[3];
};

template <class R>
void grad(const Field& F, int f, Pt p, R out[3]) {
  for (int k = 0; k < 3; ++k) out[k] = D1<R>(F, f, p, k);
}

template <class R>
void hess(const Field& F, int f, Pt p, R out[3][3]) {
  for (int k = 0; k < 3; ++k) out[k][k] = D2<R>(F, f, p, k);
  for (int k = 0; k < 3; ++k)
    for (int l = k + 1; l < 3; ++l) out[k][l] = out[l][k] = Dmix<R>(F, f, p, k, l);
}

template <class R>
void gather(const Field& F, const Params& P, Pt p, Local<R>& L) {
  L.chi = load<R>(F, CHI, p);
  L.K = load<R>(F, TRK, p);
  L.alpha = load<R>(F, ALP, p);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      L.gt[i][j] = load<R>(F, GT + sym(i, j), p);
      L.At[i][j] = load<R>(F, AT + sym(i, j), p);
    }
  for (int i = 0; i < 3; ++i) {
    L.Gt[i] = load<R>(F, GAM + i, p);
    L.beta[i] = load<R>(F, BET + i, p);
    L.B[i] = load<R>(F, BB + i, p);
  }
  grad<R>(F, CHI, p, L.dchi);
  grad<R>(F, TRK, p, L.dK);
  grad<R>(F, ALP, p, L.dalpha);
  hess<R>(F, CHI, p, L.ddchi);
  hess<R>(F, ALP, p, L.ddalpha);
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      R g[3], a[3], hh[3][3];
      grad<R>(F, GT + sym(i, j), p, g);
      grad<R>(F, AT + sym(i, j), p, a);
      hess<R>(F, GT + sym(i, j), p, hh);
      for (int k = 0; k < 3; ++k) {
        L.dgt[k][i][j] = L.dgt[k][j][i] = g[k];
        L.dAt[k][i][j] = L.dAt[k][j][i] = a[k];
        for (int l = 0; l < 3; ++l) L.ddgt[k][l][i][j] = L.ddgt[k][l][j][i] = hh[k][l];
      }
    }
  for (int i = 0; i < 3; ++i) {
    R g[3], b[3], bb[3], hh[3][3];
    grad<R>(F, GAM + i, p, g);
    grad<R>(F, BET + i, p, b);
    grad<R>(F, BB + i, p, bb);
    hess<R>(F, BET + i, p, hh);
    for (int k = 0; k < 3; ++k) {
      L.dGt[k][i] = g[k];
      L.dbeta[k][i] = b[k];
      L.dB[k][i] = bb[k];
      for (int l = 0; l < 3; ++l) L.ddbeta[k][l][i] = hh[k][l];
    }
  }
  if (P.scalar) {
    int s = P.isc();
    L.phi = load<R>(F, s, p);
    L.Pi = load<R>(F, s + 1, p);
    grad<R>(F, s, p, L.dphi);
    grad<R>(F, s + 1, p, L.dPi);
    hess<R>(F, s, p, L.ddphi);
  }
  if (P.fluid) {
    int q = P.ifl();
    L.tau = load<R>(F, q, p);
    for (int i = 0; i < 3; ++i) L.St[i] = load<R>(F, q + 1 + i, p);
  }
}

/* ------------------------------------------------------------------------ */
/* Matter: the 3+1 projections of T^FL and T^SC (section "Physical system    */
/* settings"): rho_H = n n T, J_i = -n gamma_i T, S_ij = gamma gamma T.      */
/* ------------------------------------------------------------------------ */
template <class R>
struct Matter {
  R rho, J[3], S[3][3], Str;        // total sources for the BSSN equations
  // fluid-only pieces (the fluid's own equations use only its own stress)
  R E, Jf[3], Sf[3][3], rho0, P;
};

/* Fluid primitive recovery from E = rho_H and J_i for P = w rho (w > 0).
 * With h W^2 = (1+w) rho W^2:  E = h W^2 - w rho,  J_i = h W^2 v_i,
 * J^2 = (E + w rho)(E - rho), i.e. w rho^2 + (1-w) E rho + (J^2 - E^2) = 0;
 * rho is the positive root. */
template <class R>
R fluid_rho(R E, R J2, double w) {
  R a = R(1.0 - w) * E;
  return (sqrt(a * a + R(4.0 * w) * (E * E - J2)) - a) / R(2.0 * w);
}

template <class R>
void matter_sources(const Local<R>& L, const Params& P, const R gtu[3][3], Matter<R>& M) {
  M.rho = R(0.0);
  M.Str = R(0.0);
  for (int i = 0; i < 3; ++i) {
    M.J[i] = R(0.0);
    for (int j = 0; j < 3; ++j) M.S[i][j] = R(0.0);
  }
  R gu[3][3];  // physical inverse metric gamma^ij = chi gt^ij
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) gu[i][j] = gu[j][i] = L.chi * gtu[i][j];
  R gdn[3][3];  // physical metric gamma_ij = gt_ij / chi
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) gdn[i][j] = gdn[j][i] = L.gt[i][j] / L.chi;
  if (P.fluid) {
    R chi32 = L.chi * sqrt(L.chi);  // 1/sqrt(gamma) = chi^{3/2}
    M.E = L.tau * chi32;
    for (int i = 0; i < 3; ++i) M.Jf[i] = L.St[i] * chi32;
    R J2 = R(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) J2 = J2 + gu[i][j] * M.Jf[i] * M.Jf[j];
    M.rho0 = fluid_rho<R>(M.E, J2, P.w);
    M.P = R(P.w) * M.rho0;
    R EP = M.E + M.P;
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) M.Sf[i][j] = M.Sf[j][i] = M.Jf[i] * M.Jf[j] / EP + M.P * gdn[i][j];
    M.rho = M.rho + M.E;
    for (int i = 0; i < 3; ++i) M.J[i] = M.J[i] + M.Jf[i];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) M.S[i][j] = M.S[j][i] = M.S[i][j] + M.Sf[i][j];
    M.Str = M.Str + J2 / EP + R(3.0) * M.P;
  }
  if (P.scalar) {
    R dphi2 = R(0.0);  // |D phi|^2 = gamma^ij d_i phi d_j phi
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) dphi2 = dphi2 + gu[i][j] * L.dphi[i] * L.dphi[j];
    R Pi2 = L.Pi * L.Pi;
    M.rho = M.rho + R(0.5) * Pi2 + R(0.5) * dphi2;
    for (int i = 0; i < 3; ++i) M.J[i] = M.J[i] + L.Pi * L.dphi[i];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j)
        M.S[i][j] = M.S[j][i] = M.S[i][j] + L.dphi[i] * L.dphi[j] - R(0.5) * gdn[i][j] * (dphi2 - Pi2);
    M.Str = M.Str + R(1.5) * Pi2 - R(0.5) * dphi2;
  }
}

/* ------------------------------------------------------------------------ */
/* Conformal geometry at a point: inverse metric, Christoffels, Ricci        */
/* ------------------------------------------------------------------------ */
template <class R>
struct Geom {
  R gtu[3][3];
  R Gl[3][3][3];   // Gt_kij = 1/2 (d_i gt_kj + d_j gt_ki - d_k gt_ij)   (first index lowered)
  R Gu[3][3][3];   // Gt^k_ij = gt^kl Gt_lij
  R Gd[3];         // Gt^k_d = gt^ij Gt^k_ij
  R Ric[3][3];     // R_ij = Rt_ij + Rchi_ij
  R Rs;            // R = chi gt^ij R_ij
  R Atu[3][3];     // At^ij
  R Aud[3][3];     // At^i_j = gt^ik At_kj
  R AA;            // At_ij At^ij
};

template <class R>
void geometry(const Local<R>& L, Geom<R>& G) {
  inverse_sym3<R>(L.gt, G.gtu, nullptr);
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j)
        G.Gl[k][i][j] = G.Gl[k][j][i] = R(0.5) * (L.dgt[i][k][j] + L.dgt[j][k][i] - L.dgt[k][i][j]);
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) {
        R s = R(0.0);
        for (int l = 0; l < 3; ++l) s = s + G.gtu[k][l] * G.Gl[l][i][j];
        G.Gu[k][i][j] = G.Gu[k][j][i] = s;
      }
  for (int k = 0; k < 3; ++k) {
    R s = R(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) s = s + G.gtu[i][j] * G.Gu[k][i][j];
    G.Gd[k] = s;
  }
  /* Conformal Ricci tensor (textbook BSSN form):
   * Rt_ij = -1/2 gt^lm d_l d_m gt_ij + gt_k(i d_j) Gt^k + Gt^k_d Gt_(ij)k
   *        + gt^lm (Gt^k_li Gt_jkm + Gt^k_lj Gt_ikm + Gt^k_im Gt_klj)
   * with the evolved Gt^k under the derivative and Gt^k_d elsewhere. */
  R Rt[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      R t1 = R(0.0);
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) t1 = t1 + G.gtu[l][m] * L.ddgt[l][m][i][j];
      R t2 = R(0.0);
      for (int k = 0; k < 3; ++k) t2 = t2 + L.gt[k][i] * L.dGt[j][k] + L.gt[k][j] * L.dGt[i][k];
      R t3 = R(0.0);
      for (int k = 0; k < 3; ++k) t3 = t3 + G.Gd[k] * (G.Gl[i][j][k] + G.Gl[j][i][k]);
      R t4 = R(0.0);
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          R s = R(0.0);
          for (int k = 0; k < 3; ++k)
            s = s + G.Gu[k][l][i] * G.Gl[j][k][m] + G.Gu[k][l][j] * G.Gl[i][k][m] + G.Gu[k][i][m] * G.Gl[k][l][j];
          t4 = t4 + G.gtu[l][m] * s;
        }
      Rt[i][j] = Rt[j][i] = R(-0.5) * t1 + R(0.5) * t2 + R(0.5) * t3 + t4;
    }
  /* Ricci part from the conformal factor chi (chi = exp(-4 phi) form):
   * Rchi_ij = (Dt_i Dt_j chi + gt_ij gt^lm Dt_l Dt_m chi)/(2 chi)
   *          - d_i chi d_j chi/(4 chi^2) - 3 gt_ij gt^lm d_l chi d_m chi/(4 chi^2) */
  R DDchi[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      R s = L.ddchi[i][j];
      for (int k = 0; k < 3; ++k) s = s - G.Gu[k][i][j] * L.dchi[k];
      DDchi[i][j] = DDchi[j][i] = s;
    }
  R trDD = R(0.0), dchi2 = R(0.0);
  for (int l = 0; l < 3; ++l)
    for (int m = 0; m < 3; ++m) {
      trDD = trDD + G.gtu[l][m] * DDchi[l][m];
      dchi2 = dchi2 + G.gtu[l][m] * L.dchi[l] * L.dchi[m];
    }
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      R Rc = (DDchi[i][j] + L.gt[i][j] * trDD) / (R(2.0) * L.chi) - L.dchi[i] * L.dchi[j] / (R(4.0) * L.chi * L.chi) -
             R(3.0) * L.gt[i][j] * dchi2 / (R(4.0) * L.chi * L.chi);
      G.Ric[i][j] = G.Ric[j][i] = Rt[i][j] + Rc;
    }
  R trR = R(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trR = trR + G.gtu[i][j] * G.Ric[i][j];
  G.Rs = L.chi * trR;
  // At with raised indices
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      R s = R(0.0);
      for (int k = 0; k < 3; ++k) s = s + G.gtu[i][k] * L.At[k][j];
      G.Aud[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      R s = R(0.0);
      for (int k = 0; k < 3; ++k) s = s + G.Aud[i][k] * G.gtu[k][j];
      G.Atu[i][j] = G.Atu[j][i] = s;
    }
  R aa = R(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) aa = aa + L.At[i][j] * G.Atu[i][j];
  G.AA = aa;
}

/* ------------------------------------------------------------------------ */
/* BSSN right-hand side at one point (vacuum part + matter sources + gauge)  */
/* Output order = state field order; fluid entries get only their geometric  */
/* source here (the flux divergence is added by the caller).                 */
/* ------------------------------------------------------------------------ */
template <class R>
void point_algebra(const Local<R>& L, const Params& P, double t, R* out) {
  Geom<R> G;
  geometry<R>(L, G);
  Matter<R> M;
  matter_sources<R>(L, P, G.gtu, M);
  const R chi = L.chi, alpha = L.alpha, K = L.K;
  const R pi4 = R(4.0 * PI), pi8 = R(8.0 * PI), pi16 = R(16.0 * PI);

  R divb = L.dbeta[0][0] + L.dbeta[1][1] + L.dbeta[2][2];
  // second covariant derivative of the lapse (physical metric)
  R dchi_dalpha = R(0.0);
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) dchi_dalpha = dchi_dalpha + G.gtu[k][l] * L.dchi[k] * L.dalpha[l];
  R DDa[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      R s = L.ddalpha[i][j];
      for (int k = 0; k < 3; ++k) s = s - G.Gu[k][i][j] * L.dalpha[k];
      s = s + (L.dchi[i] * L.dalpha[j] + L.dchi[j] * L.dalpha[i] - L.gt[i][j] * dchi_dalpha) / (R(2.0) * chi);
      DDa[i][j] = DDa[j][i] = s;
    }
  R lap_a = R(0.0);
  {
    R a1 = R(0.0), a2 = R(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) a1 = a1 + G.gtu[i][j] * L.ddalpha[i][j];
    for (int k = 0; k < 3; ++k) a2 = a2 + G.Gd[k] * L.dalpha[k];
    lap_a = chi * a1 - chi * a2 - R(0.5) * dchi_dalpha;
  }

  // chi
  {
    R adv = R(0.0);
    for (int k = 0; k < 3; ++k) adv = adv + L.beta[k] * L.dchi[k];
    out[CHI] = adv + R(2.0 / 3.0) * chi * (alpha * K - divb);
  }
  // conformal metric
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      R s = R(0.0);
      for (int k = 0; k < 3; ++k) s = s + L.beta[k] * L.dgt[k][i][j];
      for (int k = 0; k < 3; ++k) s = s + L.gt[i][k] * L.dbeta[j][k] + L.gt[j][k] * L.dbeta[i][k];
      s = s - R(2.0 / 3.0) * L.gt[i][j] * divb - R(2.0) * alpha * L.At[i][j];
      out[GT + sym(i, j)] = s;
    }
  // trace of the extrinsic curvature
  {
    R adv = R(0.0);
    for (int k = 0; k < 3; ++k) adv = adv + L.beta[k] * L.dK[k];
    out[TRK] = adv - lap_a + alpha * (G.AA + K * K / R(3.0)) + pi4 * alpha * (M.rho + M.Str);
  }
  // trace-free conformal extrinsic curvature
  {
    R X[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) X[i][j] = X[j][i] = -DDa[i][j] + alpha * (G.Ric[i][j] - pi8 * M.S[i][j]);
    R trX = R(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) trX = trX + G.gtu[i][j] * X[i][j];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) {
        R s = R(0.0);
        for (int k = 0; k < 3; ++k) s = s + L.beta[k] * L.dAt[k][i][j];
        for (int k = 0; k < 3; ++k) s = s + L.At[i][k] * L.dbeta[j][k] + L.At[j][k] * L.dbeta[i][k];
        s = s - R(2.0 / 3.0) * L.At[i][j] * divb;
        s = s + chi * (X[i][j] - L.gt[i][j] * trX / R(3.0));
        R AA_ij = R(0.0);
        for (int k = 0; k < 3; ++k) AA_ij = AA_ij + L.At[i][k] * G.Aud[k][j];
        s = s + alpha * (K * L.At[i][j] - R(2.0) * AA_ij);
        out[AT + sym(i, j)] = s;
      }
  }
  // conformal connection functions
  R Gt_rhs[3];
  for (int i = 0; i < 3; ++i) {
    R s = R(0.0);
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s = s + G.gtu[j][k] * L.ddbeta[j][k][i];
    R t = R(0.0);
    for (int j = 0; j < 3; ++j) {
      R dd = R(0.0);
      for (int k = 0; k < 3; ++k) dd = dd + L.ddbeta[j][k][k];
      t = t + G.gtu[i][j] * dd;
    }
    s = s + t / R(3.0);
    for (int j = 0; j < 3; ++j) s = s + L.beta[j] * L.dGt[j][i];
    for (int j = 0; j < 3; ++j) s = s - G.Gd[j] * L.dbeta[j][i];
    s = s + R(2.0 / 3.0) * G.Gd[i] * divb;
    for (int j = 0; j < 3; ++j) s = s - R(2.0) * G.Atu[i][j] * L.dalpha[j];
    R u = R(0.0);
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) u = u + G.Gu[i][j][k] * G.Atu[j][k];
    R v = R(0.0);
    for (int j = 0; j < 3; ++j) v = v + G.Atu[i][j] * L.dchi[j];
    R q = R(0.0);
    for (int j = 0; j < 3; ++j) q = q + G.gtu[i][j] * L.dK[j];
    s = s + R(2.0) * alpha * (u - R(1.5) * v / chi - R(2.0 / 3.0) * q);
    R mj = R(0.0);
    for (int j = 0; j < 3; ++j) mj = mj + G.gtu[i][j] * M.J[j];
    s = s - pi16 * alpha * mj;
    Gt_rhs[i] = s;
    out[GAM + i] = s;
  }
  // gauge: 1+log or harmonic slicing, Gamma-driver or frozen shift
  {
    R adv = R(0.0);
    for (int k = 0; k < 3; ++k) adv = adv + L.beta[k] * L.dalpha[k];
    R dK = K - R(K_ref(P, t));
    if (P.slicing == 0)
      out[ALP] = adv - R(2.0) * alpha * dK;
    else
      out[ALP] = adv - alpha * alpha * dK;
  }
  for (int i = 0; i < 3; ++i) {
    if (P.shift == 1) {
      R ab = R(0.0), aB = R(0.0), aG = R(0.0);
      for (int j = 0; j < 3; ++j) {
        ab = ab + L.beta[j] * L.dbeta[j][i];
        aB = aB + L.beta[j] * L.dB[j][i];
        aG = aG + L.beta[j] * L.dGt[j][i];
      }
      out[BET + i] = ab + R(0.75) * L.B[i];
      out[BB + i] = aB + (Gt_rhs[i] - aG) - R(P.eta) * L.B[i];
    } else {
      out[BET + i] = R(0.0);
      out[BB + i] = R(0.0);
    }
  }
  // massless scalar field, Pi = -n^mu d_mu phi
  if (P.scalar) {
    int s = P.isc();
    R adv_phi = R(0.0), adv_Pi = R(0.0);
    for (int k = 0; k < 3; ++k) {
      adv_phi = adv_phi + L.beta[k] * L.dphi[k];
      adv_Pi = adv_Pi + L.beta[k] * L.dPi[k];
    }
    R a1 = R(0.0), a2 = R(0.0), a3 = R(0.0), a4 = R(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        a1 = a1 + G.gtu[i][j] * L.ddphi[i][j];
        a3 = a3 + G.gtu[i][j] * L.dchi[i] * L.dphi[j];
        a4 = a4 + G.gtu[i][j] * L.dalpha[i] * L.dphi[j];
      }
    for (int k = 0; k < 3; ++k) a2 = a2 + G.Gd[k] * L.dphi[k];
    R lap_phi = chi * a1 - chi * a2 - R(0.5) * a3;
    out[s] = adv_phi - alpha * L.Pi;
    out[s + 1] = adv_Pi + alpha * K * L.Pi - alpha * lap_phi - chi * a4;
  }
  /* fluid geometric sources (conservative 3+1 form of div T^FL = 0):
   *  d_t(sqrt(g) E)   + d_j[...] = sqrt(g) (alpha K_ij S^ij - J^j d_j alpha)
   *  d_t(sqrt(g) J_i) + d_j[...] = sqrt(g) (-E d_i alpha + J_k d_i beta^k + alpha/2 S^jk d_i gamma_jk) */
  if (P.fluid) {
    int q = P.ifl();
    R sqrtg = R(1.0) / (chi * sqrt(chi));
    R gu[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) gu[i][j] = gu[j][i] = chi * G.gtu[i][j];
    R Su[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) {
        R s = R(0.0);
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) s = s + gu[i][k] * gu[j][l] * M.Sf[k][l];
        Su[i][j] = Su[j][i] = s;
      }
    R Ju[3];
    for (int j = 0; j < 3; ++j) {
      R s = R(0.0);
      for (int k = 0; k < 3; ++k) s = s + gu[j][k] * M.Jf[k];
      Ju[j] = s;
    }
    R KS = R(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        R Kij = (L.At[i][j] + L.gt[i][j] * K / R(3.0)) / chi;
        KS = KS + Kij * Su[i][j];
      }
    R Jda = R(0.0);
    for (int j = 0; j < 3; ++j) Jda = Jda + Ju[j] * L.dalpha[j];
    out[q] = sqrtg * (alpha * KS - Jda);
    for (int i = 0; i < 3; ++i) {
      R s = -M.E * L.dalpha[i];
      for (int k = 0; k < 3; ++k) s = s + M.Jf[k] * L.dbeta[i][k];
      R sg = R(0.0);
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
          R dgam = L.dgt[i][j][k] / chi - L.gt[j][k] * L.dchi[i] / (chi * chi);
          sg = sg + Su[j][k] * dgam;
        }
      s = s + R(0.5) * alpha * sg;
      out[q + 1 + i] = sqrtg * s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Kurganov-Tadmor flux of the fluid through the face between cell p and     */
/* cell p + e_d.  Primitives (rho, v_i) reconstructed with minmod-limited    */
/* linear slopes; face metric = average of the two neighbouring cells.       */
/* ------------------------------------------------------------------------ */
template <class R>
R minmod(R a, R b) {
  if (a > R(0.0) && b > R(0.0)) return rmin<R>(a, b);
  if (a < R(0.0) && b < R(0.0)) return rmax<R>(a, b);
  return R(0.0);
}

template <class R>
struct Prim { R rho, v[3]; };

/* Cell-centred primitive variables.  In the forward and counting modes they
 * are evaluated in plain double (each cell's own recovery is charged once, in
 * matter_sources, by the flop tally); reverse mode tapes them. */
template <class R>
Prim<R> cell_prim(const Field& F, const Params& P, Pt p) {
  R chi = load<R>(F, CHI, p);
  R gt[3][3], gtu[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) gt[i][j] = load<R>(F, GT + sym(i, j), p);
  inverse_sym3<R>(gt, gtu, nullptr);
  R chi32 = chi * sqrt(chi);
  int q = P.ifl();
  R E = load<R>(F, q, p) * chi32, J[3];
  for (int i = 0; i < 3; ++i) J[i] = load<R>(F, q + 1 + i, p) * chi32;
  R J2 = R(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) J2 = J2 + chi * gtu[i][j] * J[i] * J[j];
  Prim<R> r;
  r.rho = fluid_rho<R>(E, J2, P.w);
  R EP = E + R(P.w) * r.rho;
  for (int i = 0; i < 3; ++i) r.v[i] = J[i] / EP;
  return r;
}

template <class R>
void kt_face_flux(const Field& F, const Params& P, Pt p, int d, R H[4]) {
  using PT = typename std::conditional<is_ad<R>::value, R, double>::type;
  Prim<PT> c[4];
  for (int o = -1; o <= 2; ++o) c[o + 1] = cell_prim<PT>(F, P, shift(p, d, o));
  // reconstructed left (from cell p) and right (from cell p+1) face states
  R qL[4], qR[4];
  for (int m = 0; m < 4; ++m) {
    R q0 = R(m == 0 ? c[0].rho : c[0].v[m - 1]);
    R q1 = R(m == 0 ? c[1].rho : c[1].v[m - 1]);
    R q2 = R(m == 0 ? c[2].rho : c[2].v[m - 1]);
    R q3 = R(m == 0 ? c[3].rho : c[3].v[m - 1]);
    qL[m] = q1 + R(0.5) * minmod<R>(q1 - q0, q2 - q1);
    qR[m] = q2 - R(0.5) * minmod<R>(q2 - q1, q3 - q2);
  }
  // face geometry
  Pt p1 = shift(p, d, 1);
  R chi = R(0.5) * (load<R>(F, CHI, p) + load<R>(F, CHI, p1));
  R alpha = R(0.5) * (load<R>(F, ALP, p) + load<R>(F, ALP, p1));
  R betad = R(0.5) * (load<R>(F, BET + d, p) + load<R>(F, BET + d, p1));
  R gt[3][3], gtu[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j)
      gt[i][j] = gt[j][i] = R(0.5) * (load<R>(F, GT + sym(i, j), p) + load<R>(F, GT + sym(i, j), p1));
  inverse_sym3<R>(gt, gtu, nullptr);
  R gu[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) gu[i][j] = gu[j][i] = chi * gtu[i][j];
  R sqrtg = R(1.0) / (chi * sqrt(chi));
  const double w = P.w;
  R U[2][4], Fl[2][4], lam[2][2];
  for (int side = 0; side < 2; ++side) {
    const R* q = side == 0 ? qL : qR;
    R rho = q[0];
    R v[3] = {q[1], q[2], q[3]};
    R vu[3];
    for (int i = 0; i < 3; ++i) {
      R s = R(0.0);
      for (int k = 0; k < 3; ++k) s = s + gu[i][k] * v[k];
      vu[i] = s;
    }
    R v2 = R(0.0);
    for (int i = 0; i < 3; ++i) v2 = v2 + vu[i] * v[i];
    R W2 = R(1.0) / (R(1.0) - v2);
    R Pr = R(w) * rho;
    R hW2 = (rho + Pr) * W2;
    R E = hW2 - Pr;
    U[side][0] = sqrtg * E;
    Fl[side][0] = sqrtg * (alpha * hW2 * vu[d] - betad * E);
    for (int i = 0; i < 3; ++i) {
      R Ji = hW2 * v[i];
      R Sdi = hW2 * vu[d] * v[i] + (i == d ? Pr : R(0.0));
      U[side][1 + i] = sqrtg * Ji;
      Fl[side][1 + i] = sqrtg * (alpha * Sdi - betad * Ji);
    }
    // characteristic speeds along d (sound speed^2 = w)
    R disc = (R(1.0) - v2) * (gu[d][d] * (R(1.0) - v2 * R(w)) - vu[d] * vu[d] * R(1.0 - w));
    R root = R(std::sqrt(w)) * sqrt(disc);
    R pre = alpha / (R(1.0) - v2 * R(w));
    lam[side][0] = pre * (vu[d] * R(1.0 - w) + root) - betad;
    lam[side][1] = pre * (vu[d] * R(1.0 - w) - root) - betad;
  }
  R a = rmax<R>(rmax<R>(fabs(lam[0][0]), fabs(lam[0][1])), rmax<R>(fabs(lam[1][0]), fabs(lam[1][1])));
  for (int m = 0; m < 4; ++m) H[m] = R(0.5) * (Fl[0][m] + Fl[1][m]) - R(0.5) * a * (U[1][m] - U[0][m]);
}

/* Full right-hand side at one point. */
template <class R>
void point_rhs(const Field& F, const Params& P, Pt p, double t, R* out) {
  Local<R> L;
  gather<R>(F, P, p, L);
  point_algebra<R>(L, P, t, out);
  // Kreiss-Oliger dissipation on every field except the fluid
  const int nf = P.nf();
  for (int f = 0; f < nf; ++f) {
    if (P.fluid && f >= P.ifl() && f < P.ifl() + 4) continue;
    out[f] = out[f] + KO<R>(F, f, p, P.sigma);
  }
  // fluid flux divergence
  if (P.fluid) {
    int q = P.ifl();
    for (int d = 0; d < 3; ++d) {
      R Hp[4], Hm[4];
      kt_face_flux<R>(F, P, p, d, Hp);
      if constexpr (is_ad<R>::value) {
        kt_face_flux<R>(F, P, shift(p, d, -1), d, Hm);
      } else {
        double hm[4];
        kt_face_flux<double>(F, P, shift(p, d, -1), d, hm);  // the neighbour's own face
        for (int m = 0; m < 4; ++m) Hm[m] = R(hm[m]);
      }
      for (int m = 0; m < 4; ++m) out[q + m] = out[q + m] - (Hp[m] - Hm[m]) / R(F.g->h[d]);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Constraints: H = R + 2/3 K^2 - At_ij At^ij - 16 pi rho_H,                */
/* M^i = gt^ik gt^jl Dt_j At_kl - 3/(2 chi) At^ij d_j chi                   */
/*       - 2/3 gt^ij d_j K - 8 pi gt^ij J_j                                  */
/* (M^i is the conformal momentum constraint, = physical M^i / chi).         */
/* ------------------------------------------------------------------------ */
void point_constraints(const Field& F, const Params& P, Pt p, double out[4]) {
  Local<double> L;
  gather<double>(F, P, p, L);
  Geom<double> G;
  geometry<double>(L, G);
  Matter<double> M;
  matter_sources<double>(L, P, G.gtu, M);
  out[0] = G.Rs + 2.0 / 3.0 * L.K * L.K - G.AA - 16.0 * PI * M.rho;
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) {
          double DA = L.dAt[j][k][l];
          for (int m = 0; m < 3; ++m) DA = DA - G.Gu[m][j][k] * L.At[m][l] - G.Gu[m][j][l] * L.At[k][m];
          s = s + G.gtu[i][k] * G.gtu[j][l] * DA;
        }
    double v = 0.0, q = 0.0, mj = 0.0;
    for (int j = 0; j < 3; ++j) {
      v = v + G.Atu[i][j] * L.dchi[j];
      q = q + G.gtu[i][j] * L.dK[j];
      mj = mj + G.gtu[i][j] * M.J[j];
    }
    out[1 + i] = s - 1.5 * v / L.chi - 2.0 / 3.0 * q - 8.0 * PI * mj;
  }
}

/* ------------------------------------------------------------------------ */
/* Grid-wide drivers                                                         */
/* ------------------------------------------------------------------------ */
void rhs_all(const Grid& g, const Params& P, const double* state, double t, double* rhs) {
  Field F{&g, state};
  const int nf = P.nf();
  const long N = g.npts();
#pragma omp parallel for schedule(static)
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        double out[NFMAX];
        Pt p{{i, j, k}};
        point_rhs<double>(F, P, p, t, out);
        long idx = (k * g.n[1] + j) * g.n[0] + i;
        for (int f = 0; f < nf; ++f) rhs[f * N + idx] = out[f];
      }
}

/* Classic RK4:  k1 = F(U, t), k2 = F(U + dt/2 k1, t + dt/2),
 * k3 = F(U + dt/2 k2, t + dt/2), k4 = F(U + dt k3, t + dt),
 * U <- U + dt/6 (k1 + 2 k2 + 2 k3 + k4). */
void rk4_step(const Grid& g, const Params& P, double* state, double t, double dt) {
  const long M = (long)P.nf() * g.npts();
  std::vector<double> k1(M), k2(M), k3(M), k4(M), U(M);
  rhs_all(g, P, state, t, k1.data());
  for (long m = 0; m < M; ++m) U[m] = state[m] + 0.5 * dt * k1[m];
  rhs_all(g, P, U.data(), t + 0.5 * dt, k2.data());
  for (long m = 0; m < M; ++m) U[m] = state[m] + 0.5 * dt * k2[m];
  rhs_all(g, P, U.data(), t + 0.5 * dt, k3.data());
  for (long m = 0; m < M; ++m) U[m] = state[m] + dt * k3[m];
  rhs_all(g, P, U.data(), t + dt, k4.data());
  for (long m = 0; m < M; ++m) state[m] = state[m] + dt / 6.0 * (k1[m] + 2.0 * k2[m] + 2.0 * k3[m] + k4[m]);
}

/* ------------------------------------------------------------------------ */
/* Initial data                                                              */
/*  kind 0: gauge wave  ds^2 = -H dt^2 + H dx^2 + dy^2 + dz^2,               */
/*          H = 1 - A sin(2 pi (x - t)/L_x), at time t (flat spacetime).     */
/*  kind 1: FLRW + curvature perturbation at leading gradient order:         */
/*          gamma_ij = a0^2 e^{2 zeta} delta_ij, K = -3 H0, At = 0, alpha = 1,*/
/*          beta = B = 0, fluid at rest, E fixed by the discrete Hamiltonian */
/*          constraint;  zeta = mu exp(-r_e^2/(2 sigma^2)),                  */
/*          r_e^2 = sum_i ((x_i - c_i)/q_i)^2.                               */
/*  kind 2: kind 1 plus a massless-scalar isocurvature profile (section     */
/*          "Examples", spherically symmetric iso-curvature): the scalar    */
/*          is not part of the background metric; at leading gradient      */
/*          order phi = Upsilon(x) = A exp(-r_e^2/(2 sigma^2)), Pi = 0, and  */
/*          the fluid E takes the rest of the discrete Hamiltonian          */
/*          constraint: E = (R + 2/3 K^2 - At.At)/(16 pi) - rho_phi with    */
/*          rho_phi = 1/2 chi gt^ij d_i phi d_j phi (fluid and scalar on).  */
/*  kind 3: kind 1 carried to the next-to-leading order of the gradient     */
/*          expansion (section "Physical system settings", initial-data     */
/*          paragraph: growing mode up to next-leading order in k/(aH));   */
/*          the formulas are derived here, see init_nlo.                    */
/* id[] = {kind, A, mu, sigma, q0, q1, q2, c0, c1, c2, a0, t}               */
/* ------------------------------------------------------------------------ */
/* Lx: wavelength of the gauge wave (0: the grid's own length n_x h_x). */
void init_nlo(const Grid& g, const Params& P, const double* id, double* state);

void init_all(const Grid& g, const Params& P, const double* id, double* state, double Lx_wave = 0.0) {
  const int kind = (int)id[0];
  if (kind == 3) {
    init_nlo(g, P, id, state);
    return;
  }
  const long N = g.npts();
  const int nf = P.nf();
  std::fill(state, state + (long)nf * N, 0.0);
  const double t = id[11];
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        long idx = (k * g.n[1] + j) * g.n[0] + i;
        double x[3] = {g.x0[0] + i * g.h[0], g.x0[1] + j * g.h[1], g.x0[2] + k * g.h[2]};
        double v[NBSSN];
        for (int f = 0; f < NBSSN; ++f) v[f] = 0.0;
        if (kind == 0) {
          double A = id[1], Lx = Lx_wave > 0.0 ? Lx_wave : g.n[0] * g.h[0];
          double ph = 2.0 * PI * (x[0] - t) / Lx;
          double H = 1.0 - A * std::sin(ph);
          double dtH = A * (2.0 * PI / Lx) * std::cos(ph);
          double dxH = -dtH;
          double Kxx = -dtH / (2.0 * std::sqrt(H));
          double Ktr = Kxx / H;
          double chi = std::pow(H, -1.0 / 3.0);
          v[CHI] = chi;
          v[GT + 0] = std::pow(H, 2.0 / 3.0);
          v[GT + 3] = chi;
          v[GT + 5] = chi;
          v[TRK] = Ktr;
          v[AT + 0] = chi * (Kxx - H * Ktr / 3.0);
          v[AT + 3] = -chi * Ktr / 3.0;
          v[AT + 5] = -chi * Ktr / 3.0;
          v[GAM + 0] = 2.0 / 3.0 * std::pow(H, -5.0 / 3.0) * dxH;
          v[ALP] = std::sqrt(H);
        } else {
          double mu = id[2], sig = id[3], a0 = id[10];
          double r2 = 0.0;
          for (int d = 0; d < 3; ++d) {
            double u = (x[d] - id[7 + d]) / id[4 + d];
            r2 = r2 + u * u;
          }
          double zeta = mu * std::exp(-r2 / (2.0 * sig * sig));
          v[CHI] = std::exp(-2.0 * zeta) / (a0 * a0);
          v[GT + 0] = v[GT + 3] = v[GT + 5] = 1.0;
          v[TRK] = -3.0 * P.H0;
          v[ALP] = 1.0;
          if (kind == 2) state[(long)P.isc() * N + idx] = id[1] * std::exp(-r2 / (2.0 * sig * sig));  // phi
        }
        for (int f = 0; f < NBSSN; ++f) state[f * N + idx] = v[f];
      }
  if ((kind == 1 || kind == 2) && P.fluid) {
    // E from the discrete Hamiltonian constraint with the fluid at rest
    std::vector<double> E(N);
    Params Pv = P;
    Pv.fluid = 0;
    Pv.scalar = 0;
    Field F{&g, state};
#pragma omp parallel for schedule(static)
    for (long k = 0; k < g.n[2]; ++k)
      for (long j = 0; j < g.n[1]; ++j)
        for (long i = 0; i < g.n[0]; ++i) {
          Pt p{{i, j, k}};
          Local<double> L;
          gather<double>(F, Pv, p, L);
          Geom<double> G;
          geometry<double>(L, G);
          double e = (G.Rs + 2.0 / 3.0 * L.K * L.K - G.AA) / (16.0 * PI);
          if (kind == 2) {
            double dphi[3], s2 = 0.0;
            grad<double>(F, P.isc(), p, dphi);
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) s2 = s2 + G.gtu[a][b] * dphi[a] * dphi[b];
            e = e - 0.5 * L.chi * s2;  // rho of the scalar with Pi = 0
          }
          E[(k * g.n[1] + j) * g.n[0] + i] = e;
        }
    int q = P.ifl();
    for (long m = 0; m < N; ++m) {
      double chi = state[CHI * N + m];
      state[q * N + m] = E[m] / (chi * std::sqrt(chi));
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Next-to-leading-order long-wavelength data (kind 3).  The paper takes     */
/* the growing mode of the gradient expansion in eps = k/(aH) up to the next */
/* order and leaves the formulas to the papers it cites; they are derived    */
/* here.  Background: flat FLRW filled with P = w rho, a ~ t^{2/(3(1+w))},  */
/* slices of constant mean curvature K = -3 H(t), zero shift.  Leading       */
/* order: gamma_ij = a^2 psi^4 delta_ij with psi = e^{zeta/2} fixed in time */
/* (chi0 = a^-2 psi^-4), K_ij = -H gamma_ij, alpha = 1.  Every O(eps^2)      */
/* correction of the growing mode is proportional to g(t) = 1/(a H)^2, whose */
/* rate is d ln g/dt = (1 + 3w) H.  With R_ij the Ricci tensor of the        */
/* leading-order metric (lower indices, the same for any constant scale),    */
/* M_ij = R_ij - 1/3 delta_ij delta^kl R_kl and R = chi0 delta^kl R_kl:      */
/*  - trace-free evolution d_t At_ij = chi R_ij^TF - 3 H At_ij + O(eps^4)    */
/*    (D_i D_j alpha and S_ij^TF are O(eps^4)); its growing solution         */
/*    At_ij = 2 chi0 M_ij / ((5 + 3w) H);                                   */
/*  - d_t gt_ij = -2 At_ij: gt_ij = delta_ij + h_ij,                         */
/*    h_ij = -4 chi0 M_ij / ((5 + 3w)(1 + 3w) H^2), taken to unit            */
/*    determinant (which changes it at O(eps^4));                           */
/*  - Hamiltonian constraint: delta = (E - E_b)/E_b = R / (6 H^2);           */
/*  - d_t K = 0 (constant mean curvature) with the K equation fixes the      */
/*    lapse: alpha = 1 - (1 + 3w) delta / (3 (1 + w));                      */
/*  - d_t ln chi = -2 alpha H puts that lapse into the conformal factor:     */
/*    chi = chi0 (1 + 2 delta / (3 (1 + w)));                                */
/*  - beta = B = 0; Gt^i = gt^jk Gt^i_jk of the new gt (4th-order            */
/*    differences, so the conformal-connection constraint holds to           */
/*    rounding); E and J_i from the discrete Hamiltonian and momentum        */
/*    constraints of the new metric (J = O(eps^3): the fluid is no longer   */
/*    at rest), as the paper's data meet the constraints to rounding.       */
/* R_ij and R are those of the right-hand side (geometry()) on the          */
/* leading-order data; H = H0 and a = a0 at the initial time.  Needs the     */
/* fluid on and H0 > 0.                                                      */
/* ------------------------------------------------------------------------ */
void init_nlo(const Grid& g, const Params& P, const double* id, double* state) {
  const long N = g.npts();
  const int nf = P.nf();
  const double w = P.w, H0 = P.H0;
  std::fill(state, state + (long)nf * N, 0.0);
  // leading-order metric (kind 1 without its fluid)
  Params Pv = P;
  Pv.fluid = 0;
  Pv.scalar = 0;
  std::vector<double> lo((size_t)NBSSN * N);
  std::vector<double> id1(id, id + 12);
  id1[0] = 1.0;
  init_all(g, Pv, id1.data(), lo.data());
  // O(eps^2) corrections from the leading-order Ricci tensor
  std::vector<double> nlo(lo);
  Field F0{&g, lo.data()};
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        const long m = (k * g.n[1] + j) * g.n[0] + i;
        Pt p{{i, j, k}};
        Local<double> L;
        gather<double>(F0, Pv, p, L);
        Geom<double> G;
        geometry<double>(L, G);
        const double chi0 = L.chi;
        const double trR = G.Ric[0][0] + G.Ric[1][1] + G.Ric[2][2];
        const double delta = G.Rs / (6.0 * H0 * H0);
        double M[3][3], gm[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            M[a][b] = G.Ric[a][b] - (a == b ? trR / 3.0 : 0.0);
            const double h = -4.0 * chi0 * M[a][b] / ((5.0 + 3.0 * w) * (1.0 + 3.0 * w) * H0 * H0);
            gm[a][b] = (a == b ? 1.0 : 0.0) + h;
          }
        const double det = gm[0][0] * (gm[1][1] * gm[2][2] - gm[1][2] * gm[2][1]) -
                           gm[0][1] * (gm[1][0] * gm[2][2] - gm[1][2] * gm[2][0]) +
                           gm[0][2] * (gm[1][0] * gm[2][1] - gm[1][1] * gm[2][0]);
        const double s = 1.0 / std::cbrt(det);
        for (int a = 0; a < 3; ++a)
          for (int b = a; b < 3; ++b) {
            nlo[(GT + sym(a, b)) * N + m] = gm[a][b] * s;
            nlo[(AT + sym(a, b)) * N + m] = 2.0 * chi0 * M[a][b] / ((5.0 + 3.0 * w) * H0);
          }
        nlo[CHI * N + m] = chi0 * (1.0 + 2.0 * delta / (3.0 * (1.0 + w)));
        nlo[ALP * N + m] = 1.0 - (1.0 + 3.0 * w) * delta / (3.0 * (1.0 + w));
      }
  // conformal connection functions of the new conformal metric
  std::vector<double> gam(3 * (size_t)N);
  Field F1{&g, nlo.data()};
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        Pt p{{i, j, k}};
        Local<double> L;
        gather<double>(F1, Pv, p, L);
        Geom<double> G;
        geometry<double>(L, G);
        for (int a = 0; a < 3; ++a) gam[a * N + (k * g.n[1] + j) * g.n[0] + i] = G.Gd[a];
      }
  for (int a = 0; a < 3; ++a)
    for (long m = 0; m < N; ++m) nlo[(GAM + a) * N + m] = gam[a * N + m];
  // fluid E and J_i from the discrete constraints of the final metric (no matter in Pv)
  for (int f = 0; f < NBSSN; ++f)
    for (long m = 0; m < N; ++m) state[f * N + m] = nlo[f * N + m];
  Field F2{&g, nlo.data()};
  const int q = P.ifl();
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        const long m = (k * g.n[1] + j) * g.n[0] + i;
        Pt p{{i, j, k}};
        double c[4];
        point_constraints(F2, Pv, p, c);  // H = 16 pi E, M^i = 8 pi gt^ij J_j when they vanish
        const double chi = nlo[CHI * N + m];
        const double chi32 = chi * std::sqrt(chi);
        state[q * N + m] = c[0] / (16.0 * PI) / chi32;
        for (int a = 0; a < 3; ++a) {
          double Ja = 0.0;
          for (int b = 0; b < 3; ++b) Ja = Ja + nlo[(GT + sym(a, b)) * N + m] * c[1 + b];
          state[(q + 1 + a) * N + m] = Ja / (8.0 * PI) / chi32;
        }
      }
}

/* ------------------------------------------------------------------------ */
/* Fixed mesh refinement (section "Statement of need": a fixed set of       */
/* nested refinement levels resolves the collapsing region; the figure of   */
/* the lapse at horizon formation shows the lowest level and two refined    */
/* ones).  The paper gives no scheme for it; the readings taken here:       */
/*  - level 0 is the periodic box; level l >= 1 is one box of points with   */
/*    spacing h_l = h_{l-1}/2 whose point 0 lies at x0_{l-1} + origin h_l,  */
/*    so that every other point of level l sits on a point of level l-1;    */
/*  - the points of level l outside its interior box [lo, hi) are ghost     */
/*    points (at least 3 layers, the reach of the Kreiss-Oliger stencil),   */
/*    set from level l-1 before every RK4 stage; along an axis on which     */
/*    level l-1 is periodic, level l may instead be periodic too (lo = 0,   */
/*    hi = n = 2 n_{l-1}, origin 0);                                        */
/*  - ghost values in space: the tensor product of 1D Lagrange interpolation*/
/*    through the 6 nearest parent points (degree 5) where the child point  */
/*    falls half-way between parent points, the parent value where it       */
/*    falls on one;                                                         */
/*  - in time (Berger-Oliger subcycling: level l takes two steps of         */
/*    dt_{l-1}/2 after each step of level l-1): the continuous extension of */
/*    order 3 of classic RK4 over the parent's step,                        */
/*      U(t + theta dt) = U_n + dt sum_s b_s(theta) k_s,                     */
/*      b_1 = theta - 3/2 theta^2 + 2/3 theta^3,                             */
/*      b_2 = b_3 = theta^2 - 2/3 theta^3,  b_4 = -1/2 theta^2 + 2/3 theta^3 */
/*    (the polynomials that satisfy the order conditions sum b_s = theta,   */
/*    sum b_s c_s = theta^2/2, sum b_s c_s^2 = theta^3/3 and                 */
/*    sum b_s a_sr c_r = theta^3/6 for c = (0, 1/2, 1/2, 1));               */
/*  - after the two substeps, the interior points of level l that lie on   */
/*    points of level l-1 overwrite those values (injection).               */
/* The right-hand side of a level >= 1 is evaluated at its interior points */
/* only; their stencils (reach 3) stay inside the level's own array.        */
/* ------------------------------------------------------------------------ */
constexpr int FMR_MAXL = 8;

struct Hier {
  int L;
  Grid g[FMR_MAXL];
  long origin[FMR_MAXL][3], lo[FMR_MAXL][3], hi[FMR_MAXL][3];
  bool per[FMR_MAXL][3];  // axis periodic on this level
};

Hier make_hier(int L, const int* n, const double* h, const double* x0, const int* origin, const int* lo,
               const int* hi) {
  Hier H;
  H.L = L;
  for (int l = 0; l < L; ++l) {
    H.g[l] = make_grid(n + 3 * l, h + 3 * l, x0 + 3 * l);
    for (int d = 0; d < 3; ++d) {
      H.origin[l][d] = l ? origin[3 * l + d] : 0;
      H.lo[l][d] = l ? lo[3 * l + d] : 0;
      H.hi[l][d] = l ? hi[3 * l + d] : n[3 * l + d];
      H.per[l][d] = l == 0 || (H.per[l - 1][d] && H.lo[l][d] == 0 && H.hi[l][d] == n[3 * l + d] &&
                               H.origin[l][d] == 0 && n[3 * l + d] == 2 * n[3 * (l - 1) + d]);
    }
  }
  return H;
}

bool interior(const Hier& H, int l, long i, long j, long k) {
  const long q[3] = {i, j, k};
  for (int d = 0; d < 3; ++d)
    if (q[d] < H.lo[l][d] || q[d] >= H.hi[l][d]) return false;
  return true;
}

inline long floordiv2(long a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

/* Lagrange weights at x = 0 for nodes x_m = m - 2.5, m = 0..5 (the six parent
 * points around a half-way child point, in parent spacings). */
void lagrange6_half(double w[6]) {
  for (int m = 0; m < 6; ++m) {
    double num = 1.0, den = 1.0;
    const double xm = m - 2.5;
    for (int q = 0; q < 6; ++q) {
      if (q == m) continue;
      const double xq = q - 2.5;
      num = num * (0.0 - xq);
      den = den * (xm - xq);
    }
    w[m] = num / den;
  }
}

/* Parent taps of child index i along axis d of level l (1 or 6 points). */
int parent_taps(const Hier& H, int l, int d, long i, long idx[6], double w[6]) {
  const long X2 = H.origin[l][d] + i;  // child point position in child spacings from parent point 0
  const long np = H.g[l - 1].n[d];
  if (X2 % 2 == 0) {
    idx[0] = X2 / 2;
    w[0] = 1.0;
  } else {
    const long base = floordiv2(X2);  // parent point just below
    lagrange6_half(w);
    for (int m = 0; m < 6; ++m) idx[m] = base - 2 + m;
  }
  const int nt = (X2 % 2 == 0) ? 1 : 6;
  if (H.per[l - 1][d])
    for (int m = 0; m < nt; ++m) idx[m] = wrapi(idx[m], np);
  return nt;
}

/* Ghost points of level l from a parent state P (level l-1 layout). */
void prolong(const Hier& H, int l, int nf, const double* P, double* C) {
  const Grid& gc = H.g[l];
  const Grid& gp = H.g[l - 1];
  const long Nc = gc.npts(), Np = gp.npts();
#pragma omp parallel for schedule(static)
  for (long k = 0; k < gc.n[2]; ++k)
    for (long j = 0; j < gc.n[1]; ++j)
      for (long i = 0; i < gc.n[0]; ++i) {
        if (interior(H, l, i, j, k)) continue;
        long ix[6], iy[6], iz[6];
        double wx[6], wy[6], wz[6];
        const int nx = parent_taps(H, l, 0, i, ix, wx);
        const int ny = parent_taps(H, l, 1, j, iy, wy);
        const int nz = parent_taps(H, l, 2, k, iz, wz);
        const long c = (k * gc.n[1] + j) * gc.n[0] + i;
        for (int f = 0; f < nf; ++f) {
          double s = 0.0;
          for (int c3 = 0; c3 < nz; ++c3)
            for (int b = 0; b < ny; ++b)
              for (int a = 0; a < nx; ++a)
                s = s + wz[c3] * wy[b] * wx[a] * P[f * Np + (iz[c3] * gp.n[1] + iy[b]) * gp.n[0] + ix[a]];
          C[f * Nc + c] = s;
        }
      }
}

/* Interior points of level l lying on level l-1 points overwrite those. */
void restrict_to_parent(const Hier& H, int l, int nf, const double* C, double* P) {
  const Grid& gc = H.g[l];
  const Grid& gp = H.g[l - 1];
  const long Nc = gc.npts(), Np = gp.npts();
  for (long k = H.lo[l][2]; k < H.hi[l][2]; ++k)
    for (long j = H.lo[l][1]; j < H.hi[l][1]; ++j)
      for (long i = H.lo[l][0]; i < H.hi[l][0]; ++i) {
        const long q[3] = {i, j, k};
        long pq[3];
        bool on = true;
        for (int d = 0; d < 3; ++d) {
          const long X2 = H.origin[l][d] + q[d];
          if (X2 % 2 != 0) on = false;
          pq[d] = H.per[l - 1][d] ? wrapi(floordiv2(X2), gp.n[d]) : floordiv2(X2);
        }
        if (!on) continue;
        const long cc = (k * gc.n[1] + j) * gc.n[0] + i;
        const long pc = (pq[2] * gp.n[1] + pq[1]) * gp.n[0] + pq[0];
        for (int f = 0; f < nf; ++f) P[f * Np + pc] = C[f * Nc + cc];
      }
}

/* The continuous extension of RK4: out = U_n + dt sum_s b_s(theta) k_s. */
void rk4_dense(long M, const double* Un, const double* const k[4], double dt, double theta, double* out) {
  const double t2 = theta * theta, t3 = t2 * theta;
  const double b[4] = {theta - 1.5 * t2 + 2.0 / 3.0 * t3, t2 - 2.0 / 3.0 * t3, t2 - 2.0 / 3.0 * t3,
                       -0.5 * t2 + 2.0 / 3.0 * t3};
  for (long m = 0; m < M; ++m)
    out[m] = Un[m] + dt * (b[0] * k[0][m] + b[1] * k[1][m] + b[2] * k[2][m] + b[3] * k[3][m]);
}

/* One parent step kept for the child's ghost values. */
struct Saved {
  std::vector<double> Un, k[4];
  double dt;
};

/* Right-hand side at the interior points of level l (zero at ghost points). */
void rhs_level(const Hier& H, const Params& P, int l, const double* state, double t, double* rhs) {
  const Grid& g = H.g[l];
  Field F{&g, state};
  const int nf = P.nf();
  const long N = g.npts();
#pragma omp parallel for schedule(static)
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        const long idx = (k * g.n[1] + j) * g.n[0] + i;
        if (!interior(H, l, i, j, k)) {
          for (int f = 0; f < nf; ++f) rhs[f * N + idx] = 0.0;
          continue;
        }
        double out[NFMAX];
        Pt p{{i, j, k}};
        point_rhs<double>(F, P, p, t, out);
        for (int f = 0; f < nf; ++f) rhs[f * N + idx] = out[f];
      }
}

/* Ghost values of the RK4 stages of a child substep.  The stage states of
 * classic RK4 applied to a solution u with time derivatives u1 = u',
 * u2 = u'', u3 = u''' at the substep's start (step tau) are, to the order
 * that matters here,
 *   Y_1 = u,  Y_2 = u + tau/2 u1,  Y_3 = u + tau/2 u1 + tau^2/4 u2,
 *   Y_4 = u + tau u1 + tau^2/2 u2 + tau^3/4 u3
 * (exact for a linear autonomous system: Y_2 = u + tau/2 L u, Y_3 = u +
 * tau/2 L Y_2, Y_4 = u + tau L Y_3).  Setting the ghost points of stage s to
 * Y_s built from the parent's continuous extension u(theta), instead of to u
 * at the stage time, keeps the ghost data consistent with the interior's
 * stage states (the stage-consistent interpolation of McCorquodale and
 * Colella, 2011); plain values at the stage times lose about one order.
 * With tau = r dt_parent and d/dt = (1/dt_parent) d/dtheta, the ghost value
 * of stage s is U_n + dt_parent sum_q beta_q k_q, beta built from b_q(theta0)
 * and its theta-derivatives. */
void ghost_stage_coeffs(double theta0, int stage, double r, double beta[4]) {
  const double th = theta0, t2 = th * th, t3 = t2 * th;
  // b_q(theta) of the continuous extension and its first three derivatives
  const double b0[4] = {th - 1.5 * t2 + 2.0 / 3.0 * t3, t2 - 2.0 / 3.0 * t3, t2 - 2.0 / 3.0 * t3,
                        -0.5 * t2 + 2.0 / 3.0 * t3};
  const double b1[4] = {1.0 - 3.0 * th + 2.0 * t2, 2.0 * th - 2.0 * t2, 2.0 * th - 2.0 * t2, -th + 2.0 * t2};
  const double b2[4] = {-3.0 + 4.0 * th, 2.0 - 4.0 * th, 2.0 - 4.0 * th, -1.0 + 4.0 * th};
  const double b3[4] = {4.0, -4.0, -4.0, 4.0};
  double c1 = 0.0, c2 = 0.0, c3 = 0.0;  // weights of the first, second, third theta-derivative
  if (stage == 2) c1 = r / 2.0;
  if (stage == 3) {
    c1 = r / 2.0;
    c2 = r * r / 4.0;
  }
  if (stage == 4) {
    c1 = r;
    c2 = r * r / 2.0;
    c3 = r * r * r / 4.0;
  }
  for (int q = 0; q < 4; ++q) beta[q] = b0[q] + c1 * b1[q] + c2 * b2[q] + c3 * b3[q];
}

/* Ghost points of level l for stage `stage` of its substep that starts at
 * theta0 of the parent's saved step (child step = half the parent's). */
void fill_ghosts(const Hier& H, const Params& P, int l, const Saved& S, double theta0, int stage, double* C) {
  const long Mp = (long)P.nf() * H.g[l - 1].npts();
  double beta[4];
  ghost_stage_coeffs(theta0, stage, 0.5, beta);
  std::vector<double> Y(Mp);
  for (long m = 0; m < Mp; ++m)
    Y[m] = S.Un[m] + S.dt * (beta[0] * S.k[0][m] + beta[1] * S.k[1][m] + beta[2] * S.k[2][m] +
                             beta[3] * S.k[3][m]);
  prolong(H, l, P.nf(), Y.data(), C);
}

/* One step of level l from t (starting at theta0 of the parent's step)
 * followed, when level l+1 exists, by its two substeps and the injection. */
void fmr_advance(const Hier& H, const Params& P, double* const* U, std::vector<Saved>& S, int l, double t,
                 double dt, double theta0) {
  const long M = (long)P.nf() * H.g[l].npts();
  double* u = U[l];
  std::vector<double> k[4], Y(M);
  for (int s = 0; s < 4; ++s) k[s].resize(M);
  auto ghosts = [&](double* X, int stage) {
    if (l > 0) fill_ghosts(H, P, l, S[l - 1], theta0, stage, X);
  };
  ghosts(u, 1);
  std::vector<double> Un(u, u + M);
  rhs_level(H, P, l, Un.data(), t, k[0].data());
  for (long m = 0; m < M; ++m) Y[m] = Un[m] + 0.5 * dt * k[0][m];
  ghosts(Y.data(), 2);
  rhs_level(H, P, l, Y.data(), t + 0.5 * dt, k[1].data());
  for (long m = 0; m < M; ++m) Y[m] = Un[m] + 0.5 * dt * k[1][m];
  ghosts(Y.data(), 3);
  rhs_level(H, P, l, Y.data(), t + 0.5 * dt, k[2].data());
  for (long m = 0; m < M; ++m) Y[m] = Un[m] + dt * k[2][m];
  ghosts(Y.data(), 4);
  rhs_level(H, P, l, Y.data(), t + dt, k[3].data());
  for (long m = 0; m < M; ++m) u[m] = Un[m] + dt / 6.0 * (k[0][m] + 2.0 * k[1][m] + 2.0 * k[2][m] + k[3][m]);
  if (l + 1 < H.L) {
    S[l].Un = Un;
    for (int s = 0; s < 4; ++s) S[l].k[s] = k[s];
    S[l].dt = dt;
    fmr_advance(H, P, U, S, l + 1, t, 0.5 * dt, 0.0);
    fmr_advance(H, P, U, S, l + 1, t + 0.5 * dt, 0.5 * dt, 0.5);
    restrict_to_parent(H, l + 1, P.nf(), U[l + 1], u);
  }
}

/* One step of the hierarchy (level 0 by dt0, level l by 2^l steps of
 * dt0/2^l), then the ghost points of every level from its parent's new state. */
void fmr_step(const Hier& H, const Params& P, double* const* U, double t, double dt0) {
  std::vector<Saved> S(H.L);
  fmr_advance(H, P, U, S, 0, t, dt0, 0.0);
  for (int l = 1; l < H.L; ++l) prolong(H, l, P.nf(), U[l - 1], U[l]);
}

/* Initial data on every level (each from its own points and discrete
 * constraint), injection from the finest level down, then the ghost points
 * of every level from its parent. */
void fmr_init(const Hier& H, const Params& P, const double* id, double* const* U) {
  const double Lx = H.g[0].n[0] * H.g[0].h[0];  // the gauge wave's wavelength is the periodic box
  for (int l = 0; l < H.L; ++l) init_all(H.g[l], P, id, U[l], Lx);
  for (int l = H.L - 1; l >= 1; --l) restrict_to_parent(H, l, P.nf(), U[l], U[l - 1]);
  for (int l = 1; l < H.L; ++l) prolong(H, l, P.nf(), U[l - 1], U[l]);
}

}  // namespace

/* ------------------------------------------------------------------------ */
/* Collapse diagnostics and initial data from a per-point zeta: the        */
/* quantities a threshold search differentiates (the paper's PBH examples  */
/* follow the lapse at the centre and the compaction of the overdensity,   */
/* section "Examples"; it defines neither).  Readings taken here:           */
/*  - zeta map: the leading-order FLRW + curvature-perturbation data of     */
/*    init_all kind 1 with zeta given at every grid point instead of the    */
/*    Gaussian: chi = exp(-2 zeta)/a0^2, gt = delta, K = -3 H0, At = 0,     */
/*    Gt = 0, alpha = 1, beta = B = 0, fluid at rest, E from the discrete   */
/*    Hamiltonian constraint, tau~ = E chi^{-3/2} (section "Physical system */
/*    settings", initial-data paragraph);                                   */
/*  - central lapse: alpha at the grid point c = (nx/2, ny/2, nz/2); its    */
/*    minimum over the time levels t_0 .. t_N of a run;                     */
/*  - compaction function about c on a grid of equal spacing h:             */
/*      C(r_k) = 2 dM(r_k) / R(r_k),  r_k = k h,  k = 1 .. kmax,            */
/*      dM(r_k) = h^3 sum over the points with |x - c| < r_k of             */
/*                (tau~ - Ebar sqrt(gamma)),  sqrt(gamma) = chi^{-3/2},     */
/*      Ebar = (box sum of tau~) / (box sum of sqrt(gamma)): the volume-    */
/*             weighted mean energy density, so dM is the mass excess;      */
/*      R(r_k) = r_k times the mean of chi^{-1/2} over the six grid points  */
/*             on the axes through c at distance r_k (the areal radius of   */
/*             the conformally flat metric delta/chi);                      */
/*    |x - c| < r_k is decided in integers: di^2 + dj^2 + dk^2 < k^2;       */
/*    the peak compaction is the largest C(r_k).                            */
/* The reverse modes are tapes over these same templated functions.         */
/* ------------------------------------------------------------------------ */
template <class R>
void init_zeta(const Grid& g, const Params& P, const R* zeta, double a0, std::vector<R>& st) {
  const long N = g.npts();
  const int nf = P.nf();
  st.assign((size_t)nf * N, R(0.0));
  for (long m = 0; m < N; ++m) {
    st[CHI * N + m] = exp(R(-2.0) * zeta[m]) / R(a0 * a0);
    st[(GT + 0) * N + m] = R(1.0);
    st[(GT + 3) * N + m] = R(1.0);
    st[(GT + 5) * N + m] = R(1.0);
    st[TRK * N + m] = R(-3.0 * P.H0);
    st[ALP * N + m] = R(1.0);
  }
  if (!P.fluid) return;
  // E from the discrete Hamiltonian constraint of the metric just set
  std::vector<double> v((size_t)nf * N);
  std::vector<long> ids((size_t)nf * N);
  for (size_t q = 0; q < v.size(); ++q) {
    v[q] = val(st[q]);
    ids[q] = tape_id(st[q]);
  }
  Field F{&g, v.data(), is_ad<R>::value ? ids.data() : nullptr};
  Params Pv = P;
  Pv.fluid = 0;
  Pv.scalar = 0;
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        Pt p{{i, j, k}};
        Local<R> L;
        gather<R>(F, Pv, p, L);
        Geom<R> G;
        geometry<R>(L, G);
        R E = (G.Rs + R(2.0 / 3.0) * L.K * L.K - G.AA) / R(16.0 * PI);
        st[(long)P.ifl() * N + (k * g.n[1] + j) * g.n[0] + i] = E / (L.chi * sqrt(L.chi));
      }
}

template <class R>
void compaction(const Grid& g, const Params& P, const Field& F, int kmax, R* C) {
  const long c[3] = {g.n[0] / 2, g.n[1] / 2, g.n[2] / 2};
  const double h = g.h[0];
  const int q = P.ifl();
  R St = R(0.0), Sg = R(0.0);
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        Pt p{{i, j, k}};
        R chi = load<R>(F, CHI, p);
        St = St + load<R>(F, q, p);
        Sg = Sg + R(1.0) / (chi * sqrt(chi));
      }
  R Ebar = St / Sg;
  for (int kk = 1; kk <= kmax; ++kk) {
    R dM = R(0.0);
    for (long k = 0; k < g.n[2]; ++k)
      for (long j = 0; j < g.n[1]; ++j)
        for (long i = 0; i < g.n[0]; ++i) {
          const long di = i - c[0], dj = j - c[1], dk = k - c[2];
          if (di * di + dj * dj + dk * dk >= (long)kk * kk) continue;
          Pt p{{i, j, k}};
          R chi = load<R>(F, CHI, p);
          dM = dM + (load<R>(F, q, p) - Ebar / (chi * sqrt(chi)));
        }
    R s6 = R(0.0);
    for (int d = 0; d < 3; ++d)
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        Pt p{{c[0], c[1], c[2]}};
        p.i[d] += sgn * kk;
        s6 = s6 + R(1.0) / sqrt(load<R>(F, CHI, p));
      }
    R Rk = R(kk * h) * (s6 / R(6.0));
    C[kk - 1] = R(2.0 * h * h * h) * dM / Rk;
  }
}

/* ======================================================================== */
/* C API (ctypes)                                                            */
/*   n[3] grid points, h[3] spacings, x0[3] coordinate of point 0,           */
/*   params[9] = {slicing, shift, eta, ko_sigma, w, fluid, scalar, H0, t0}   */
/* ======================================================================== */
extern "C" {

int oracle_nfields(const double* params) { return unpack_params(params).nf(); }

/* Fluid rest-frame density from E and J^2 = gamma^ij J_i J_j (the recovery
 * used by the right-hand side), for n values. */
void oracle_fluid_rho(const double* E, const double* J2, long n, double w, double* rho) {
  for (long m = 0; m < n; ++m) rho[m] = fluid_rho<double>(E[m], J2[m], w);
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_rhs(const int* n, const double* h, const double* x0, const double* params, const double* state,
                double t, double* rhs) {
  Grid g = make_grid(n, h, x0);
  rhs_all(g, unpack_params(params), state, t, rhs);
}

/* RHS at a list of points only: pts = (i, j, k) triples; out[npts][nf]. */
void oracle_rhs_points(const int* n, const double* h, const double* x0, const double* params, const double* state,
                       double t, long npts, const long* pts, double* out) {
  Grid g = make_grid(n, h, x0);
  Params P = unpack_params(params);
  Field F{&g, state};
  const int nf = P.nf();
#pragma omp parallel for schedule(dynamic, 1)
  for (long m = 0; m < npts; ++m) {
    Pt p{{pts[3 * m], pts[3 * m + 1], pts[3 * m + 2]}};
    point_rhs<double>(F, P, p, t, out + m * nf);
  }
}

/* RHS on the z-planes [k0, k1) only (rhs holds only those planes). */
void oracle_rhs_planes(const int* n, const double* h, const double* x0, const double* params, const double* state,
                       double t, long k0, long k1, double* rhs) {
  Grid g = make_grid(n, h, x0);
  Params P = unpack_params(params);
  Field F{&g, state};
  const int nf = P.nf();
  const long plane = g.n[0] * g.n[1], M = (k1 - k0) * plane;
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
  for (long k = k0; k < k1; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        double out[NFMAX];
        Pt p{{i, j, k}};
        point_rhs<double>(F, P, p, t, out);
        long idx = (k - k0) * plane + j * g.n[0] + i;
        for (int f = 0; f < nf; ++f) rhs[f * M + idx] = out[f];
      }
}

void oracle_rk4_step(const int* n, const double* h, const double* x0, const double* params, double* state, double t,
                     double dt) {
  Grid g = make_grid(n, h, x0);
  rk4_step(g, unpack_params(params), state, t, dt);
}

/* Pointwise constraints (ham_mom[4][n] or NULL) and norms[8] =
 * {L2(H), L2(Mx), L2(My), L2(Mz), Linf(H), Linf(Mx), Linf(My), Linf(Mz)},
 * L2 = sqrt(mean of squares) over all points. */
void oracle_constraints(const int* n, const double* h, const double* x0, const double* params, const double* state,
                        double* ham_mom, double* norms) {
  Grid g = make_grid(n, h, x0);
  Params P = unpack_params(params);
  Field F{&g, state};
  const long N = g.npts();
  std::vector<double> c(4 * N);
#pragma omp parallel for schedule(static)
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        double o[4];
        Pt p{{i, j, k}};
        point_constraints(F, P, p, o);
        long idx = (k * g.n[1] + j) * g.n[0] + i;
        for (int m = 0; m < 4; ++m) c[m * N + idx] = o[m];
      }
  for (int m = 0; m < 4; ++m) {
    double s2 = 0.0, mx = 0.0;
    for (long q = 0; q < N; ++q) {
      double v = c[m * N + q];
      s2 = s2 + v * v;
      mx = std::max(mx, std::fabs(v));
    }
    norms[m] = std::sqrt(s2 / (double)N);
    norms[4 + m] = mx;
  }
  if (ham_mom) std::memcpy(ham_mom, c.data(), sizeof(double) * 4 * N);
}

void oracle_init(const int* n, const double* h, const double* x0, const double* params, const double* id,
                 double* state) {
  Grid g = make_grid(n, h, x0);
  init_all(g, unpack_params(params), id, state);
}

/* Reverse mode of the right-hand side: out = (dF/dU)^T w, w and out in state
 * layout, by recording F(U) on a tape (every point, every operation) and one
 * reverse sweep.  Single-threaded; meant for tiny grids (tape ~1e4 nodes per
 * point). */
void oracle_rhs_vjp(const int* n, const double* h, const double* x0, const double* params, const double* state,
                    double t, const double* w, double* out) {
  Grid g = make_grid(n, h, x0);
  Params P = unpack_params(params);
  Field F{&g, state};
  const int nf = P.nf();
  const long N = g.npts(), M = (long)nf * N;
  g_tape.clear();
  g_tape.reserve((size_t)M + (size_t)N * 20000);
  for (long m = 0; m < M; ++m) g_tape.push_back(TapeNode{-1, -1, 0.0, 0.0});  // leaves = state entries
  std::vector<std::pair<long, double>> seeds;
  for (long k = 0; k < g.n[2]; ++k)
    for (long j = 0; j < g.n[1]; ++j)
      for (long i = 0; i < g.n[0]; ++i) {
        AD o[NFMAX];
        Pt p{{i, j, k}};
        point_rhs<AD>(F, P, p, t, o);
        long idx = (k * g.n[1] + j) * g.n[0] + i;
        for (int f = 0; f < nf; ++f)
          if (o[f].id >= 0) seeds.push_back({o[f].id, w[f * N + idx]});
      }
  std::vector<double> adj(g_tape.size(), 0.0);
  for (auto& sd : seeds) adj[sd.first] += sd.second;
  for (long q = (long)g_tape.size() - 1; q >= M; --q) {
    const double a = adj[q];
    if (a == 0.0) continue;
    const TapeNode& nd = g_tape[q];
    if (nd.a >= 0) adj[nd.a] += a * nd.da;
    if (nd.b >= 0) adj[nd.b] += a * nd.db;
  }
  for (long m = 0; m < M; ++m) out[m] = adj[m];
  g_tape.clear();
  g_tape.shrink_to_fit();
}

/* Algorithmic operation count of one RHS evaluation at one point:
 * counts[5] = {add/sub, mul, div, sqrt, compare}.  Evaluated at point
 * (n/2, n/2, n/2) of the supplied state. */
void oracle_flop_count(const int* n, const double* h, const double* x0, const double* params, const double* state,
                       double t, double* counts) {
  Grid g = make_grid(n, h, x0);
  Params P = unpack_params(params);
  Field F{&g, state};
  g_tally = Tally{0, 0, 0, 0, 0};
  Cnt out[NFMAX];
  Pt p{{g.n[0] / 2, g.n[1] / 2, g.n[2] / 2}};
  point_rhs<Cnt>(F, P, p, t, out);
  counts[0] = g_tally.add;
  counts[1] = g_tally.mul;
  counts[2] = g_tally.div;
  counts[3] = g_tally.sqrt;
  counts[4] = g_tally.cmp;
}

/* The same count split by part of the right-hand side: parts[4][5] =
 * {derivatives (first, second, mixed), Kreiss-Oliger, pointwise algebra
 * (incl. matter sources), fluid flux divergence} x {add, mul, div, sqrt, cmp}. */
void oracle_flop_count_parts(const int* n, const double* h, const double* x0, const double* params,
                             const double* state, double t, double* parts) {
  Grid g = make_grid(n, h, x0);
  Params P = unpack_params(params);
  Field F{&g, state};
  Pt p{{g.n[0] / 2, g.n[1] / 2, g.n[2] / 2}};
  auto snap = [&](int part) {
    parts[5 * part + 0] = g_tally.add;
    parts[5 * part + 1] = g_tally.mul;
    parts[5 * part + 2] = g_tally.div;
    parts[5 * part + 3] = g_tally.sqrt;
    parts[5 * part + 4] = g_tally.cmp;
    g_tally = Tally{0, 0, 0, 0, 0};
  };
  g_tally = Tally{0, 0, 0, 0, 0};
  Local<Cnt> L;
  gather<Cnt>(F, P, p, L);
  snap(0);
  Cnt out[NFMAX];
  const int nf = P.nf();
  for (int f = 0; f < nf; ++f) {
    if (P.fluid && f >= P.ifl() && f < P.ifl() + 4) continue;
    out[f] = KO<Cnt>(F, f, p, P.sigma);
  }
  snap(1);
  point_algebra<Cnt>(L, P, t, out);
  // the KO terms are added to the algebra's outputs: one addition per field
  for (int f = 0; f < nf; ++f)
    if (!(P.fluid && f >= P.ifl() && f < P.ifl() + 4)) g_tally.add += 1;
  snap(2);
  if (P.fluid) {
    for (int d = 0; d < 3; ++d) {
      Cnt Hp[4];
      kt_face_flux<Cnt>(F, P, p, d, Hp);
      for (int m = 0; m < 4; ++m) out[m] = (Hp[m] - Cnt(0.0)) / Cnt(F.g->h[d]);  // difference + scaling
    }
  }
  snap(3);
}

/* Fixed mesh refinement.  Hierarchy of L levels: per level l, n[3l..3l+2],
 * h[3l..], x0[3l..], origin[3l..], lo[3l..], hi[3l..] (origin, lo, hi are
 * ignored for level 0).  states[l]: level l state, oracle layout. */
void oracle_fmr_step(int L, const int* n, const double* h, const double* x0, const int* origin, const int* lo,
                     const int* hi, const double* params, double* const* states, double t, double dt0) {
  Hier H = make_hier(L, n, h, x0, origin, lo, hi);
  fmr_step(H, unpack_params(params), states, t, dt0);
}

void oracle_fmr_init(int L, const int* n, const double* h, const double* x0, const int* origin, const int* lo,
                     const int* hi, const double* params, const double* id, double* const* states) {
  Hier H = make_hier(L, n, h, x0, origin, lo, hi);
  fmr_init(H, unpack_params(params), id, states);
}

/* Ghost points of level `level` from the parent state `parent` (nf fields). */
void oracle_fmr_prolong(int L, const int* n, const double* h, const double* x0, const int* origin, const int* lo,
                        const int* hi, int level, int nf, const double* parent, double* child) {
  Hier H = make_hier(L, n, h, x0, origin, lo, hi);
  prolong(H, level, nf, parent, child);
}

/* Injection of level `level`'s interior into its parent (nf fields). */
void oracle_fmr_restrict(int L, const int* n, const double* h, const double* x0, const int* origin, const int* lo,
                         const int* hi, int level, int nf, const double* child, double* parent) {
  Hier H = make_hier(L, n, h, x0, origin, lo, hi);
  restrict_to_parent(H, level, nf, child, parent);
}

/* Continuous extension of one RK4 step: out = U_n + dt sum_s b_s(theta) k_s
 * over M values (k = k1..k4 stacked, 4 M values). */
void oracle_rk4_dense(long M, const double* Un, const double* k, double dt, double theta, double* out) {
  const double* ks[4] = {k, k + M, k + 2 * M, k + 3 * M};
  rk4_dense(M, Un, ks, dt, theta, out);
}


/* Initial data from a per-point zeta (one value per point, [k][j][i]); see
 * the collapse-diagnostics section for the map. */
void oracle_init_zeta(const int* n, const double* h, const double* x0, const double* params, const double* zeta,
                      double a0, double* state) {
  Grid g = make_grid(n, h, x0);
  Params P = unpack_params(params);
  std::vector<double> st;
  init_zeta<double>(g, P, zeta, a0, st);
  std::memcpy(state, st.data(), sizeof(double) * st.size());
}

/* zeta_bar = (d state0 / d zeta)^T lam0 for the map of oracle_init_zeta, by a
 * tape whose leaves are the zeta values.  Single-threaded; tiny grids. */
void oracle_init_zeta_vjp(const int* n, const double* h, const double* x0, const double* params,
                          const double* zeta, double a0, const double* lam0, double* zeta_bar) {
  Grid g = make_grid(n, h, x0);
  Params P = unpack_params(params);
  const long N = g.npts();
  g_tape.clear();
  std::vector<AD> z(N);
  for (long m = 0; m < N; ++m) {
    g_tape.push_back(TapeNode{-1, -1, 0.0, 0.0});
    z[m] = AD(zeta[m], m);
  }
  std::vector<AD> st;
  init_zeta<AD>(g, P, z.data(), a0, st);
  std::vector<std::pair<long, double>> seeds;
  for (size_t q = 0; q < st.size(); ++q)
    if (st[q].id >= 0) seeds.push_back({st[q].id, lam0[q]});
  std::vector<double> adj = reverse_sweep(N, seeds);
  for (long m = 0; m < N; ++m) zeta_bar[m] = adj[m];
  g_tape.clear();
  g_tape.shrink_to_fit();
}

/* alpha at the centre grid point (nx/2, ny/2, nz/2). */
double oracle_central_lapse(const int* n, const double* state) {
  const long N = (long)n[0] * n[1] * n[2];
  return state[ALP * N + ((long)(n[2] / 2) * n[1] + n[1] / 2) * n[0] + n[0] / 2];
}

/* Compaction C(r_k), k = 1..kmax, into C[kmax] (equal spacing; fluid on). */
void oracle_compaction(const int* n, const double* h, const double* x0, const double* params, const double* state,
                       int kmax, double* C) {
  Grid g = make_grid(n, h, x0);
  Field F{&g, state};
  compaction<double>(g, unpack_params(params), F, kmax, C);
}

/* lam = cbar d C(r_kstar) / d state (state layout), by a tape over the same
 * function whose leaves are the state entries. */
void oracle_compaction_vjp(const int* n, const double* h, const double* x0, const double* params,
                           const double* state, int kmax, int kstar, double cbar, double* lam) {
  Grid g = make_grid(n, h, x0);
  Params P = unpack_params(params);
  Field F{&g, state};
  const long M = (long)P.nf() * g.npts();
  g_tape.clear();
  for (long m = 0; m < M; ++m) g_tape.push_back(TapeNode{-1, -1, 0.0, 0.0});
  std::vector<AD> C(kmax);
  compaction<AD>(g, P, F, kmax, C.data());
  std::vector<std::pair<long, double>> seeds;
  if (C[kstar - 1].id >= 0) seeds.push_back({C[kstar - 1].id, cbar});
  std::vector<double> adj = reverse_sweep(M, seeds);
  for (long m = 0; m < M; ++m) lam[m] = adj[m];
  g_tape.clear();
  g_tape.shrink_to_fit();
}

}  // extern "C"

// Fixed mesh refinement (section "Statement of need": a fixed set of nested
// refinement levels resolves the collapsing region; the paper's figure of the
// lapse at horizon formation shows the lowest level and two refined ones).
//
// Level 0 is the periodic box.  Level l >= 1 is one box of points with spacing
// h_{l-1}/2 whose every other point lies on a point of level l-1; its points
// outside the interior box [lo, hi) are ghost points (at least 3 layers, the
// Kreiss-Oliger reach).  Along an axis on which level l-1 is periodic, level l
// may be periodic too (lo = 0, hi = n = 2 n_{l-1}, origin 0).
//
// A level is stored as an ordinary grid array (ghost points included) and is
// advanced by the very same stage kernels as a periodic grid: their periodic
// index wrap never reaches an interior point's stencil (reach 3 <= ghost
// width), so interior results are exactly those of the non-periodic level;
// what the stage writes at ghost points is never read, because the ghost
// points of every stage input are set from level l-1 first.
//
// Berger-Oliger subcycling: after each step of level l-1, level l takes two
// steps of half its size, then its interior points that lie on level l-1
// points overwrite those (injection).  Ghost values of each of the child's RK4
// stages come from the parent's step: the continuous extension of order 3 of
// classic RK4, u(theta) = U_n + dt sum_q b_q(theta) k_q, and its theta-
// derivatives at the substep's start give the stage states that RK4 forms
// from a smooth solution (Y_1 = u, Y_2 = u + tau/2 u', Y_3 = Y_2 + tau^2/4 u'',
// Y_4 = u + tau u' + tau^2/2 u'' + tau^3/4 u'''), the stage-consistent
// interpolation of McCorquodale and Colella (2011); then, in space, the
// tensor product of 6-point (degree-5) Lagrange interpolation at half-way
// points and injection at coincident points, applied one axis at a time.
//
// The parent's k_q are not stored: with the stage states U_2 = U_n + dt/2 k_1,
// U_3 = U_n + dt/2 k_2, U_4 = U_n + dt k_3 and U_{n+1} = U_n + dt/6 (k_1 + 2 k_2
// + 2 k_3 + k_4), U_n + dt sum_q beta_q k_q = U_n + w_2 (U_2 - U_n)
// + w_3 (U_3 - U_n) + w_4 (U_4 - U_n) + w_1 (U_{n+1} - U_n) with
// w_2 = 2 beta_1 - 2 beta_4, w_3 = 2 beta_2 - 4 beta_4, w_4 = beta_3 - 2 beta_4,
// w_1 = 6 beta_4.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "host.cuh"

namespace cosmos {
namespace {

#define FCK(expr)                                 \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return cuda_error(e_); \
  } while (0)

// Lagrange weights at a point half-way between the 3rd and 4th of six
// equally spaced nodes (x = -5/2 .. 5/2, evaluated at 0).
__constant__ double W6[6] = {3.0 / 256.0, -25.0 / 256.0, 150.0 / 256.0, 150.0 / 256.0, -25.0 / 256.0, 3.0 / 256.0};

__host__ __device__ inline int floordiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

struct Level {
  cosmos_grid g;
  DevGrid dg;
  int per[3];           // axis periodic
  int origin[3], lo[3], hi[3];
  int blo[3], bn[3];    // parent index box read by this level's ghost interpolation (unwrapped)
  size_t fs;            // field stride
};

struct Hier {
  int L, nf;
  Level lv[COSMOS_FMR_MAX_LEVELS];
};

// first and last parent index of the interpolation taps of child point X2
// (child spacings from parent point 0)
inline void tap_range(int X2, int* first, int* last) {
  if (X2 % 2 == 0) {
    *first = *last = X2 / 2;
  } else {
    const int b = floordiv2(X2);
    *first = b - 2;
    *last = b + 3;
  }
}

int describe(const cosmos_fmr* m, const cosmos_params* p, Hier* H) {
  if (!m || !p) return COSMOS_EINVAL;
  if (m->levels < 1 || m->levels > COSMOS_FMR_MAX_LEVELS) return COSMOS_EINVAL;
  H->L = m->levels;
  H->nf = 24 + 4 * (p->fluid != 0) + 2 * (p->scalar != 0);
  for (int l = 0; l < H->L; ++l) {
    Level& v = H->lv[l];
    v.g = m->grid[l];
    int e = validate(&v.g, p);
    if (e) return e;
    v.dg = make_devgrid(&v.g);
    v.fs = (size_t)v.g.pitch * v.g.ny * v.g.nz;
    const int n[3] = {v.g.nx, v.g.ny, v.g.nz};
    for (int d = 0; d < 3; ++d) {
      if (l == 0) {
        v.per[d] = 1;
        v.origin[d] = 0;
        v.lo[d] = 0;
        v.hi[d] = n[d];
        v.blo[d] = 0;
        v.bn[d] = 0;
        continue;
      }
      const Level& q = H->lv[l - 1];
      const int np[3] = {q.g.nx, q.g.ny, q.g.nz};
      v.origin[d] = m->origin[l][d];
      v.lo[d] = m->lo[l][d];
      v.hi[d] = m->hi[l][d];
      if (2.0 * v.g.h[d] != q.g.h[d]) return COSMOS_EINVAL;  // ratio 2, exactly
      const double x0 = q.g.x0[d] + v.origin[d] * v.g.h[d];
      if (fabs(v.g.x0[d] - x0) > 1e-12 * (fabs(q.g.x0[d]) + np[d] * q.g.h[d])) return COSMOS_EINVAL;
      v.per[d] = q.per[d] && v.lo[d] == 0 && v.hi[d] == n[d] && v.origin[d] == 0 && n[d] == 2 * np[d];
      if (!v.per[d] && (v.lo[d] < 3 || n[d] - v.hi[d] < 3 || v.lo[d] >= v.hi[d])) return COSMOS_EINVAL;
      // taps of every child index 0 .. n-1 (the extremes bound them)
      int f0, l0, f1, l1, f2, l2, f3, l3;
      tap_range(v.origin[d], &f0, &l0);
      tap_range(v.origin[d] + (n[d] > 1 ? 1 : 0), &f1, &l1);
      tap_range(v.origin[d] + n[d] - 1, &f2, &l2);
      tap_range(v.origin[d] + (n[d] > 1 ? n[d] - 2 : 0), &f3, &l3);
      const int first = f0 < f1 ? f0 : f1;
      const int last = l2 > l3 ? l2 : l3;
      if (!q.per[d] && (first < q.lo[d] || last >= q.hi[d])) return COSMOS_EINVAL;  // must read parent interior
      v.blo[d] = first;
      v.bn[d] = last - first + 1;
    }
  }
  return COSMOS_OK;
}

struct WsPlan {
  size_t rk, saved[COSMOS_FMR_MAX_LEVELS], tmp, A, B;  // doubles from ws (saved: 4 states per level with a child)
  size_t rk_bytes, total;                              // bytes
};

size_t al256(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

WsPlan plan_ws(const Hier& H, const cosmos_params* p) {
  WsPlan W;
  memset(&W, 0, sizeof(W));
  size_t rk = 0, box = 0, ax = 0, ay = 0, off = 0;
  for (int l = 0; l < H.L; ++l) {
    const WsLayout a = ws_layout(&H.lv[l].g, p, COSMOS_OP_RK4);
    const WsLayout b = ws_layout(&H.lv[l].g, p, COSMOS_OP_INIT);
    rk = rk > a.total_bytes ? rk : a.total_bytes;
    rk = rk > b.total_bytes ? rk : b.total_bytes;
    if (l > 0) {
      const Level& v = H.lv[l];
      const size_t vb = (size_t)v.bn[0] * v.bn[1] * v.bn[2];
      const size_t va = (size_t)v.g.nx * v.bn[1] * v.bn[2];
      const size_t vy = (size_t)v.g.nx * v.g.ny * v.bn[2];
      box = box > vb ? box : vb;
      ax = ax > va ? ax : va;
      ay = ay > vy ? ay : vy;
    }
  }
  W.rk = 0;
  W.rk_bytes = al256(rk);
  off = W.rk_bytes;
  for (int l = 0; l + 1 < H.L; ++l) {
    W.saved[l] = off / sizeof(double);
    off += 4 * al256(H.nf * H.lv[l].fs * sizeof(double));
  }
  W.tmp = off / sizeof(double);
  off += al256(H.nf * box * sizeof(double));
  W.A = off / sizeof(double);
  off += al256(H.nf * ax * sizeof(double));
  W.B = off / sizeof(double);
  off += al256(H.nf * ay * sizeof(double));
  W.total = off;
  return W;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
struct TimeArgs {
  const double* Un;
  const double* U2;  // null: plain copy of Un
  const double* U3;
  const double* U4;
  const double* U1;
  double w2, w3, w4, w1;
  DevGrid gp;
  int blo[3], bn[3];
  int nf;
  double* tmp;  // [nf][bn2][bn1][bn0]
};

// Parent values over the interpolation box at the requested stage (see top).
__global__ void fmr_time_kernel(const TimeArgs a) {
  const long vol = (long)a.bn[0] * a.bn[1] * a.bn[2];
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= vol) return;
  const int bx = (int)(q % a.bn[0]);
  const int by = (int)((q / a.bn[0]) % a.bn[1]);
  const int bz = (int)(q / ((long)a.bn[0] * a.bn[1]));
  const int i = wrap_index(a.blo[0] + bx, a.gp.nx);
  const int j = wrap_index(a.blo[1] + by, a.gp.ny);
  const int k = wrap_index(a.blo[2] + bz, a.gp.nz);
  const long c = ((long)k * a.gp.ny + j) * a.gp.pitch + i;
  for (int f = 0; f < a.nf; ++f) {
    const long o = f * a.gp.fstride + c;
    const double un = a.Un[o];
    double y = un;
    if (a.U2)
      y = un + a.w2 * (a.U2[o] - un) + a.w3 * (a.U3[o] - un) + a.w4 * (a.U4[o] - un) + a.w1 * (a.U1[o] - un);
    a.tmp[f * vol + q] = y;
  }
}

// Spatial interpolation in three 1D passes over the interpolation box:
// x (parent box -> child x columns), y (-> child x-y planes), then z at the
// ghost points only.  Each output takes 1 tap (coincident) or the 6 Lagrange
// taps (half-way); threads run along x, so every access is contiguous.
struct ProlongArgs {
  DevGrid gc;
  int origin[3], lo[3], hi[3];
  int blo[3], bn[3];
  int nf;
  const double* tmp;  // [nf][bn2][bn1][bn0]   parent values
  double* A;          // [nf][bn2][bn1][nx]    after x
  double* B;          // [nf][bn2][ny][nx]     after y
  double* C;          // child state
};

// value at child position X2 from a line of box values (stride s, box start blo)
__device__ __forceinline__ double interp1(const double* line, long s, int X2, int blo) {
  if ((X2 & 1) == 0) return line[(long)(X2 / 2 - blo) * s];
  const double* q = line + (long)(floordiv2(X2) - 2 - blo) * s;
  return W6[0] * q[0] + W6[1] * q[s] + W6[2] * q[2 * s] + W6[3] * q[3 * s] + W6[4] * q[4 * s] + W6[5] * q[5 * s];
}

__global__ void fmr_prolong_x_kernel(const ProlongArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int by = blockIdx.y * BY + threadIdx.y;
  const int bz = blockIdx.z;
  if (i >= a.gc.nx || by >= a.bn[1]) return;
  for (int f = 0; f < a.nf; ++f) {
    const long row = ((long)f * a.bn[2] + bz) * a.bn[1] + by;
    a.A[row * a.gc.nx + i] = interp1(a.tmp + row * a.bn[0], 1, a.origin[0] + i, a.blo[0]);
  }
}

__global__ void fmr_prolong_y_kernel(const ProlongArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int bz = blockIdx.z;
  if (i >= a.gc.nx || j >= a.gc.ny) return;
  for (int f = 0; f < a.nf; ++f) {
    const long plane = (long)f * a.bn[2] + bz;
    a.B[(plane * a.gc.ny + j) * a.gc.nx + i] =
        interp1(a.A + plane * a.bn[1] * a.gc.nx + i, a.gc.nx, a.origin[1] + j, a.blo[1]);
  }
}

__global__ void fmr_prolong_z_kernel(const ProlongArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.gc.nx || j >= a.gc.ny) return;
  if (i >= a.lo[0] && i < a.hi[0] && j >= a.lo[1] && j < a.hi[1] && k >= a.lo[2] && k < a.hi[2]) return;
  const long c = ((long)k * a.gc.ny + j) * a.gc.pitch + i;
  const long plane = (long)a.gc.ny * a.gc.nx;
  for (int f = 0; f < a.nf; ++f)
    a.C[f * a.gc.fstride + c] =
        interp1(a.B + (long)f * a.bn[2] * plane + (long)j * a.gc.nx + i, plane, a.origin[2] + k, a.blo[2]);
}

struct RestrictArgs {
  DevGrid gc, gp;
  int origin[3], first[3], cnt[3];
  int nf;
  const double* C;
  double* P;
};

// Interior points of a level that lie on parent points overwrite those.
__global__ void fmr_restrict_kernel(const RestrictArgs a) {
  const int mx = blockIdx.x * BX + threadIdx.x;
  const int my = blockIdx.y * BY + threadIdx.y;
  const int mz = blockIdx.z;
  if (mx >= a.cnt[0] || my >= a.cnt[1]) return;
  const int i = a.first[0] + 2 * mx, j = a.first[1] + 2 * my, k = a.first[2] + 2 * mz;
  const int pi = wrap_index((a.origin[0] + i) / 2, a.gp.nx);
  const int pj = wrap_index((a.origin[1] + j) / 2, a.gp.ny);
  const int pk = wrap_index((a.origin[2] + k) / 2, a.gp.nz);
  const long c = ((long)k * a.gc.ny + j) * a.gc.pitch + i;
  const long pc = ((long)pk * a.gp.ny + pj) * a.gp.pitch + pi;
  for (int f = 0; f < a.nf; ++f) a.P[f * a.gp.fstride + pc] = a.C[f * a.gc.fstride + c];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Coefficients beta_q of the ghost value of stage `stage` of a child substep
// of r times the parent's step that starts at theta0 of the parent's step.
void stage_beta(double theta0, int stage, double r, double beta[4]) {
  const double th = theta0, th2 = th * th, th3 = th2 * th;
  const double b[4] = {th - 1.5 * th2 + 2.0 / 3.0 * th3, th2 - 2.0 / 3.0 * th3, th2 - 2.0 / 3.0 * th3,
                       -0.5 * th2 + 2.0 / 3.0 * th3};
  const double db[4] = {1.0 - 3.0 * th + 2.0 * th2, 2.0 * th - 2.0 * th2, 2.0 * th - 2.0 * th2, -th + 2.0 * th2};
  const double d2b[4] = {4.0 * th - 3.0, 2.0 - 4.0 * th, 2.0 - 4.0 * th, 4.0 * th - 1.0};
  const double d3b[4] = {4.0, -4.0, -4.0, 4.0};
  // Y_s = u + e1 tau u' + e2 tau^2 u'' + e3 tau^3 u'''
  static const double e1[4] = {0.0, 0.5, 0.5, 1.0}, e2[4] = {0.0, 0.0, 0.25, 0.5}, e3[4] = {0.0, 0.0, 0.0, 0.25};
  const int s = stage - 1;
  for (int q = 0; q < 4; ++q) beta[q] = b[q] + e1[s] * r * db[q] + e2[s] * r * r * d2b[q] + e3[s] * r * r * r * d3b[q];
}

struct Ctx {
  Hier H;
  const cosmos_params* p;
  double* const* U;
  double* ws;
  WsPlan W;
  cudaStream_t s;
  double* saved(int l, int q) const {
    return ws + W.saved[l] + q * (al256(H.nf * H.lv[l].fs * sizeof(double)) / sizeof(double));
  }
};

int fill_box(const Ctx& c, int l, const TimeArgs& base) {
  const Level& v = c.H.lv[l];
  TimeArgs a = base;
  a.gp = c.H.lv[l - 1].dg;
  for (int d = 0; d < 3; ++d) {
    a.blo[d] = v.blo[d];
    a.bn[d] = v.bn[d];
  }
  a.nf = c.H.nf;
  a.tmp = c.ws + c.W.tmp;
  const long vol = (long)v.bn[0] * v.bn[1] * v.bn[2];
  fmr_time_kernel<<<(unsigned)((vol + 255) / 256), 256, 0, c.s>>>(a);
  FCK(cudaGetLastError());
  return COSMOS_OK;
}

int prolong_into(const Ctx& c, int l, double* X) {
  const Level& v = c.H.lv[l];
  ProlongArgs a;
  a.gc = v.dg;
  for (int d = 0; d < 3; ++d) {
    a.origin[d] = v.origin[d];
    a.lo[d] = v.lo[d];
    a.hi[d] = v.hi[d];
    a.blo[d] = v.blo[d];
    a.bn[d] = v.bn[d];
  }
  a.nf = c.H.nf;
  a.tmp = c.ws + c.W.tmp;
  a.A = c.ws + c.W.A;
  a.B = c.ws + c.W.B;
  a.C = X;
  const dim3 blk(BX, BY);
  fmr_prolong_x_kernel<<<dim3((v.g.nx + BX - 1) / BX, (v.bn[1] + BY - 1) / BY, v.bn[2]), blk, 0, c.s>>>(a);
  FCK(cudaGetLastError());
  fmr_prolong_y_kernel<<<dim3((v.g.nx + BX - 1) / BX, (v.g.ny + BY - 1) / BY, v.bn[2]), blk, 0, c.s>>>(a);
  FCK(cudaGetLastError());
  fmr_prolong_z_kernel<<<point_grid(v.dg), blk, 0, c.s>>>(a);
  FCK(cudaGetLastError());
  return COSMOS_OK;
}

// ghost points of level l from a parent state (no time interpolation)
int fill_plain(const Ctx& c, int l, const double* parent, double* X) {
  TimeArgs a;
  memset(&a, 0, sizeof(a));
  a.Un = parent;
  int e = fill_box(c, l, a);
  return e ? e : prolong_into(c, l, X);
}

// ghost points of level l for RK4 stage `stage` of its substep starting at
// theta0 of level l-1's step (saved stage states of level l-1)
int fill_stage(const Ctx& c, int l, double theta0, int stage, double* X) {
  double beta[4];
  stage_beta(theta0, stage, 0.5, beta);
  TimeArgs a;
  memset(&a, 0, sizeof(a));
  a.Un = c.saved(l - 1, 0);
  a.U2 = c.saved(l - 1, 1);
  a.U3 = c.saved(l - 1, 2);
  a.U4 = c.saved(l - 1, 3);
  a.U1 = c.U[l - 1];
  a.w2 = 2.0 * beta[0] - 2.0 * beta[3];
  a.w3 = 2.0 * beta[1] - 4.0 * beta[3];
  a.w4 = beta[2] - 2.0 * beta[3];
  a.w1 = 6.0 * beta[3];
  int e = fill_box(c, l, a);
  return e ? e : prolong_into(c, l, X);
}

int restrict_level(const Hier& H, int l, const double* C, double* P, cudaStream_t s) {
  const Level& v = H.lv[l];
  RestrictArgs a;
  a.gc = v.dg;
  a.gp = H.lv[l - 1].dg;
  a.nf = H.nf;
  a.C = C;
  a.P = P;
  for (int d = 0; d < 3; ++d) {
    int f = v.lo[d];
    if ((v.origin[d] + f) % 2 != 0) ++f;
    a.origin[d] = v.origin[d];
    a.first[d] = f;
    a.cnt[d] = f < v.hi[d] ? (v.hi[d] - f + 1) / 2 : 0;
  }
  if (a.cnt[0] == 0 || a.cnt[1] == 0 || a.cnt[2] == 0) return COSMOS_OK;
  const dim3 grid((a.cnt[0] + BX - 1) / BX, (a.cnt[1] + BY - 1) / BY, a.cnt[2]);
  fmr_restrict_kernel<<<grid, dim3(BX, BY), 0, s>>>(a);
  FCK(cudaGetLastError());
  return COSMOS_OK;
}

// One step of level l from t (starting at theta0 of level l-1's step), then,
// when level l+1 exists, its two substeps and the injection.
int advance(const Ctx& c, int l, double t, double dt, double theta0) {
  const Level& v = c.H.lv[l];
  const cosmos_grid* g = &v.g;
  const WsLayout W = ws_layout(g, c.p, COSMOS_OP_RK4);
  double* w = c.ws + c.W.rk;
  double* acc = w + W.acc;
  double* U = c.U[l];
  const bool child = l + 1 < c.H.L;
  double* Y2 = child ? c.saved(l, 1) : w + W.stageA;
  double* Y3 = child ? c.saved(l, 2) : w + W.stageB;
  double* Y4 = child ? c.saved(l, 3) : w + W.stageA;
  const double dt2 = 0.5 * dt;
  // on a refined level the algebra pass skips the ghost z-planes: whatever it
  // would write there is replaced from the parent before it is read
  const int k_lo = v.lo[2], k_cnt = v.hi[2] - v.lo[2];
  int e;
  if (l > 0 && (e = fill_stage(c, l, theta0, 1, U))) return e;
  if (child) FCK(cudaMemcpyAsync(c.saved(l, 0), U, c.H.nf * v.fs * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
  if ((e = run_stage(g, c.p, MODE_S1, U, U, Y2, acc, t, dt2, 2.0, w, W, c.s, 7, 0, 0, k_lo, k_cnt))) return e;
  if (l > 0 && (e = fill_stage(c, l, theta0, 2, Y2))) return e;
  if ((e = run_stage(g, c.p, MODE_S23, Y2, U, Y3, acc, t + dt2, dt2, 2.0, w, W, c.s, 7, 0, 0, k_lo, k_cnt))) return e;
  if (l > 0 && (e = fill_stage(c, l, theta0, 3, Y3))) return e;
  if ((e = run_stage(g, c.p, MODE_S23, Y3, U, Y4, acc, t + dt2, dt, 2.0, w, W, c.s, 7, 0, 0, k_lo, k_cnt))) return e;
  if (l > 0 && (e = fill_stage(c, l, theta0, 4, Y4))) return e;
  if ((e = run_stage(g, c.p, MODE_S4, Y4, U, nullptr, acc, t + dt, dt / 6.0, 2.0, w, W, c.s, 7, 0, 0, k_lo, k_cnt)))
    return e;
  if (child) {
    if ((e = advance(c, l + 1, t, dt2, 0.0))) return e;
    if ((e = advance(c, l + 1, t + dt2, dt2, 0.5))) return e;
    if ((e = restrict_level(c.H, l + 1, c.U[l + 1], U, c.s))) return e;
  }
  return COSMOS_OK;
}

int check_states(const Hier& H, double* const* states) {
  if (!states) return COSMOS_EINVAL;
  for (int l = 0; l < H.L; ++l) {
    if (!states[l]) return COSMOS_EINVAL;
    if (!aligned16(states[l])) return COSMOS_EALIGN;
    for (int q = 0; q < l; ++q)
      if (states[q] == states[l]) return COSMOS_EINVAL;
  }
  return COSMOS_OK;
}

int prepare(const cosmos_fmr* m, const cosmos_params* p, void* ws, size_t ws_bytes, cudaStream_t s, Ctx* c) {
  int e = describe(m, p, &c->H);
  if (e) return e;
  c->p = p;
  c->W = plan_ws(c->H, p);
  if (!ws) return COSMOS_EINVAL;
  if (ws_bytes < c->W.total) return COSMOS_EWORKSPACE;
  if (((uintptr_t)ws & 255u) != 0) return COSMOS_EALIGN;
  c->ws = (double*)ws;
  c->s = s;
  return COSMOS_OK;
}

}  // namespace
}  // namespace cosmos

using namespace cosmos;

extern "C" {

size_t cosmos_fmr_workspace_bytes(const cosmos_fmr* m, const cosmos_params* p) {
  Hier H;
  if (describe(m, p, &H) != COSMOS_OK) return 0;
  return plan_ws(H, p).total;
}

int cosmos_fmr_init(const cosmos_fmr* m, const cosmos_params* p, const cosmos_id* id, double* const* states,
                    void* ws, size_t ws_bytes, void* stream) {
  Ctx c;
  int e = prepare(m, p, ws, ws_bytes, (cudaStream_t)stream, &c);
  if (e) return e;
  if ((e = check_states(c.H, states))) return e;
  c.U = states;
  const double Lx = c.H.lv[0].g.nx * c.H.lv[0].g.h[0];  // the gauge wave's wavelength is the periodic box
  for (int l = 0; l < c.H.L; ++l)
    if ((e = init_grid(&c.H.lv[l].g, p, id, states[l], c.ws + c.W.rk, c.W.rk_bytes, c.s, Lx))) return e;
  for (int l = c.H.L - 1; l >= 1; --l)
    if ((e = restrict_level(c.H, l, states[l], states[l - 1], c.s))) return e;
  for (int l = 1; l < c.H.L; ++l)
    if ((e = fill_plain(c, l, states[l - 1], states[l]))) return e;
  return COSMOS_OK;
}

int cosmos_fmr_step(const cosmos_fmr* m, const cosmos_params* p, double* const* states, double t, double dt0,
                    void* ws, size_t ws_bytes, void* stream) {
  Ctx c;
  int e = prepare(m, p, ws, ws_bytes, (cudaStream_t)stream, &c);
  if (e) return e;
  if ((e = check_states(c.H, states))) return e;
  if (!(dt0 > 0.0) || !isfinite(dt0)) return COSMOS_EINVAL;
  c.U = states;
  if ((e = advance(c, 0, t, dt0, 0.0))) return e;
  for (int l = 1; l < c.H.L; ++l)
    if ((e = fill_plain(c, l, states[l - 1], states[l]))) return e;
  return COSMOS_OK;
}

int cosmos_fmr_prolong(const cosmos_fmr* m, const cosmos_params* p, int level, const double* parent, double* child,
                       void* ws, size_t ws_bytes, void* stream) {
  Ctx c;
  int e = prepare(m, p, ws, ws_bytes, (cudaStream_t)stream, &c);
  if (e) return e;
  if (level < 1 || level >= c.H.L || !parent || !child || parent == child) return COSMOS_EINVAL;
  if (!aligned16(parent) || !aligned16(child)) return COSMOS_EALIGN;
  return fill_plain(c, level, parent, child);
}

int cosmos_fmr_restrict(const cosmos_fmr* m, const cosmos_params* p, int level, const double* child, double* parent,
                        void* stream) {
  Hier H;
  int e = describe(m, p, &H);
  if (e) return e;
  if (level < 1 || level >= H.L || !parent || !child || parent == child) return COSMOS_EINVAL;
  if (!aligned16(parent) || !aligned16(child)) return COSMOS_EALIGN;
  return restrict_level(H, level, child, parent, (cudaStream_t)stream);
}

}  // extern "C"

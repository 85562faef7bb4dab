// Reverse mode of the evolution (declared in include/cosmos.h): the
// vector-Jacobian product of the right-hand side, the adjoint of one RK4
// step, initial data from a per-point curvature perturbation zeta and its
// reverse, and the compaction diagnostic with its reverse.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "adjoint_kernel.cuh"

namespace cosmos {

constexpr int kAlphaField = 17;  // the lapse's place in the state's field order

static size_t a256(size_t doubles) { return ((doubles * 8 + 255) & ~(size_t)255) / 8; }

struct AdjLayout {
  size_t U2, U3, U4, KB, KB2, LAM, Dfw, CB, prim, flux, vprim, FC, VF, CB10, limbs, expo, total_bytes;
};

static int nin_of(const cosmos_params* p) {
  if (p->fluid) return p->scalar ? alg_fluid_scalar::NIN : alg_fluid::NIN;
  return p->scalar ? alg_scalar::NIN : alg_vac::NIN;
}

// Forward stage and reverse launchers of the matter variant.
static cudaError_t launch_stage_for(const cosmos_params* p, const StageArgs& a, int mode, cudaStream_t s) {
  if (p->fluid) return p->scalar ? launch_stage_fluid_scalar(a, mode, s) : launch_stage_fluid(a, mode, s);
  return p->scalar ? launch_stage_scalar(a, mode, s) : launch_stage_vac(a, mode, s);
}

static cudaError_t launch_vjp_for(const cosmos_params* p, const VjpArgs& a, cudaStream_t s) {
  if (p->fluid) return p->scalar ? launch_vjp_fluid_scalar(a, s) : launch_vjp_fluid(a, s);
  return p->scalar ? launch_vjp_scalar(a, s) : launch_vjp_vac(a, s);
}

static AdjLayout adj_layout(const cosmos_grid* g, const cosmos_params* p, int op) {
  const size_t fs = (size_t)g->pitch * g->ny * g->nz;
  const int nf = 24 + 4 * p->fluid + 2 * p->scalar;
  AdjLayout L;
  memset(&L, 0, sizeof(L));
  size_t off = 0;
  auto take = [&](size_t doubles) {
    size_t o = off;
    off += a256(doubles);
    return o;
  };
  if (op == COSMOS_OP_ADJOINT) {
    L.U2 = take(nf * fs);
    L.U3 = take(nf * fs);
    L.U4 = take(nf * fs);
    L.KB = take(nf * fs);
    L.KB2 = take(nf * fs);
    L.LAM = take(nf * fs);
    L.Dfw = take((size_t)nder(p->scalar) * fs);
  }
  if (op == COSMOS_OP_VJP) L.Dfw = take((size_t)nder(p->scalar) * fs);  // derivative pass of the linearisation point
  if (op == COSMOS_OP_ADJOINT || op == COSMOS_OP_VJP) {
    // limb copy for the integer derivative pass (the forward stages and the
    // linearisation points use the same derivative pass as cosmos_rk4_step)
    const int nslot = 24 + 2 * p->scalar;
    L.limbs = take((size_t)nslot * fs);
    L.expo = take(((size_t)nslot + 1) / 2);
    L.CB = take(nin_of(p) * fs);
    if (p->fluid) {
      L.prim = take(4 * fs);
      L.flux = take(12 * fs);
      L.vprim = take(4 * fs);
      L.FC = take(102 * fs);
      L.VF = take(nf * fs);
    }
  }
  if (op == COSMOS_OP_INIT_VJP) L.CB10 = take(10 * fs);
  L.total_bytes = off * 8;
  return L;
}

static int check_adj(const cosmos_grid* g, const cosmos_params* p) {
  const int e = validate(g, p);
  if (e) return e;
  return COSMOS_OK;
}

static int check_ws_adj(size_t need, void* ws, size_t ws_bytes) {
  if (need == 0) return COSMOS_OK;
  if (!ws) return COSMOS_EINVAL;
  if (ws_bytes < need) return COSMOS_EWORKSPACE;
  if ((uintptr_t)ws & 255u) return COSMOS_EALIGN;
  return COSMOS_OK;
}

// Limb copy of every derivative field of U for the integer derivative pass.
static cudaError_t limbs_of(const cosmos_params* p, const DevGrid& g, const double* U, double* ws, const AdjLayout& L,
                            StageArgs& a, cudaStream_t s) {
  const int nslot = 24 + 2 * p->scalar;
  a.L = (const long long*)(ws + L.limbs);
  a.E = (const int*)(ws + L.expo);
  return launch_limbs(g, U, p->fluid, 0, nslot, (int*)(ws + L.expo), (long long*)(ws + L.limbs), s);
}

static FluidParams fparams(double w) {
  FluidParams f;
  f.w = w;
  f.sqrt_w = sqrt(w);
  return f;
}

// lam += (dF/dU at U, time t)^T W;  knext = a_lam lam0 + a_v v (if knext)
static cudaError_t vjp_once(const cosmos_grid* g, const cosmos_params* p, const double* U, double t, const double* W,
                            double* lam, const double* lam0, double* knext, double a_lam, double a_v, double* ws,
                            const AdjLayout& L, cudaStream_t s) {
  VjpArgs a;
  memset(&a, 0, sizeof(a));
  a.g = make_devgrid(g);
  a.c = make_coef(g, p->ko_sigma);
  a.ap = algebra_params(p, t);
  a.fp = fparams(p->w);
  a.U = U;
  a.W = W;
  a.CB = ws + L.CB;
  a.lam = lam;
  a.lam0 = lam0;
  a.knext = knext;
  a.a_lam = a_lam;
  a.a_v = a_v;
  // finite differences of U (the forward inputs of the algebra) into D; the
  // forward stages of an adjoint step have all run before the first vjp_once
  StageArgs d;
  memset(&d, 0, sizeof(d));
  d.g = a.g;
  d.c = a.c;
  d.U = U;
  d.D = ws + L.Dfw;
  d.skip_ko = 1;
  a.D = d.D;
  {
    cudaError_t e = limbs_of(p, d.g, U, ws, L, d, s);
    if (e == cudaSuccess) e = launch_stage_for(p, d, -1, s);
    if (e != cudaSuccess) return e;
  }
  if (p->fluid) {
    double* vp = ws + L.vprim;
    cudaError_t e = launch_fluid_prim(a.g, U, vp, p->w, s);
    if (e != cudaSuccess) return e;
    a.prim = vp;
    a.FC = ws + L.FC;
    a.VF = ws + L.VF;
  }
  return launch_vjp_for(p, a, s);
}

__global__ void scale_copy(const double* __restrict__ x, double a, double* __restrict__ y, long n) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    y[q] = a * x[q];
}

static cudaError_t launch_scale_copy(const double* x, double a, double* y, long n, cudaStream_t s) {
  const int blocks = (int)std::min<long>((n + 255) / 256, 152L * 16);
  scale_copy<<<blocks, 256, 0, s>>>(x, a, y, n);
  return cudaGetLastError();
}

// One forward stage into `out` (= U_n + cdt F(U_s, ts)) using the stage kernel.
static cudaError_t fwd_stage(const cosmos_grid* g, const cosmos_params* p, const double* U_s, const double* U_n,
                             double* out, double* acc, double ts, double cdt, double* ws, const AdjLayout& L,
                             cudaStream_t s) {
  StageArgs a;
  memset(&a, 0, sizeof(a));
  a.g = make_devgrid(g);
  a.c = make_coef(g, p->ko_sigma);
  a.ap = algebra_params(p, ts);
  a.U = U_s;
  a.U0 = U_n;
  a.out = out;
  a.acc = acc;
  a.cdt = cdt;
  a.bk = 2.0;
  a.D = ws + L.Dfw;
  if (p->fluid) {
    cudaError_t e = launch_fluid_prim(a.g, U_s, ws + L.prim, p->w, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_fluid_flux(a.g, U_s, ws + L.prim, ws + L.flux, p->w, 24, s)) != cudaSuccess) return e;
    a.prim = ws + L.prim;
    a.flux = ws + L.flux;
  }
  const cudaError_t e = limbs_of(p, a.g, U_s, ws, L, a, s);
  if (e != cudaSuccess) return e;
  return launch_stage_for(p, a, MODE_S1, s);
}

// Compaction: per-block partial histograms over shells k = floor(sqrt(m)) + 1,
// m = di^2 + dj^2 + dk^2 (distance to the centre point in grid units), of
// tau~ = sqrt(gamma) E and sqrt(gamma) = chi^{-3/2}; bin kmax + 1 collects the rest.
__global__ void compaction_partials(const DevGrid g, const double* __restrict__ U, int ic, int jc, int kc, int kmax,
                                    double* __restrict__ part) {
  __shared__ int bins[BX * BY];
  __shared__ double tv[BX * BY], sv[BX * BY];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  bins[tid] = -1;
  if (i < g.nx && j < g.ny) {
    const long c = ((long)k * g.ny + j) * g.pitch + i;
    const double chi = U[c];
    tv[tid] = U[24 * g.fstride + c];
    sv[tid] = 1.0 / (chi * sqrt(chi));
    const long di = i - ic, dj = j - jc, dk = k - kc;
    const long m = di * di + dj * dj + dk * dk;
    long r = (long)sqrt((double)m);
    while (r * r > m) --r;
    while ((r + 1) * (r + 1) <= m) ++r;
    bins[tid] = (int)(r + 1 < kmax + 1 ? r + 1 : kmax + 1);
  }
  __syncthreads();
  // one thread per bin sums the block's entries in thread order (deterministic)
  const int nb = kmax + 2;
  const long b = ((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  for (int q = tid; q < nb; q += BX * BY) {
    double st = 0.0, ss = 0.0;
    for (int t = 0; t < BX * BY; ++t)
      if (bins[t] == q) {
        st += tv[t];
        ss += sv[t];
      }
    part[b * 2 * nb + 2 * q] = st;
    part[b * 2 * nb + 2 * q + 1] = ss;
  }
}

__global__ void compaction_reduce(const double* __restrict__ part, long nblocks, int width,
                                  double* __restrict__ out) {
  for (int q = threadIdx.x; q < width; q += blockDim.x) {
    double s = 0.0;
    for (long b = 0; b < nblocks; ++b) s += part[b * width + q];
    out[q] = s;
  }
}

// chi at the 6 axis points at distance k, k = 1..kmax: out[6 (k-1) + a]
__global__ void axis_gather(const DevGrid g, const double* __restrict__ U, int ic, int jc, int kc, int kmax,
                            double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 6 * kmax) return;
  const int k = t / 6 + 1, a = t % 6;
  int i = ic, j = jc, z = kc;
  const int sgn = (a & 1) ? -1 : 1;
  if (a < 2) i += sgn * k;
  else if (a < 4) j += sgn * k;
  else z += sgn * k;
  out[t] = U[((long)z * g.ny + j) * g.pitch + i];
}

// Reverse of the peak compaction C_k* = 2 dM/R:  writes the state cotangent.
struct CompVjp {
  DevGrid g;
  int ic, jc, kc, kstar, nf;
  double h3, cbar, R, C, V, Vall, Ebar, rstar;
};

__global__ void compaction_vjp_kernel(const CompVjp q, const double* __restrict__ U, double* __restrict__ lam) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= q.g.nx || j >= q.g.ny) return;
  const long c = ((long)k * q.g.ny + j) * q.g.pitch + i;
  const long fs = q.g.fstride;
  const long di = i - q.ic, dj = j - q.jc, dk = k - q.kc;
  const long m = di * di + dj * dj + dk * dk;
  const double in = (m < (long)q.kstar * q.kstar) ? 1.0 : 0.0;
  const double chi = U[c];
  // dM = h^3 (S_k - Ebar V_k), Ebar = S_all / V_all;  C = 2 dM / R
  const double tau_bar = q.cbar * 2.0 * q.h3 / q.R * (in - q.V / q.Vall);
  const double sg_bar = q.cbar * 2.0 * q.h3 / q.R * q.Ebar * (q.V / q.Vall - in);
  double chi_bar = sg_bar * (-1.5) / (chi * chi * sqrt(chi));
  // R = r* mean_6(chi^{-1/2}) over the axis points at distance k*
  const bool axis = (m == (long)q.kstar * q.kstar) && ((di == 0) + (dj == 0) + (dk == 0) == 2);
  if (axis) chi_bar += q.cbar * (-q.C / q.R) * q.rstar / 6.0 * (-0.5) / (chi * sqrt(chi));
  for (int f = 0; f < q.nf; ++f) lam[f * fs + c] = 0.0;
  lam[c] = chi_bar;
  lam[24 * fs + c] = tau_bar;
}

// Central lapse of one time level: series[index] = alpha at the centre point.
__global__ void central_lapse_kernel(const double* __restrict__ U, long idx, double* __restrict__ series, int index) {
  series[index] = U[idx];
}

// Reverse of the central-lapse read: lam[idx] += abar.
__global__ void central_lapse_vjp_kernel(double* __restrict__ lam, long idx, double abar) { lam[idx] += abar; }

// (minimum, first index attaining it) of v[0 .. count-1] by one warp: lane l
// scans l, l + 32, ... keeping the first strict minimum, then the lanes are
// merged pairwise preferring the smaller value and, on equal values, the
// smaller index.  A NaN never wins against a number.  Deterministic.
__global__ void series_argmin_kernel(const double* __restrict__ v, int count, double* __restrict__ out) {
  const int lane = threadIdx.x;
  double best = NAN;
  int bi = count;  // "none yet"
  for (int q = lane; q < count; q += 32) {
    const double x = v[q];
    if (bi == count || x < best || (isnan(best) && !isnan(x))) {
      best = x;
      bi = q;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    const bool take = oi < count && (bi == count || ob < best || (ob == best && oi < bi) ||
                                     (isnan(best) && !isnan(ob)) || (isnan(best) && isnan(ob) && oi < bi));
    if (take) {
      best = ob;
      bi = oi;
    }
  }
  if (lane == 0) {
    out[0] = best;
    out[1] = (double)bi;
  }
}

__global__ void init_zeta_metric(const DevGrid g, const double* __restrict__ zeta, double a0, double H0, int nf,
                                 double* __restrict__ U) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long c = ((long)k * g.ny + j) * g.pitch + i;
  const long fs = g.fstride;
  for (int f = 0; f < nf; ++f) U[f * fs + c] = 0.0;
  U[c] = exp(-2.0 * zeta[c]) / (a0 * a0);
  U[1 * fs + c] = U[4 * fs + c] = U[6 * fs + c] = 1.0;
  U[7 * fs + c] = -3.0 * H0;
  U[17 * fs + c] = 1.0;
}

__global__ void init_zeta_tau(const DevGrid g, const double* __restrict__ hm, double* __restrict__ U) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long c = ((long)k * g.ny + j) * g.pitch + i;
  const double chi = U[c];
  U[24 * g.fstride + c] = hm[c] / (16.0 * PI) / (chi * sqrt(chi));
}

}  // namespace cosmos

using namespace cosmos;

extern "C" {

size_t cosmos_adjoint_workspace_bytes(const cosmos_grid* g, const cosmos_params* p, int op) {
  if (check_adj(g, p) != COSMOS_OK) return 0;
  if (op == COSMOS_OP_INIT_VJP) {
    const size_t fs = (size_t)g->pitch * g->ny * g->nz;
    return ((10 * fs * 8 + 255) & ~(size_t)255) + cosmos_workspace_bytes(g, p, COSMOS_OP_INIT);
  }
  if (op == COSMOS_OP_DIAG) {
    const dim3 b = point_grid(make_devgrid(g));
    const long nb = (long)b.x * b.y * b.z;
    const int kmax = std::min(std::min(g->nx, g->ny), g->nz) / 2;
    return (size_t)(nb * 2 * (kmax + 2) + 2 * (kmax + 2) + 6 * kmax + 64) * 8;
  }
  return adj_layout(g, p, op).total_bytes;
}

int cosmos_rhs_vjp(const cosmos_grid* g, const cosmos_params* p, const double* U, const double* w, double* v,
                   double t, void* ws, size_t ws_bytes, void* stream) {
  int e = check_adj(g, p);
  if (e) return e;
  if (!U || !w || !v || v == U || v == w) return COSMOS_EINVAL;
  const AdjLayout L = adj_layout(g, p, COSMOS_OP_VJP);
  if ((e = check_ws_adj(L.total_bytes, ws, ws_bytes))) return e;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = cosmos_field_stride(g) * (size_t)cosmos_nfields(p);
  if (cudaMemsetAsync(v, 0, n * sizeof(double), s) != cudaSuccess) return COSMOS_ECUDA;
  if (vjp_once(g, p, U, t, w, v, nullptr, nullptr, 0.0, 0.0, (double*)ws, L, s) != cudaSuccess) return COSMOS_ECUDA;
  return COSMOS_OK;
}

// Reverse sweep of one RK4 step given its stage states U2, U3, U4 (U_1 = U_n).
static int adjoint_sweep(const cosmos_grid* g, const cosmos_params* p, const double* U_n, const double* U2,
                         const double* U3, const double* U4, const double* lam_np1, double* lam_n, double t,
                         double dt, double* w, const AdjLayout& L, cudaStream_t s) {
  const long n = (long)cosmos_field_stride(g) * cosmos_nfields(p);
  double *KB = w + L.KB, *KB2 = w + L.KB2, *LAM = w + L.LAM;
  const double dt2 = 0.5 * dt;
  // lam_n = lam + sum_s (dF/dU at U_s)^T kbar_s
  if (cudaMemcpyAsync(LAM, lam_np1, n * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return COSMOS_ECUDA;
  if (lam_n != lam_np1 &&
      cudaMemcpyAsync(lam_n, lam_np1, n * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return COSMOS_ECUDA;
  if (launch_scale_copy(LAM, dt / 6.0, KB, n, s) != cudaSuccess) return COSMOS_ECUDA;  // kbar4
  if (vjp_once(g, p, U4, t + dt, KB, lam_n, LAM, KB2, dt / 3.0, dt, w, L, s) != cudaSuccess)   // -> kbar3
    return COSMOS_ECUDA;
  if (vjp_once(g, p, U3, t + dt2, KB2, lam_n, LAM, KB, dt / 3.0, dt2, w, L, s) != cudaSuccess)  // -> kbar2
    return COSMOS_ECUDA;
  if (vjp_once(g, p, U2, t + dt2, KB, lam_n, LAM, KB2, dt / 6.0, dt2, w, L, s) != cudaSuccess)  // -> kbar1
    return COSMOS_ECUDA;
  if (vjp_once(g, p, U_n, t, KB2, lam_n, LAM, nullptr, 0.0, 0.0, w, L, s) != cudaSuccess) return COSMOS_ECUDA;
  return COSMOS_OK;
}

int cosmos_adjoint_step(const cosmos_grid* g, const cosmos_params* p, const double* U_n, const double* lam_np1,
                        double* lam_n, double t, double dt, void* ws, size_t ws_bytes, void* stream) {
  int e = check_adj(g, p);
  if (e) return e;
  if (!U_n || !lam_np1 || !lam_n || lam_n == U_n) return COSMOS_EINVAL;
  const AdjLayout L = adj_layout(g, p, COSMOS_OP_ADJOINT);
  if ((e = check_ws_adj(L.total_bytes, ws, ws_bytes))) return e;
  cudaStream_t s = (cudaStream_t)stream;
  double* w = (double*)ws;
  double *U2 = w + L.U2, *U3 = w + L.U3, *U4 = w + L.U4, *KB = w + L.KB;
  const double dt2 = 0.5 * dt;
  // forward stage states (the same sums as cosmos_rk4_step); KB is scratch here
  if (fwd_stage(g, p, U_n, U_n, U2, KB, t, dt2, w, L, s) != cudaSuccess ||
      fwd_stage(g, p, U2, U_n, U3, KB, t + dt2, dt2, w, L, s) != cudaSuccess ||
      fwd_stage(g, p, U3, U_n, U4, KB, t + dt2, dt, w, L, s) != cudaSuccess)
    return COSMOS_ECUDA;
  return adjoint_sweep(g, p, U_n, U2, U3, U4, lam_np1, lam_n, t, dt, w, L, s);
}

int cosmos_adjoint_step_stages(const cosmos_grid* g, const cosmos_params* p, const double* U_n, const double* U2,
                               const double* U3, const double* U4, const double* lam_np1, double* lam_n, double t,
                               double dt, void* ws, size_t ws_bytes, void* stream) {
  int e = check_adj(g, p);
  if (e) return e;
  if (!U_n || !U2 || !U3 || !U4 || !lam_np1 || !lam_n) return COSMOS_EINVAL;
  if (lam_n == U_n || lam_n == U2 || lam_n == U3 || lam_n == U4) return COSMOS_EINVAL;
  const AdjLayout L = adj_layout(g, p, COSMOS_OP_ADJOINT);
  if ((e = check_ws_adj(L.total_bytes, ws, ws_bytes))) return e;
  return adjoint_sweep(g, p, U_n, U2, U3, U4, lam_np1, lam_n, t, dt, (double*)ws, L, (cudaStream_t)stream);
}

int cosmos_init_zeta(const cosmos_grid* g, const cosmos_params* p, const double* zeta, double a0, double* state,
                     void* ws, size_t ws_bytes, void* stream) {
  int e = check_adj(g, p);
  if (e) return e;
  if (!zeta || !state || !(a0 > 0.0)) return COSMOS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const DevGrid dg = make_devgrid(g);
  init_zeta_metric<<<point_grid(dg), dim3(BX, BY), 0, s>>>(dg, zeta, a0, p->H0, cosmos_nfields(p), state);
  if (cudaGetLastError() != cudaSuccess) return COSMOS_ECUDA;
  if (!p->fluid) return COSMOS_OK;
  const size_t need = cosmos_workspace_bytes(g, p, COSMOS_OP_INIT);
  if ((e = check_ws_adj(need, ws, ws_bytes))) return e;
  // H_vacuum of the metric just written, then tau~ = H/(16 pi) chi^{-3/2}
  const size_t fs = (size_t)dg.fstride;
  double* hm = (double*)ws;
  double* partial = hm + a256(4 * fs);
  ConstraintArgs c;
  memset(&c, 0, sizeof(c));
  c.g = dg;
  c.c = make_coef(g, 0.0);
  cosmos_params pv = *p;
  pv.fluid = 0;
  c.ap = algebra_params(&pv, 0.0);
  c.U = state;
  c.hm = hm;
  c.partial = partial;
  if (launch_constraints_vac(c, s) != cudaSuccess) return COSMOS_ECUDA;
  init_zeta_tau<<<point_grid(dg), dim3(BX, BY), 0, s>>>(dg, hm, state);
  return cudaGetLastError() == cudaSuccess ? COSMOS_OK : COSMOS_ECUDA;
}

int cosmos_init_zeta_vjp(const cosmos_grid* g, const cosmos_params* p, const double* state0, const double* lam0,
                         double* zeta_bar, void* ws, size_t ws_bytes, void* stream) {
  int e = check_adj(g, p);
  if (e) return e;
  if (!state0 || !lam0 || !zeta_bar) return COSMOS_EINVAL;
  const size_t fs = cosmos_field_stride(g);
  const size_t need = (10 * fs * 8 + 255) & ~(size_t)255;
  if ((e = check_ws_adj(need, ws, ws_bytes))) return e;
  const DevGrid dg = make_devgrid(g);
  cosmos_params pv = *p;
  pv.fluid = 0;
  const cudaError_t ce = launch_init_zeta_vjp(dg, make_coef(g, 0.0), algebra_params(&pv, 0.0), state0, lam0,
                                              (double*)ws, p->fluid, zeta_bar, (cudaStream_t)stream);
  return ce == cudaSuccess ? COSMOS_OK : COSMOS_ECUDA;
}

int cosmos_compaction(const cosmos_grid* g, const cosmos_params* p, const double* state, double* C_host, int kmax,
                      double* aux_host, void* ws, size_t ws_bytes, void* stream) {
  int e = check_adj(g, p);
  if (e) return e;
  if (!p->fluid || !state || !C_host || !aux_host) return COSMOS_EINVAL;
  const int kcap = std::min(std::min(g->nx, g->ny), g->nz) / 2;
  if (kmax < 1 || kmax > kcap - 1) return COSMOS_EINVAL;
  const DevGrid dg = make_devgrid(g);
  const dim3 b = point_grid(dg);
  const long nb = (long)b.x * b.y * b.z;
  const int width = 2 * (kmax + 2);
  const size_t need = (size_t)(nb * width + width + 6 * kmax) * 8;
  if ((e = check_ws_adj(need, ws, ws_bytes))) return e;
  cudaStream_t s = (cudaStream_t)stream;
  double* part = (double*)ws;
  double* sums = part + nb * width;
  double* axis = sums + width;
  const int ic = g->nx / 2, jc = g->ny / 2, kc = g->nz / 2;
  compaction_partials<<<b, dim3(BX, BY), 0, s>>>(dg, state, ic, jc, kc, kmax, part);
  compaction_reduce<<<1, 128, 0, s>>>(part, nb, width, sums);
  axis_gather<<<(6 * kmax + 127) / 128, 128, 0, s>>>(dg, state, ic, jc, kc, kmax, axis);
  if (cudaGetLastError() != cudaSuccess) return COSMOS_ECUDA;
  std::vector<double> hs(width), ha(6 * kmax);
  if (cudaMemcpyAsync(hs.data(), sums, width * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(ha.data(), axis, 6 * kmax * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return COSMOS_ECUDA;
  // cumulative shells k = 1..kmax, totals over the whole box
  double S_all = 0.0, V_all = 0.0;
  for (int q = 0; q < kmax + 2; ++q) {
    S_all += hs[2 * q];
    V_all += hs[2 * q + 1];
  }
  const double Ebar = S_all / V_all;
  const double h3 = g->h[0] * g->h[1] * g->h[2];
  double S = 0.0, V = 0.0;
  for (int k = 1; k <= kmax; ++k) {
    S += hs[2 * k];
    V += hs[2 * k + 1];
    double A = 0.0;
    for (int a = 0; a < 6; ++a) A += 1.0 / sqrt(ha[6 * (k - 1) + a]);
    A /= 6.0;
    const double R = k * g->h[0] * A;
    const double dM = h3 * (S - Ebar * V);
    C_host[k - 1] = 2.0 * dM / R;
    aux_host[4 * (k - 1) + 0] = S;
    aux_host[4 * (k - 1) + 1] = V;
    aux_host[4 * (k - 1) + 2] = R;
    aux_host[4 * (k - 1) + 3] = dM;
  }
  aux_host[4 * kmax + 0] = S_all;
  aux_host[4 * kmax + 1] = V_all;
  return COSMOS_OK;
}

int cosmos_central_lapse(const cosmos_grid* g, const cosmos_params* p, const double* state, double* series,
                         int index, void* stream) {
  int e = check_adj(g, p);
  if (e) return e;
  if (!state || !series || index < 0) return COSMOS_EINVAL;
  const long idx = (long)kAlphaField * cosmos_field_stride(g) + ((long)(g->nz / 2) * g->ny + g->ny / 2) * g->pitch + g->nx / 2;
  central_lapse_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(state, idx, series, index);
  return cudaGetLastError() == cudaSuccess ? COSMOS_OK : COSMOS_ECUDA;
}

int cosmos_central_lapse_vjp(const cosmos_grid* g, const cosmos_params* p, double abar, double* lam, void* stream) {
  int e = check_adj(g, p);
  if (e) return e;
  if (!lam) return COSMOS_EINVAL;
  const long idx = (long)kAlphaField * cosmos_field_stride(g) + ((long)(g->nz / 2) * g->ny + g->ny / 2) * g->pitch + g->nx / 2;
  central_lapse_vjp_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(lam, idx, abar);
  return cudaGetLastError() == cudaSuccess ? COSMOS_OK : COSMOS_ECUDA;
}

int cosmos_series_argmin(const double* series, int count, double* result, void* stream) {
  if (!series || !result || count < 1) return COSMOS_EINVAL;
  series_argmin_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(series, count, result);
  return cudaGetLastError() == cudaSuccess ? COSMOS_OK : COSMOS_ECUDA;
}

int cosmos_compaction_vjp(const cosmos_grid* g, const cosmos_params* p, const double* state, int kstar, int kmax,
                          const double* aux_host, double cbar, double* lam, void* stream) {
  int e = check_adj(g, p);
  if (e) return e;
  if (!p->fluid || !state || !lam || !aux_host || kstar < 1 || kstar > kmax) return COSMOS_EINVAL;
  CompVjp q;
  q.g = make_devgrid(g);
  q.ic = g->nx / 2;
  q.jc = g->ny / 2;
  q.kc = g->nz / 2;
  q.kstar = kstar;
  q.nf = cosmos_nfields(p);
  q.h3 = g->h[0] * g->h[1] * g->h[2];
  q.cbar = cbar;
  q.V = aux_host[4 * (kstar - 1) + 1];
  q.R = aux_host[4 * (kstar - 1) + 2];
  q.C = 2.0 * aux_host[4 * (kstar - 1) + 3] / q.R;
  q.Vall = aux_host[4 * kmax + 1];
  q.Ebar = aux_host[4 * kmax + 0] / q.Vall;
  q.rstar = kstar * g->h[0];
  compaction_vjp_kernel<<<point_grid(q.g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(q, state, lam);
  return cudaGetLastError() == cudaSuccess ? COSMOS_OK : COSMOS_ECUDA;
}

}  // extern "C"

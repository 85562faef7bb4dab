// C ABI of libcosmos_gb300 (declared in include/cosmos.h): argument
// validation, workspace layout, initial-data and reduction kernels, and the
// launch sequences of the right-hand side, RK4 and constraint calls.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "host.cuh"

namespace cosmos {

static thread_local int g_last_cuda_error = 0;

static int cuda_fail(cudaError_t e) {
  g_last_cuda_error = (int)e;
  return COSMOS_ECUDA;
}

int cuda_error(cudaError_t e) { return cuda_fail(e); }

#define CK(expr)                             \
  do {                                       \
    cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

Coef make_coef(const cosmos_grid* g, double sigma) {
  Coef c;
  for (int d = 0; d < 3; ++d) {
    const double h = g->h[d];
    c.d1a[d] = 8.0 / (12.0 * h);
    c.d1b[d] = 1.0 / (12.0 * h);
    c.d2a[d] = 16.0 / (12.0 * h * h);
    c.d2b[d] = 1.0 / (12.0 * h * h);
    c.ko[d] = sigma / (64.0 * h);
    c.ih[d] = 1.0 / h;
  }
  c.mix[0] = 1.0 / (144.0 * g->h[0] * g->h[1]);
  c.mix[1] = 1.0 / (144.0 * g->h[0] * g->h[2]);
  c.mix[2] = 1.0 / (144.0 * g->h[1] * g->h[2]);
  c.ko_s = (c.ko[0] == c.ko[1] && c.ko[1] == c.ko[2]) ? c.ko[0] : 1.0;
  return c;
}

DevGrid make_devgrid(const cosmos_grid* g) {
  DevGrid d;
  d.nx = g->nx;
  d.ny = g->ny;
  d.nz = g->nz;
  d.pitch = g->pitch;
  d.fstride = (long)g->pitch * g->ny * g->nz;
  for (int k = 0; k < 3; ++k) d.h[k] = g->h[k];
  return d;
}

double K_ref(const cosmos_params* p, double t) {
  if (p->H0 == 0.0) return 0.0;
  return -3.0 * p->H0 / (1.0 + 1.5 * (1.0 + p->w) * p->H0 * (t - p->t0));
}

AlgebraParams algebra_params(const cosmos_params* p, double t) {
  AlgebraParams a;
  a.eta = p->eta;
  a.Kref = K_ref(p, t);
  a.lapse_c1 = p->slicing == 0 ? 2.0 : 0.0;
  a.lapse_c2 = p->slicing == 0 ? 0.0 : 1.0;
  a.shift_on = p->shift ? 1.0 : 0.0;
  a.w = p->w;
  return a;
}

static long n_blocks(const DevGrid& g) {
  const dim3 b = point_grid(g);
  return (long)b.x * b.y * b.z;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int validate(const cosmos_grid* g, const cosmos_params* p) {
  if (!g || !p) return COSMOS_EINVAL;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->pitch < g->nx) return COSMOS_EINVAL;
  if (g->nz > 65535 || (g->ny + BY - 1) / BY > 65535) return COSMOS_EINVAL;
  // the derivative pass forms neighbour offsets within one field in 32 bits
  if ((long long)g->pitch * g->ny * g->nz >= (1ll << 31)) return COSMOS_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!(g->h[d] > 0.0) || !isfinite(g->h[d])) return COSMOS_EINVAL;
  if (p->slicing != 0 && p->slicing != 1) return COSMOS_EINVAL;
  if (p->shift != 0 && p->shift != 1) return COSMOS_EINVAL;
  if (p->fluid != 0 && p->fluid != 1) return COSMOS_EINVAL;
  if (p->scalar != 0 && p->scalar != 1) return COSMOS_EINVAL;
  if (!(p->ko_sigma >= 0.0) || !isfinite(p->eta)) return COSMOS_EINVAL;
  if (p->fluid && !(p->w > 0.0 && p->w <= 1.0)) return COSMOS_EINVAL;
  return COSMOS_OK;
}

WsLayout ws_layout(const cosmos_grid* g, const cosmos_params* p, int op) {
  const DevGrid d = make_devgrid(g);
  const size_t fs = (size_t)d.fstride;
  const int nf = 24 + 4 * p->fluid + 2 * p->scalar;
  WsLayout L;
  memset(&L, 0, sizeof(L));
  size_t off = 0;
  auto take = [&](size_t doubles) {
    size_t o = off;
    off += align256(doubles * sizeof(double));
    return o / sizeof(double);
  };
  const bool fluid = p->fluid != 0;
  if (op == COSMOS_OP_RHS || op == COSMOS_OP_RK4) {
    if (fluid) {
      L.prim = take(4 * fs);
      L.flux = take(12 * fs);
    }
    L.D = take((size_t)nder(p->scalar) * fs);
    // limb copy of the stage state (8 bytes per value) for the integer
    // derivative pass, one slot per field with derivatives, and their exponents
    const int nslot = 24 + 2 * p->scalar;
    L.limbs = take((size_t)nslot * fs);
    L.expo = take(((size_t)nslot + 1) / 2);
    L.erec = take(16 * (size_t)nslot);  // 32 unsigned per slot, one cache line each
    if (op == COSMOS_OP_RK4) {
      L.stageA = take(nf * fs);
      L.stageB = take(nf * fs);
      L.acc = take(nf * fs);
    }
  } else if (op == COSMOS_OP_CONSTRAINTS || op == COSMOS_OP_INIT) {
    if (fluid) L.prim = take(4 * fs);
    if (op == COSMOS_OP_INIT) L.hm = take(4 * fs);
    L.partial = take(8 * n_blocks(d));
    L.final_ = take(8);
  } else if (op == COSMOS_OP_SCAN) {
    L.scan = take((size_t)(nf + 1) / 2);  // one 32-bit count per field
  }
  L.total_bytes = off;
  return L;
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
// Per-field count of non-finite values (and, fluid on, of tau~ <= 0):
// blockIdx.y = field; a warp-uniform grid-stride loop over the points.
__global__ void scan_state_kernel(const DevGrid g, const double* __restrict__ U, int tau_field,
                                  unsigned* __restrict__ counts) {
  const int f = blockIdx.y;
  const long npts = (long)g.nx * g.ny * g.nz;
  const double* Uf = U + (long)f * g.fstride;
  unsigned c = 0;
  for (long base = (long)blockIdx.x * blockDim.x; base < npts; base += (long)gridDim.x * blockDim.x) {
    const long q = base + threadIdx.x;
    bool bad = false;
    if (q < npts) {
      const int i = (int)(q % g.nx);
      const long r = q / g.nx;
      const int j = (int)(r % g.ny), k = (int)(r / g.ny);
      const double v = Uf[((long)k * g.ny + j) * g.pitch + i];
      bad = !isfinite(v) || (f == tau_field && !(v > 0.0));
    }
    c += __popc(__ballot_sync(0xffffffffu, bad));
  }
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(counts + f, c);
}

__global__ void reduce_partials(const double* __restrict__ part, long nb, double* __restrict__ out) {
  // one block of 256 threads; fixed summation order
  __shared__ double s[256][8];
  double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      r[m] += part[b * 8 + m];
      r[4 + m] = fmax(r[4 + m], part[b * 8 + 4 + m]);
    }
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) s[threadIdx.x][m] = r[m];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        s[threadIdx.x][m] += s[threadIdx.x + w][m];
        s[threadIdx.x][4 + m] = fmax(s[threadIdx.x][4 + m], s[threadIdx.x + w][4 + m]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int m = 0; m < 8; ++m) out[m] = s[0][m];
}

struct InitArgs {
  DevGrid g;
  double x0[3];
  int nf;
  int isc;  // index of phi (scalar on), else -1
  cosmos_id id;
  double H0;
  double Lx;  // gauge-wave wavelength
};

__global__ void init_metric_kernel(const InitArgs a, double* __restrict__ U) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.g.nx || j >= a.g.ny) return;
  const long c = ((long)k * a.g.ny + j) * a.g.pitch + i;
  const long fs = a.g.fstride;
  double v[30];
  for (int f = 0; f < 30; ++f) v[f] = 0.0;
  const double x[3] = {a.x0[0] + i * a.g.h[0], a.x0[1] + j * a.g.h[1], a.x0[2] + k * a.g.h[2]};
  if (a.id.kind == 0) {
    // gauge wave: gamma_xx = H, alpha = sqrt(H), K_xx = -d_t H / (2 sqrt(H))
    const double Lx = a.Lx;
    const double ph = 2.0 * PI * (x[0] - a.id.t) / Lx;
    const double H = 1.0 - a.id.A * sin(ph);
    const double dtH = a.id.A * (2.0 * PI / Lx) * cos(ph);
    const double sH = sqrt(H);
    const double Kxx = -dtH / (2.0 * sH);
    const double trK = Kxx / H;
    const double chi = pow(H, -1.0 / 3.0);
    v[0] = chi;
    v[1] = pow(H, 2.0 / 3.0);
    v[4] = chi;
    v[6] = chi;
    v[7] = trK;
    v[8] = chi * (Kxx - H * trK / 3.0);
    v[11] = -chi * trK / 3.0;
    v[13] = -chi * trK / 3.0;
    v[14] = 2.0 / 3.0 * pow(H, -5.0 / 3.0) * (-dtH);  // -d_x gt^xx, d_x H = -d_t H
    v[17] = sH;
  } else {
    // FLRW + zeta, leading gradient order: gamma_ij = a0^2 exp(2 zeta) delta_ij
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double u = (x[d] - a.id.center[d]) / a.id.q[d];
      r2 += u * u;
    }
    const double shape = exp(-r2 / (2.0 * a.id.sigma * a.id.sigma));
    const double zeta = a.id.mu * shape;
    v[0] = exp(-2.0 * zeta) / (a.id.a0 * a.id.a0);
    v[1] = v[4] = v[6] = 1.0;
    v[7] = -3.0 * a.H0;
    v[17] = 1.0;
    if (a.id.kind == 2) v[a.isc] = a.id.A * shape;  // isocurvature scalar, Pi = 0
  }
  for (int f = 0; f < a.nf; ++f) U[f * fs + c] = v[f];
}

// tau~ = sqrt(gamma) E with E = (R + 2/3 K^2 - At.At)/(16 pi) = H_vacuum/(16 pi),
// less the scalar's energy 1/2 chi gt^ij d_i phi d_j phi when isc >= 0 (Pi = 0;
// these data have gt = delta, so gt^ij d_i phi d_j phi = |d phi|^2, with the
// 4th-order centred first derivative of phi).
__global__ void init_tau_kernel(const DevGrid g, const Coef cf, int isc, const double* __restrict__ hm,
                                double* __restrict__ U) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long c = ((long)k * g.ny + j) * g.pitch + i;
  const double chi = U[c];
  double E = hm[c] / (16.0 * PI);
  if (isc >= 0) {
    const Nbr n = make_nbr(g, i, j, k);
    const double* phi = U + (long)isc * g.fstride;
    double d2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long o[4] = {d == 0 ? at(n, 1, 0, 0) : d == 1 ? at(n, 0, 1, 0) : at(n, 0, 0, 1),
                         d == 0 ? at(n, -1, 0, 0) : d == 1 ? at(n, 0, -1, 0) : at(n, 0, 0, -1),
                         d == 0 ? at(n, 2, 0, 0) : d == 1 ? at(n, 0, 2, 0) : at(n, 0, 0, 2),
                         d == 0 ? at(n, -2, 0, 0) : d == 1 ? at(n, 0, -2, 0) : at(n, 0, 0, -2)};
      const double dphi = (phi[o[0]] - phi[o[1]]) * cf.d1a[d] - (phi[o[2]] - phi[o[3]]) * cf.d1b[d];
      d2 += dphi * dphi;
    }
    E -= 0.5 * chi * d2;
  }
  U[24 * g.fstride + c] = E / (chi * sqrt(chi));
}

__global__ void fp64_fma_chains(double* __restrict__ out, int iters, double a, double b) {
  double acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = (threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

typedef cudaError_t (*StageLauncher)(const StageArgs&, int, cudaStream_t);
typedef cudaError_t (*ConstraintLauncher)(const ConstraintArgs&, cudaStream_t);

static StageLauncher stage_launcher(const cosmos_params* p) {
  if (p->fluid && p->scalar) return launch_stage_fluid_scalar;
  if (p->fluid) return launch_stage_fluid;
  if (p->scalar) return launch_stage_scalar;
  return launch_stage_vac;
}

static ConstraintLauncher constraint_launcher(const cosmos_params* p) {
  if (p->fluid && p->scalar) return launch_constraints_fluid_scalar;
  if (p->fluid) return launch_constraints_fluid;
  if (p->scalar) return launch_constraints_scalar;
  return launch_constraints_vac;
}

// Shared body of cosmos_rhs / cosmos_rk4_stage / cosmos_stage_pass.
// pass_mask bit 0: fluid pre-pass (primitives, face fluxes); bit 1: derivative
// pass; bit 2: algebra pass + combine.
// f_lo, f_hi: field range of the derivative pass (f_hi = 0: all fields);
// k_lo, k_cnt: plane range of the algebra pass (k_cnt = 0: all planes).
int run_stage(const cosmos_grid* g, const cosmos_params* p, int mode, const double* U_s, double* U_n, double* out,
              double* acc, double t_stage, double cdt, double bk, double* ws, const WsLayout& L, cudaStream_t s,
              int pass_mask, int f_lo, int f_hi, int k_lo, int k_cnt, const int* E_ext, int expo_flags) {
  StageArgs a;
  memset(&a, 0, sizeof(a));
  a.f_lo = f_lo;
  a.f_hi = f_hi;
  a.k_lo = k_lo;
  a.k_cnt = k_cnt;
  a.g = make_devgrid(g);
  a.c = make_coef(g, p->ko_sigma);
  a.ap = algebra_params(p, t_stage);
  a.U = U_s;
  a.U0 = U_n;
  a.U0w = U_n;
  a.out = out;
  a.acc = acc;
  a.cdt = cdt;
  a.bk = bk;
  a.D = ws + L.D;
  if (p->fluid) {
    double* prim = ws + L.prim;
    double* flux = ws + L.flux;
    if (pass_mask & 1) {
      CK(launch_fluid_prim(a.g, U_s, prim, p->w, s));
      CK(launch_fluid_flux(a.g, U_s, prim, flux, p->w, 24, s));
    }
    a.prim = prim;
    a.flux = flux;
  }
  if (pass_mask & 2) {
    // limb copy of the fields of this derivative pass (slots of fields f_lo .. f_hi - 1)
    a.L = (const long long*)(ws + L.limbs);
    a.E = (const int*)(ws + L.expo);
    const int nf = cosmos_nfields(p), hi = f_hi > 0 ? f_hi : nf;
    int s_lo = 1 << 30, s_hi = 0;
    for (int f = f_lo; f < hi; ++f) {
      if (p->fluid && f >= 24 && f < 28) continue;  // no derivatives of the fluid fields here
      const int sl = (p->fluid && f >= 28) ? f - 4 : f;
      s_lo = sl < s_lo ? sl : s_lo;
      s_hi = sl + 1 > s_hi ? sl + 1 : s_hi;
    }
    if (E_ext) {
      a.E = E_ext;
      CK(launch_to_limbs(a.g, U_s, p->fluid, s_lo, s_hi, E_ext, (long long*)(ws + L.limbs), s));
    } else if (expo_flags & 1) {  // exponents recorded by the previous stage's algebra pass
      CK(launch_to_limbs(a.g, U_s, p->fluid, s_lo, s_hi, a.E, (long long*)(ws + L.limbs), s));
    } else {
      CK(launch_limbs(a.g, U_s, p->fluid, s_lo, s_hi, (int*)(ws + L.expo), (long long*)(ws + L.limbs), s));
    }
  }
  const int nslot = 24 + 2 * p->scalar;
  if (expo_flags & 2) {
    a.E_rec = (unsigned*)(ws + L.erec);
    if (expo_flags & 4) CK(cudaMemsetAsync(a.E_rec, 0, sizeof(unsigned) * 32 * nslot, s));
  }
  if ((pass_mask & 6) == 6) {
    CK(stage_launcher(p)(a, mode, s));
  } else if (pass_mask & 2) {
    CK(stage_launcher(p)(a, -1, s));  // derivative pass only
  } else if (pass_mask & 4) {
    CK(stage_launcher(p)(a, mode | 8, s));  // algebra pass only
  }
  if ((expo_flags & 2) && (pass_mask & 4)) CK(launch_exponents_from_record(a.E_rec, (int*)(ws + L.expo), nslot, s));
  return COSMOS_OK;
}

int check_ws(const WsLayout& L, void* ws, size_t ws_bytes) {
  if (L.total_bytes == 0) return COSMOS_OK;
  if (!ws) return COSMOS_EINVAL;
  if (ws_bytes < L.total_bytes) return COSMOS_EWORKSPACE;
  if (((uintptr_t)ws & 255u) != 0) return COSMOS_EALIGN;
  return COSMOS_OK;
}

int init_grid(const cosmos_grid* g, const cosmos_params* p, const cosmos_id* id, double* state, void* ws,
              size_t ws_bytes, cudaStream_t s, double Lx_wave) {
  int e = validate(g, p);
  if (e) return e;
  if (!id || !state) return COSMOS_EINVAL;
  if (!aligned16(state)) return COSMOS_EALIGN;
  if (id->kind < 0 || id->kind > 3) return COSMOS_EINVAL;
  if (id->kind == 0 && p->fluid) return COSMOS_EINVAL;                   // the gauge wave is vacuum
  if (id->kind == 2 && (!p->fluid || !p->scalar)) return COSMOS_EINVAL;  // isocurvature: scalar + fluid
  if (id->kind == 3 && (!p->fluid || !(p->H0 > 0.0))) return COSMOS_EINVAL;  // next order: fluid, background
  if (id->kind >= 1 && (!(id->sigma > 0.0) || !(id->a0 > 0.0) || !(id->q[0] > 0.0) || !(id->q[1] > 0.0) ||
                        !(id->q[2] > 0.0)))
    return COSMOS_EINVAL;
  const WsLayout L = ws_layout(g, p, COSMOS_OP_INIT);
  const bool need_ws = (id->kind >= 1 && p->fluid);
  if (need_ws && (e = check_ws(L, ws, ws_bytes))) return e;
  InitArgs a;
  a.g = make_devgrid(g);
  for (int d = 0; d < 3; ++d) a.x0[d] = g->x0[d];
  a.nf = cosmos_nfields(p);
  a.isc = p->scalar ? 24 + 4 * p->fluid : -1;
  a.id = *id;
  a.H0 = p->H0;
  a.Lx = Lx_wave > 0.0 ? Lx_wave : g->nx * g->h[0];
  init_metric_kernel<<<point_grid(a.g), dim3(BX, BY), 0, s>>>(a, state);
  CK(cudaGetLastError());
  if (id->kind == 3) {
    double* w = (double*)ws;
    return init_nlo(g, p, state, w + L.hm, w + L.partial, s);
  }
  if (need_ws) {
    double* w = (double*)ws;
    ConstraintArgs c;
    memset(&c, 0, sizeof(c));
    c.g = a.g;
    c.c = make_coef(g, 0.0);
    cosmos_params pv = *p;
    pv.fluid = 0;
    pv.scalar = 0;
    c.ap = algebra_params(&pv, 0.0);
    c.U = state;
    c.hm = w + L.hm;
    c.partial = w + L.partial;
    CK(launch_constraints_vac(c, s));
    init_tau_kernel<<<point_grid(a.g), dim3(BX, BY), 0, s>>>(a.g, make_coef(g, 0.0), id->kind == 2 ? a.isc : -1,
                                                             w + L.hm, state);
    CK(cudaGetLastError());
  }
  return COSMOS_OK;
}

}  // namespace cosmos

using namespace cosmos;

extern "C" {

int cosmos_nfields(const cosmos_params* p) {
  if (!p) return COSMOS_EINVAL;
  return 24 + 4 * (p->fluid != 0) + 2 * (p->scalar != 0);
}

size_t cosmos_field_stride(const cosmos_grid* g) {
  if (!g) return 0;
  return (size_t)g->pitch * g->ny * g->nz;
}

size_t cosmos_workspace_bytes(const cosmos_grid* g, const cosmos_params* p, int op) {
  if (validate(g, p) != COSMOS_OK) return 0;
  return ws_layout(g, p, op).total_bytes;
}

int cosmos_init_grid(const cosmos_grid* g, const cosmos_params* p, const cosmos_id* id, double* state, void* ws,
                     size_t ws_bytes, void* stream) {
  return init_grid(g, p, id, state, ws, ws_bytes, (cudaStream_t)stream, 0.0);
}

int cosmos_rhs(const cosmos_grid* g, const cosmos_params* p, const double* state, double* rhs, double t, void* ws,
               size_t ws_bytes, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (!state || !rhs || state == rhs) return COSMOS_EINVAL;
  if (!aligned16(state) || !aligned16(rhs)) return COSMOS_EALIGN;
  const WsLayout L = ws_layout(g, p, COSMOS_OP_RHS);
  if ((e = check_ws(L, ws, ws_bytes))) return e;
  return run_stage(g, p, MODE_RHS, state, nullptr, rhs, nullptr, t, 0.0, 0.0, (double*)ws, L,
                   (cudaStream_t)stream);
}

int cosmos_rk4_stage(const cosmos_grid* g, const cosmos_params* p, int stage, const double* U_s, double* U_n,
                     double* U_next, double* acc, double t, double dt, void* ws, size_t ws_bytes, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (stage < 1 || stage > 4 || !U_s || !U_n || !acc) return COSMOS_EINVAL;
  if (stage < 4 && !U_next) return COSMOS_EINVAL;
  if (U_s == acc || (stage < 4 && (U_s == U_next || U_next == acc || U_next == U_n))) return COSMOS_EINVAL;
  if (stage == 4 && U_s == U_n) return COSMOS_EINVAL;
  if (!aligned16(U_s) || !aligned16(U_n) || !aligned16(acc) || (U_next && !aligned16(U_next))) return COSMOS_EALIGN;
  const WsLayout L = ws_layout(g, p, COSMOS_OP_RHS);
  if ((e = check_ws(L, ws, ws_bytes))) return e;
  static const double c_stage[4] = {0.0, 0.5, 0.5, 1.0};
  static const int modes[4] = {MODE_S1, MODE_S23, MODE_S23, MODE_S4};
  const double cdt = stage == 1 || stage == 2 ? 0.5 * dt : (stage == 3 ? dt : dt / 6.0);
  return run_stage(g, p, modes[stage - 1], U_s, U_n, U_next, acc, t + c_stage[stage - 1] * dt, cdt, 2.0,
                   (double*)ws, L, (cudaStream_t)stream);
}

int cosmos_field_exponents(const cosmos_grid* g, const cosmos_params* p, const double* state, int* E,
                           void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (!state || !E) return COSMOS_EINVAL;
  const int nslot = 24 + 2 * p->scalar;
  CK(launch_field_exponents(make_devgrid(g), state, p->fluid, 0, nslot, E, (cudaStream_t)stream));
  return COSMOS_OK;
}

int cosmos_rk4_stage_slab(const cosmos_grid* g, const cosmos_params* p, int stage, const double* U_s, double* U_n,
                          double* U_next, double* acc, double t, double dt, int k_lo, int k_cnt, const int* E,
                          void* ws, size_t ws_bytes, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (stage < 1 || stage > 4 || !U_s || !U_n || !acc) return COSMOS_EINVAL;
  if (stage < 4 && !U_next) return COSMOS_EINVAL;
  if (U_s == acc || (stage < 4 && (U_s == U_next || U_next == acc || U_next == U_n))) return COSMOS_EINVAL;
  if (stage == 4 && U_s == U_n) return COSMOS_EINVAL;
  if (k_lo < 0 || k_cnt < 1 || k_lo + k_cnt > g->nz) return COSMOS_EINVAL;
  if (!aligned16(U_s) || !aligned16(U_n) || !aligned16(acc) || (U_next && !aligned16(U_next))) return COSMOS_EALIGN;
  const WsLayout L = ws_layout(g, p, COSMOS_OP_RHS);
  if ((e = check_ws(L, ws, ws_bytes))) return e;
  static const double c_stage[4] = {0.0, 0.5, 0.5, 1.0};
  static const int modes[4] = {MODE_S1, MODE_S23, MODE_S23, MODE_S4};
  const double cdt = stage == 1 || stage == 2 ? 0.5 * dt : (stage == 3 ? dt : dt / 6.0);
  return run_stage(g, p, modes[stage - 1], U_s, U_n, U_next, acc, t + c_stage[stage - 1] * dt, cdt, 2.0,
                   (double*)ws, L, (cudaStream_t)stream, 7, 0, 0, k_lo, k_cnt, E);
}

int cosmos_stage_pass(const cosmos_grid* g, const cosmos_params* p, int pass, int stage, const double* U_s,
                      double* U_n, double* U_next, double* acc, double t, double dt, void* ws, size_t ws_bytes,
                      void* stream) {
  int e = validate(g, p);
  if (e) return e;
  const int opts = pass & ~3;
  pass &= 3;
  if (pass > 2 || (opts & ~(16 | 32 | 64)) || stage < 1 || stage > 4 || !U_s || !U_n || !acc) return COSMOS_EINVAL;
  if (((opts & 16) && pass != 1) || ((opts & (32 | 64)) && (pass != 2 || stage == 4))) return COSMOS_EINVAL;
  if (stage < 4 && !U_next) return COSMOS_EINVAL;
  if (U_s == acc || (stage < 4 && (U_s == U_next || U_next == acc || U_next == U_n))) return COSMOS_EINVAL;
  if (stage == 4 && U_s == U_n) return COSMOS_EINVAL;
  const WsLayout L = ws_layout(g, p, COSMOS_OP_RHS);
  if ((e = check_ws(L, ws, ws_bytes))) return e;
  static const double c_stage[4] = {0.0, 0.5, 0.5, 1.0};
  static const int modes[4] = {MODE_S1, MODE_S23, MODE_S23, MODE_S4};
  const double cdt = stage == 1 || stage == 2 ? 0.5 * dt : (stage == 3 ? dt : dt / 6.0);
  const int expo_flags = ((opts & 16) ? 1 : 0) | ((opts & 32) ? 2 : 0) | ((opts & 64) ? 6 : 0);
  return run_stage(g, p, modes[stage - 1], U_s, U_n, U_next, acc, t + c_stage[stage - 1] * dt, cdt, 2.0,
                   (double*)ws, L, (cudaStream_t)stream, 1 << pass, 0, 0, 0, 0, nullptr, expo_flags);
}

namespace {
// One RK4 step of `state` in place on stream s (arguments already checked).
int rk4_on(const cosmos_grid* g, const cosmos_params* p, double* state, double t, double dt, double* w,
           const WsLayout& L, cudaStream_t s) {
  double* A = w + L.stageA;
  double* B = w + L.stageB;
  double* acc = w + L.acc;
  const double dt2 = 0.5 * dt;
  int e;
  // stage 1 scans U_n (the caller may have changed it); each algebra pass records the
  // exponents of the state it writes, so stages 2-4 need no scan
  if ((e = run_stage(g, p, MODE_S1, state, state, A, acc, t, dt2, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 6))) return e;
  if ((e = run_stage(g, p, MODE_S23, A, state, B, acc, t + dt2, dt2, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 3)))
    return e;
  if ((e = run_stage(g, p, MODE_S23, B, state, A, acc, t + dt2, dt, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 3)))
    return e;
  return run_stage(g, p, MODE_S4, A, state, nullptr, acc, t + dt, dt / 6.0, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 1);
}
}  // namespace

int cosmos_rk4_step(const cosmos_grid* g, const cosmos_params* p, double* state, double t, double dt, void* ws,
                    size_t ws_bytes, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (!state) return COSMOS_EINVAL;
  if (!aligned16(state)) return COSMOS_EALIGN;
  const WsLayout L = ws_layout(g, p, COSMOS_OP_RK4);
  if ((e = check_ws(L, ws, ws_bytes))) return e;
  return rk4_on(g, p, state, t, dt, (double*)ws, L, (cudaStream_t)stream);
}

int cosmos_rk4_step_stages(const cosmos_grid* g, const cosmos_params* p, double* state, double t, double dt,
                           double* U2, double* U3, double* U4, void* ws, size_t ws_bytes, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (!state || !U2 || !U3 || !U4) return COSMOS_EINVAL;
  if (U2 == state || U3 == state || U4 == state || U2 == U3 || U2 == U4 || U3 == U4) return COSMOS_EINVAL;
  if (!aligned16(state) || !aligned16(U2) || !aligned16(U3) || !aligned16(U4)) return COSMOS_EALIGN;
  const WsLayout L = ws_layout(g, p, COSMOS_OP_RK4);
  if ((e = check_ws(L, ws, ws_bytes))) return e;
  double* w = (double*)ws;
  double* acc = w + L.acc;
  cudaStream_t s = (cudaStream_t)stream;
  const double dt2 = 0.5 * dt;
  // the stages of cosmos_rk4_step, with the stage states kept in U2, U3, U4
  if ((e = run_stage(g, p, MODE_S1, state, state, U2, acc, t, dt2, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 6))) return e;
  if ((e = run_stage(g, p, MODE_S23, U2, state, U3, acc, t + dt2, dt2, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 3)))
    return e;
  if ((e = run_stage(g, p, MODE_S23, U3, state, U4, acc, t + dt2, dt, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 3)))
    return e;
  return run_stage(g, p, MODE_S4, U4, state, nullptr, acc, t + dt, dt / 6.0, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 1);
}

namespace {
// Copy stream and events of one cosmos_evolve_host call; destroyed on every
// return path (work still queued on them completes first).
// Copy stream and events of cosmos_evolve_host.  On every return, an early
// error return included, the copy stream is waited for first: no copy of the
// call writes the caller's host buffer after the call has returned.
struct HostPipeline {
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[16] = {};
  ~HostPipeline() {
    if (cs) cudaStreamSynchronize(cs);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);
  }
};
}  // namespace

int cosmos_evolve_host(const cosmos_grid* g, const cosmos_params* p, const double* host_in, double* host_out,
                       double* dev_state, int steps, double t, double dt, void* ws, size_t ws_bytes, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (!host_in || !host_out || !dev_state || steps < 0) return COSMOS_EINVAL;
  if (!aligned16(dev_state)) return COSMOS_EALIGN;
  const size_t fs = cosmos_field_stride(g);
  const int nf = cosmos_nfields(p);
  const size_t bytes = fs * (size_t)nf * sizeof(double);
  cudaStream_t s = (cudaStream_t)stream;
  if (steps == 0) {
    CK(cudaMemcpyAsync(dev_state, host_in, bytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(host_out, dev_state, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return COSMOS_OK;
  }
  const WsLayout L = ws_layout(g, p, COSMOS_OP_RK4);
  if ((e = check_ws(L, ws, ws_bytes))) return e;
  double* w = (double*)ws;
  double* A = w + L.stageA;
  double* B = w + L.stageB;
  double* acc = w + L.acc;
  const double dt2 = 0.5 * dt;
  // The copies run on their own stream: the host-to-device copy in NCH field
  // groups, each followed on `s` by the first derivative pass over those
  // fields; the device-to-host copy in NSL slabs of z-planes, each started as
  // soon as the last algebra pass has written its planes.
  constexpr int NCH = 4, NSL_MAX = 8;
  const int nsl = g->nz < NSL_MAX ? g->nz : NSL_MAX;
  const size_t plane = (size_t)g->ny * (size_t)g->pitch;
  HostPipeline hp;
  CK(cudaStreamCreateWithFlags(&hp.cs, cudaStreamNonBlocking));
  for (int m = 0; m < 1 + NCH + NSL_MAX; ++m) CK(cudaEventCreateWithFlags(&hp.ev[m], cudaEventDisableTiming));
  CK(cudaEventRecord(hp.ev[0], s));  // earlier work on `s` may still use dev_state
  CK(cudaStreamWaitEvent(hp.cs, hp.ev[0], 0));
  int fb[NCH + 1];
  for (int c = 0; c <= NCH; ++c) fb[c] = c * nf / NCH;
  for (int c = 0; c < NCH; ++c) {
    const size_t off = (size_t)fb[c] * fs, n = (size_t)(fb[c + 1] - fb[c]) * fs;
    if (n) CK(cudaMemcpyAsync(dev_state + off, host_in + off, n * sizeof(double), cudaMemcpyHostToDevice, hp.cs));
    CK(cudaEventRecord(hp.ev[1 + c], hp.cs));
  }
  for (int step = 0; step < steps; ++step) {
    const double ts = t + step * dt;
    if (step == 0) {
      for (int c = 0; c < NCH; ++c) {
        CK(cudaStreamWaitEvent(s, hp.ev[1 + c], 0));
        if (fb[c + 1] > fb[c] &&
            (e = run_stage(g, p, MODE_S1, dev_state, dev_state, A, acc, ts, dt2, 2.0, w, L, s, 2, fb[c], fb[c + 1])))
          return e;
      }
      if ((e = run_stage(g, p, MODE_S1, dev_state, dev_state, A, acc, ts, dt2, 2.0, w, L, s, 5, 0, 0, 0, 0, nullptr,
                         6)))
        return e;
    } else if ((e = run_stage(g, p, MODE_S1, dev_state, dev_state, A, acc, ts, dt2, 2.0, w, L, s, 7, 0, 0, 0, 0,
                              nullptr, 6))) {
      return e;
    }
    // as cosmos_rk4_step: stages 2-4 take the exponents the algebra pass before recorded
    if ((e = run_stage(g, p, MODE_S23, A, dev_state, B, acc, ts + dt2, dt2, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 3)))
      return e;
    if ((e = run_stage(g, p, MODE_S23, B, dev_state, A, acc, ts + dt2, dt, 2.0, w, L, s, 7, 0, 0, 0, 0, nullptr, 3)))
      return e;
    if (step + 1 < steps) {
      if ((e = run_stage(g, p, MODE_S4, A, dev_state, nullptr, acc, ts + dt, dt / 6.0, 2.0, w, L, s, 7, 0, 0, 0, 0,
                         nullptr, 1)))
        return e;
      continue;
    }
    if ((e = run_stage(g, p, MODE_S4, A, dev_state, nullptr, acc, ts + dt, dt / 6.0, 2.0, w, L, s, 3, 0, 0, 0, 0,
                       nullptr, 1)))
      return e;
    for (int sl = 0; sl < nsl; ++sl) {
      const int k0 = sl * g->nz / nsl, k1 = (sl + 1) * g->nz / nsl;
      if ((e = run_stage(g, p, MODE_S4, A, dev_state, nullptr, acc, ts + dt, dt / 6.0, 2.0, w, L, s, 4, 0, 0, k0,
                         k1 - k0)))
        return e;
      CK(cudaEventRecord(hp.ev[1 + NCH + sl], s));
      CK(cudaStreamWaitEvent(hp.cs, hp.ev[1 + NCH + sl], 0));
      for (int f = 0; f < nf; ++f) {
        const size_t off = (size_t)f * fs + (size_t)k0 * plane;
        CK(cudaMemcpyAsync(host_out + off, dev_state + off, (size_t)(k1 - k0) * plane * sizeof(double),
                           cudaMemcpyDeviceToHost, hp.cs));
      }
    }
  }
  CK(cudaStreamSynchronize(hp.cs));
  CK(cudaStreamSynchronize(s));
  return COSMOS_OK;
}

namespace {
constexpr int MANY_MAX_BUF = 16;
// Streams and per-buffer events of cosmos_evolve_host_many.  As for
// HostPipeline, the copy streams are waited for on every return.
struct ManyPipeline {
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, ev_in[MANY_MAX_BUF] = {}, ev_comp[MANY_MAX_BUF] = {}, ev_out[MANY_MAX_BUF] = {};
  ~ManyPipeline() {
    if (in) cudaStreamSynchronize(in);
    if (out) cudaStreamSynchronize(out);
    for (int b = 0; b < MANY_MAX_BUF; ++b)
      for (cudaEvent_t e : {ev_in[b], ev_comp[b], ev_out[b]})
        if (e) cudaEventDestroy(e);
    if (start) cudaEventDestroy(start);
    if (in) cudaStreamDestroy(in);
    if (out) cudaStreamDestroy(out);
  }
};

bool ranges_overlap(const void* a, const void* b, size_t bytes) {
  const char *x = (const char*)a, *y = (const char*)b;
  return x < y + bytes && y < x + bytes;
}
}  // namespace

int cosmos_evolve_host_many(const cosmos_grid* g, const cosmos_params* p, int count, const double* const* host_in,
                            double* const* host_out, double* const* dev_states, int nbuf, int steps, double t,
                            double dt, void* ws, size_t ws_bytes, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (count < 0 || steps < 0 || nbuf < 1 || nbuf > MANY_MAX_BUF) return COSMOS_EINVAL;
  if (count == 0) return COSMOS_OK;
  if (!host_in || !host_out || !dev_states) return COSMOS_EINVAL;
  const size_t fs = cosmos_field_stride(g);
  const int nf = cosmos_nfields(p);
  const size_t bytes = fs * (size_t)nf * sizeof(double);
  for (int b = 0; b < nbuf; ++b) {
    if (!dev_states[b]) return COSMOS_EINVAL;
    if (!aligned16(dev_states[b])) return COSMOS_EALIGN;
    for (int c = 0; c < b; ++c)
      if (ranges_overlap(dev_states[b], dev_states[c], bytes)) return COSMOS_EINVAL;
  }
  // a result must not land on inputs that later copies still read
  for (int i = 0; i < count; ++i) {
    if (!host_in[i] || !host_out[i]) return COSMOS_EINVAL;
    for (int j = 0; j < count; ++j)
      if (ranges_overlap(host_out[i], host_in[j], bytes)) return COSMOS_EINVAL;
  }
  WsLayout L{};
  if (steps > 0) {
    L = ws_layout(g, p, COSMOS_OP_RK4);
    if ((e = check_ws(L, ws, ws_bytes))) return e;
  }
  double* w = (double*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  // State i lives in dev_states[i % nbuf].  The copy-in stream fills a buffer
  // once the copy-out stream has emptied it; the state is advanced on `s`;
  // the copy-out stream reads it back.  Copies of other states overlap each
  // computation, and copies in and out overlap each other.
  ManyPipeline mp;
  CK(cudaStreamCreateWithFlags(&mp.in, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&mp.out, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&mp.start, cudaEventDisableTiming));
  for (int b = 0; b < nbuf; ++b) {
    CK(cudaEventCreateWithFlags(&mp.ev_in[b], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&mp.ev_comp[b], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&mp.ev_out[b], cudaEventDisableTiming));
  }
  CK(cudaEventRecord(mp.start, s));  // earlier work on `s` may still use the buffers
  CK(cudaStreamWaitEvent(mp.in, mp.start, 0));
  CK(cudaStreamWaitEvent(mp.out, mp.start, 0));
  for (int i = 0; i < count && i < nbuf; ++i) {
    CK(cudaMemcpyAsync(dev_states[i], host_in[i], bytes, cudaMemcpyHostToDevice, mp.in));
    CK(cudaEventRecord(mp.ev_in[i], mp.in));
  }
  for (int i = 0; i < count; ++i) {
    const int b = i % nbuf;
    double* d = dev_states[b];
    CK(cudaStreamWaitEvent(s, mp.ev_in[b], 0));
    for (int k = 0; k < steps; ++k)
      if ((e = rk4_on(g, p, d, t + k * dt, dt, w, L, s))) return e;
    CK(cudaEventRecord(mp.ev_comp[b], s));
    CK(cudaStreamWaitEvent(mp.out, mp.ev_comp[b], 0));
    CK(cudaMemcpyAsync(host_out[i], d, bytes, cudaMemcpyDeviceToHost, mp.out));
    CK(cudaEventRecord(mp.ev_out[b], mp.out));
    const int j = i + nbuf;  // the next state for this buffer
    if (j < count) {
      CK(cudaStreamWaitEvent(mp.in, mp.ev_out[b], 0));
      CK(cudaMemcpyAsync(d, host_in[j], bytes, cudaMemcpyHostToDevice, mp.in));
      CK(cudaEventRecord(mp.ev_in[b], mp.in));
    }
  }
  CK(cudaStreamSynchronize(mp.in));
  CK(cudaStreamSynchronize(mp.out));
  CK(cudaStreamSynchronize(s));
  return COSMOS_OK;
}

int cosmos_constraints(const cosmos_grid* g, const cosmos_params* p, const double* state, double* ham_mom,
                       double norms_host[8], void* ws, size_t ws_bytes, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (!state || !norms_host) return COSMOS_EINVAL;
  if (!aligned16(state) || (ham_mom && !aligned16(ham_mom))) return COSMOS_EALIGN;
  const WsLayout L = ws_layout(g, p, COSMOS_OP_CONSTRAINTS);
  if ((e = check_ws(L, ws, ws_bytes))) return e;
  cudaStream_t s = (cudaStream_t)stream;
  double* w = (double*)ws;
  ConstraintArgs c;
  memset(&c, 0, sizeof(c));
  c.g = make_devgrid(g);
  c.c = make_coef(g, 0.0);
  c.ap = algebra_params(p, 0.0);
  c.U = state;
  c.hm = ham_mom;
  c.partial = w + L.partial;
  if (p->fluid) {
    CK(launch_fluid_prim(c.g, state, w + L.prim, p->w, s));
    c.prim = w + L.prim;
  }
  CK(constraint_launcher(p)(c, s));
  reduce_partials<<<1, 256, 0, s>>>(w + L.partial, n_blocks(c.g), w + L.final_);
  CK(cudaGetLastError());
  double r[8];
  CK(cudaMemcpyAsync(r, w + L.final_, sizeof(r), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double npts = (double)g->nx * g->ny * g->nz;
  for (int m = 0; m < 4; ++m) {
    norms_host[m] = sqrt(r[m] / npts);
    norms_host[4 + m] = r[4 + m];
  }
  return COSMOS_OK;
}

int cosmos_scan_state(const cosmos_grid* g, const cosmos_params* p, const double* state, int* counts_host, void* ws,
                      size_t ws_bytes, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (!state) return COSMOS_EINVAL;
  if (!aligned16(state)) return COSMOS_EALIGN;
  const WsLayout L = ws_layout(g, p, COSMOS_OP_SCAN);
  if ((e = check_ws(L, ws, ws_bytes))) return e;
  cudaStream_t s = (cudaStream_t)stream;
  const int nf = 24 + 4 * p->fluid + 2 * p->scalar;
  unsigned* counts = (unsigned*)((double*)ws + L.scan);
  CK(cudaMemsetAsync(counts, 0, nf * sizeof(unsigned), s));
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const DevGrid d = make_devgrid(g);
  const long npts = (long)g->nx * g->ny * g->nz;
  const long per_field = std::max(1L, std::min((long)(4 * sms / nf + 1), (npts + 255) / 256));
  scan_state_kernel<<<dim3((unsigned)per_field, nf), 256, 0, s>>>(d, state, p->fluid ? 24 : -1, counts);
  CK(cudaGetLastError());
  unsigned h[30];
  CK(cudaMemcpyAsync(h, counts, nf * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  bool any = false;
  for (int f = 0; f < nf; ++f) {
    if (counts_host) counts_host[f] = (int)h[f];
    any = any || h[f];
  }
  return any ? COSMOS_ENONFINITE : COSMOS_OK;
}

int cosmos_probe_fp64(double* scratch, double* flops_out, void* stream) {
  if (!scratch || !flops_out) return COSMOS_EINVAL;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (sms > 152) sms = 152;  // scratch holds 152 * 8 * 256 doubles
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = sms * 8, threads = 256, iters = 4096;
  struct Events {  // destroyed on every return
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Events() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } ev;
  CK(cudaEventCreate(&ev.e0));
  CK(cudaEventCreate(&ev.e1));
  fp64_fma_chains<<<blocks, threads, 0, s>>>(scratch, iters, 0.999999, 1e-7);  // warm-up
  CK(cudaEventRecord(ev.e0, s));
  fp64_fma_chains<<<blocks, threads, 0, s>>>(scratch, iters, 0.999999, 1e-7);
  CK(cudaEventRecord(ev.e1, s));
  CK(cudaEventSynchronize(ev.e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
  *flops_out = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3);
  return COSMOS_OK;
}

int cosmos_last_cuda_error(void) { return g_last_cuda_error; }

const char* cosmos_strerror(int code) {
  switch (code) {
    case COSMOS_OK: return "ok";
    case COSMOS_EINVAL: return "invalid argument";
    case COSMOS_ECUDA: return "CUDA runtime error (see cosmos_last_cuda_error)";
    case COSMOS_EWORKSPACE: return "workspace too small";
    case COSMOS_EALIGN: return "pointer not aligned (16 bytes; workspace 256 bytes)";
    case COSMOS_ENONFINITE: return "non-finite or unphysical state";
    case COSMOS_EIO: return "file could not be opened, read or written";
    case COSMOS_ECHECKPOINT: return "checkpoint of another grid or parameters, or corrupt";
    default: return "unknown error code";
  }
}

}  // extern "C"

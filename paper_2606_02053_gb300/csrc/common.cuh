// Internal definitions shared by the CUDA translation units of libcosmos_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cosmos.h"
#include "generated/bssn_algebra.cuh"
#include "generated/fluid_algebra.cuh"

namespace cosmos {

constexpr double PI = 3.14159265358979323846;
constexpr int BX = 32;  // threads per block along x (one warp = one row)
constexpr int BY = 4;   // rows per block
#ifndef COSMOS_DERIV_ROWS
#define COSMOS_DERIV_ROWS 8
#endif
constexpr int DBY = COSMOS_DERIV_ROWS;  // rows per block of the derivative pass

// Grid description as the kernels see it.
struct DevGrid {
  int nx, ny, nz, pitch;
  long fstride;  // doubles between fields
  double h[3];
};

// Periodic neighbour offsets of one point for offsets -3..3 per direction,
// already multiplied by the memory stride of that direction.
struct Nbr {
  long x[7], y[7], z[7];
  long c;  // offset of the point itself
};

__device__ __forceinline__ int wrap_index(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

__device__ __forceinline__ Nbr make_nbr(const DevGrid& g, int i, int j, int k) {
  Nbr n;
  const long row = g.pitch, plane = (long)g.pitch * g.ny;
#pragma unroll
  for (int o = -3; o <= 3; ++o) {
    n.x[o + 3] = wrap_index(i + o, g.nx);
    n.y[o + 3] = wrap_index(j + o, g.ny) * row;
    n.z[o + 3] = wrap_index(k + o, g.nz) * plane;
  }
  n.c = n.z[3] + n.y[3] + n.x[3];
  return n;
}

// Offset of the point displaced by (dx, dy, dz), |d| <= 3.
__device__ __forceinline__ long at(const Nbr& n, int dx, int dy, int dz) {
  return n.z[dz + 3] + n.y[dy + 3] + n.x[dx + 3];
}

__device__ __forceinline__ double ldg(const double* __restrict__ p, long o) { return __ldg(p + o); }

// Stencil coefficients derived on the host from the grid spacing.
struct Coef {
  double d1a[3], d1b[3];  // D1 = a (f+1 - f-1) - b (f+2 - f-2):   a = 8/(12h), b = 1/(12h)
  double d2a[3], d2b[3];  // D2 = a s1 - b s2:                         a = 16/(12h^2), b = 1/(12h^2)
  double mix[3];          // mixed xy, xz, yz:  1/(144 h_a h_b)
  double ko[3];           // sigma/(64 h_d)
  double ih[3];           // 1/h_d (flux divergence)
  double ko_s;            // factor of the KO slots of the derivative buffer: ko[0] with equal
                          // spacing (the slots hold the bracket), else 1 (they hold the term)
};

Coef make_coef(const cosmos_grid* g, double sigma);
DevGrid make_devgrid(const cosmos_grid* g);
double K_ref(const cosmos_params* p, double t);                 // background trace at time t
AlgebraParams algebra_params(const cosmos_params* p, double t); // runtime parameters of the algebra
int validate(const cosmos_grid* g, const cosmos_params* p);     // COSMOS_OK or COSMOS_EINVAL

// RK4 stage modes of the fused kernel
enum StageMode { MODE_RHS = 0, MODE_S1 = 1, MODE_S23 = 2, MODE_S4 = 3 };

struct StageArgs {
  DevGrid g;
  Coef c;
  AlgebraParams ap;
  const double* __restrict__ U;    // stencil input (stage state)
  const double* __restrict__ U0;   // U_n (pointwise) -- MODE_S1/S23/S4
  double* U0w;                     // U_n written in MODE_S4
  double* out;                     // MODE_RHS: rhs;  MODE_S1/S23: U_next
  double* acc;                     // accumulator
  const double* __restrict__ prim; // fluid primitives [4][pts] (fluid only)
  const double* __restrict__ flux; // fluid face fluxes [3][4][pts] (fluid only)
  double* D;                       // derivative-pass output [NDER][pts] (see stage_kernel.cuh)
  double cdt;                      // dt * c_{s+1}, or dt/6 in MODE_S4
  double bk;                       // accumulator weight (2 for stages 2, 3)
  int f_lo, f_hi;                  // derivative pass: only fields f_lo <= f < f_hi (f_hi = 0: all)
  int k_lo, k_cnt;                 // algebra pass: only planes k_lo .. k_lo + k_cnt - 1 (k_cnt = 0: all)
  int skip_ko;                     // derivative pass: leave the Kreiss-Oliger slots of D unwritten
  const long long* __restrict__ L; // limb copy of U (stage_int.cuh); null: the FP64 derivative pass
  const int* __restrict__ E;       // reference exponent of each limb slot
  unsigned* E_rec;                 // algebra pass, stages 1-3: records the largest biased exponent of
                                   // each limb slot of U_next at E_rec[32 slot] (null: no record)
};

// Doubles per point of the derivative-pass buffer: first and second
// derivatives plus the Kreiss-Oliger term of every non-fluid field.
inline int nder(int scalar) { return 3 * (24 + 2 * scalar) + 6 * (11 + scalar) + 24 + 2 * scalar; }

// One work item of a batch: instance `inst`; for 2D tiles (a, b, c) = (block
// column, block row, z-plane), for linear runs a = first point index.
struct BatchTile {
  int inst, a, b, c;
};
enum BatchMapping { BATCH_MAP_TILE2D = 0, BATCH_MAP_LINEAR = 1 };

struct ConstraintArgs {
  DevGrid g;
  Coef c;
  AlgebraParams ap;
  const double* __restrict__ U;
  const double* __restrict__ prim;
  double* hm;        // [4][pts] or null
  double* partial;   // [nblocks][8]: sum of squares (4) and max abs (4)
};

#ifndef COSMOS_IDERIV_MIN_BLOCKS
#define COSMOS_IDERIV_MIN_BLOCKS 4  // integer derivative pass: resident blocks (of BX x DBY threads) per SM
#endif

// Launchers implemented per matter variant (stage_<variant>.cu).
cudaError_t launch_stage_vac(const StageArgs& a, int mode, cudaStream_t s);
cudaError_t launch_stage_fluid(const StageArgs& a, int mode, cudaStream_t s);
cudaError_t launch_stage_scalar(const StageArgs& a, int mode, cudaStream_t s);
cudaError_t launch_stage_fluid_scalar(const StageArgs& a, int mode, cudaStream_t s);
// batched stage: derivative pass over the BX x DBY tile list (dtiles), algebra
// pass over the tuned work list (tiles, mapping)
// (last two: resident blocks of the integer derivative pass, 0 for the FP64
// pass; whether near_indices holds for every grid of the batch)
typedef cudaError_t (*BatchStageLauncher)(const StageArgs*, const BatchTile*, long, int, const double*, int, dim3,
                                          dim3, cudaStream_t, const BatchTile*, long, int, bool);
cudaError_t launch_batch_stage_vac(const StageArgs*, const BatchTile*, long, int, const double*, int, dim3, dim3,
                                   cudaStream_t, const BatchTile*, long, int, bool);
cudaError_t launch_batch_stage_fluid(const StageArgs*, const BatchTile*, long, int, const double*, int, dim3, dim3,
                                     cudaStream_t, const BatchTile*, long, int, bool);
cudaError_t launch_batch_stage_scalar(const StageArgs*, const BatchTile*, long, int, const double*, int, dim3, dim3,
                                      cudaStream_t, const BatchTile*, long, int, bool);
cudaError_t launch_batch_stage_fluid_scalar(const StageArgs*, const BatchTile*, long, int, const double*, int, dim3,
                                            dim3, cudaStream_t, const BatchTile*, long, int, bool);
cudaError_t launch_batch_fluid(const StageArgs* args, const BatchTile* tiles, long ntiles, int mapping, double w,
                               dim3 grid, dim3 block, cudaStream_t s);
cudaError_t launch_constraints_vac(const ConstraintArgs& a, cudaStream_t s);
cudaError_t launch_constraints_fluid(const ConstraintArgs& a, cudaStream_t s);
cudaError_t launch_constraints_scalar(const ConstraintArgs& a, cudaStream_t s);
cudaError_t launch_constraints_fluid_scalar(const ConstraintArgs& a, cudaStream_t s);

// adjoint_<variant>.cu
struct VjpArgs;
cudaError_t launch_vjp_vac(const VjpArgs& a, cudaStream_t s);
cudaError_t launch_vjp_fluid(const VjpArgs& a, cudaStream_t s);
cudaError_t launch_vjp_scalar(const VjpArgs& a, cudaStream_t s);
cudaError_t launch_vjp_fluid_scalar(const VjpArgs& a, cudaStream_t s);
cudaError_t launch_init_zeta_vjp(const DevGrid& g, const Coef& c, const AlgebraParams& ap, const double* U,
                                 const double* lam, double* CB10, int fluid, double* zbar, cudaStream_t s);

// limbs.cu: exponents of limb slots s_lo .. s_hi - 1 of U and its limb copy
// (slot s = field s, or s + 4 past the fluid fields when the fluid is on)
cudaError_t launch_limbs(const DevGrid& g, const double* U, int fluid, int s_lo, int s_hi, int* E, long long* L,
                         cudaStream_t s);
// the limb copy with given exponents E (no scan); the exponent scan alone
cudaError_t launch_to_limbs(const DevGrid& g, const double* U, int fluid, int s_lo, int s_hi, const int* E,
                            long long* L, cudaStream_t s);
cudaError_t launch_field_exponents(const DevGrid& g, const double* U, int fluid, int s_lo, int s_hi, int* E,
                                   cudaStream_t s);
// E[s] = rec[32 s] and rec[32 s] = 0 for s < nslot (the exponents an algebra pass recorded)
cudaError_t launch_exponents_from_record(unsigned* rec, int* E, int nslot, cudaStream_t s);
// the batched limb copy with the exponents already in args[i].E
cudaError_t launch_batch_to_limbs(const StageArgs* args, int n, int nslot, int fluid, cudaStream_t s);
// the same for every instance of a batch (args[i] = instance i's stage arguments;
// E_all = the n x nslot exponents, contiguous, args[i].E = E_all + i nslot)
cudaError_t launch_batch_limbs(const StageArgs* args, int n, int nslot, int fluid, int* E_all, cudaStream_t s);

// fluid.cu
cudaError_t launch_fluid_prim(const DevGrid& g, const double* U, double* prim, double w, cudaStream_t s);
cudaError_t launch_fluid_flux(const DevGrid& g, const double* U, const double* prim, double* flux, double w,
                              int nf_offset_fluid, cudaStream_t s);

inline dim3 point_grid(const DevGrid& g) { return dim3((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz); }
// integer derivative pass: one BX x DBY tile of one z-plane per block
inline dim3 ideriv_grid(const DevGrid& g) { return dim3((g.nx + BX - 1) / BX, (g.ny + DBY - 1) / DBY, g.nz); }
// Every index the integer derivative pass forms for a tile lies in [-n, 2n)
// along each axis, so one compare and select wraps it (stage_int.cuh,
// wrap_near): x in [i0 - 3, i0 + BX + 2] with i0 <= nx - 1, y in
// [j0 - 3, j0 + DBY + 2] with j0 <= ny - 1, z in [k - 3, k + 3] with k <= nz - 1.
__host__ __device__ inline bool near_indices(const DevGrid& g) { return g.nx >= BX + 3 && g.ny >= DBY + 3 && g.nz >= 3; }

}  // namespace cosmos

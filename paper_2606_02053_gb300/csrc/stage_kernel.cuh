// BSSN right-hand side + RK4 stage, as two passes per stage:
//
//  * derivative pass: for one BX x DBY tile of a z-plane, every 4th-order
//    centred first and second derivative the algebra needs and the
//    6th-derivative Kreiss-Oliger term of every non-fluid field, written to
//    the derivative buffer D.  The launchers run it in exact integer
//    arithmetic on a fixed-point copy of the state (stage_int.cuh:
//    ideriv_kernel, batch_ideriv_kernel); the launchers refuse arguments
//    without that copy;
//  * algebra pass (stage_kernel, batch_stage_kernel): one point per thread,
//    the generated pointwise BSSN + matter algebra on the state and D, the KO
//    term or the Kurganov-Tadmor flux divergence, and the RK4 stage combine.
//
// Every stencil is written so that its large cancellations happen in exact
// neighbour differences.  Also here: the constraint kernel and the per-variant
// launchers (COSMOS_DEFINE_VARIANT).
#pragma once

#include "common.cuh"

#ifndef COSMOS_STAGE_MIN_BLOCKS
#define COSMOS_STAGE_MIN_BLOCKS 3  // resident 128-thread blocks per SM the register budget is sized for
#endif

namespace cosmos {

template <int D>
__device__ __forceinline__ long disp(const Nbr& n, int o) {
  if (D == 0) return n.z[3] + n.y[3] + n.x[o + 3];
  if (D == 1) return n.z[3] + n.y[o + 3] + n.x[3];
  return n.z[o + 3] + n.y[3] + n.x[3];
}

template <int A, int B>
__device__ __forceinline__ long disp2(const Nbr& n, int oa, int ob) {
  int o[3] = {0, 0, 0};
  o[A] = oa;
  o[B] = ob;
  return n.z[o[2] + 3] + n.y[o[1] + 3] + n.x[o[0] + 3];
}

// D_d f = a (f+1 - f-1) - b (f+2 - f-2)
template <int D>
__device__ __forceinline__ double fd1(const double* __restrict__ F, const Nbr& n, const Coef& c) {
  const double a = ldg(F, disp<D>(n, 1)) - ldg(F, disp<D>(n, -1));
  const double b = ldg(F, disp<D>(n, 2)) - ldg(F, disp<D>(n, -2));
  return a * c.d1a[D] - b * c.d1b[D];
}

// D_dd f = a ((f+1 - f0) + (f-1 - f0)) - b ((f+2 - f0) + (f-2 - f0))
template <int D>
__device__ __forceinline__ double fd2(const double* __restrict__ F, const Nbr& n, const Coef& c, double f0) {
  const double s1 = (ldg(F, disp<D>(n, 1)) - f0) + (ldg(F, disp<D>(n, -1)) - f0);
  const double s2 = (ldg(F, disp<D>(n, 2)) - f0) + (ldg(F, disp<D>(n, -2)) - f0);
  return s1 * c.d2a[D] - s2 * c.d2b[D];
}

// D_A D_B f = [64 Q11 - 8 (Q12 + Q21) + Q22] / (144 h_A h_B),
// Q_pq = (f(p, q) - f(-p, q)) - (f(p, -q) - f(-p, -q))  (the 16-point product stencil)
template <int A, int B>
__device__ __forceinline__ double fdmix(const double* __restrict__ F, const Nbr& n, double cm) {
  double q[2][2];
#pragma unroll
  for (int p = 1; p <= 2; ++p)
#pragma unroll
    for (int r = 1; r <= 2; ++r) {
      const double u = ldg(F, disp2<A, B>(n, p, r)) - ldg(F, disp2<A, B>(n, -p, r));
      const double v = ldg(F, disp2<A, B>(n, p, -r)) - ldg(F, disp2<A, B>(n, -p, -r));
      q[p - 1][r - 1] = u - v;
    }
  const double cross = q[0][1] + q[1][0];
  return q[0][0] * (64.0 * cm) + (q[1][1] * cm - cross * (8.0 * cm));
}

// rhs + sigma/64 sum_d (1/h_d) [ (f+3 + f-3) - 6 (f+2 + f-2) + 15 (f+1 + f-1) - 20 f0 ]
// grouped as (s3 - s2) - 5 (s2 - s1) + 10 (s1 - 2 f0), s_k = f+k + f-k: the same
// coefficients, and every bracket is exactly zero when the neighbours equal f0.
template <int D>
__device__ __forceinline__ double ko_dir(const double* __restrict__ F, const Nbr& n, double f0) {
  const double s1 = ldg(F, disp<D>(n, 1)) + ldg(F, disp<D>(n, -1));
  const double s2 = ldg(F, disp<D>(n, 2)) + ldg(F, disp<D>(n, -2));
  const double s3 = ldg(F, disp<D>(n, 3)) + ldg(F, disp<D>(n, -3));
  const double t = fma(-2.0, f0, s1);
  return fma(10.0, t, fma(-5.0, s2 - s1, s3 - s2));
}

__device__ __forceinline__ double ko_add(const double* __restrict__ F, const Nbr& n, const Coef& c, double f0,
                                         double r) {
  r = fma(c.ko[0], ko_dir<0>(F, n, f0), r);
  r = fma(c.ko[1], ko_dir<1>(F, n, f0), r);
  r = fma(c.ko[2], ko_dir<2>(F, n, f0), r);
  return r;
}

// Kreiss-Oliger term of a field on a grid with equal spacing along the three
// axes (one coefficient c.ko[0]): the bracket is linear in s_k, so the three
// axes are summed first, P_k = sum_d (f(+k e_d) + f(-k e_d)), and combined once:
// (P3 - P2) - 5 (P2 - P1) + 10 (P1 - 6 f0).  For a constant field every P_k and
// 6 f0 are the same single rounding of 6 f0, so each bracket is exactly zero.
// ko_bracket returns the bracket; the term is c.ko[0] times it.
__device__ __forceinline__ double ko_bracket(const double* __restrict__ F, const Nbr& n, double f0) {
  double P[3];
#pragma unroll
  for (int k = 1; k <= 3; ++k)
    P[k - 1] = ((ldg(F, disp<0>(n, k)) + ldg(F, disp<0>(n, -k))) + (ldg(F, disp<1>(n, k)) + ldg(F, disp<1>(n, -k)))) +
               (ldg(F, disp<2>(n, k)) + ldg(F, disp<2>(n, -k)));
  const double t = P[0] - __dmul_rn(6.0, f0);  // __dmul_rn: the product is rounded, never fused
  return fma(10.0, t, fma(-5.0, P[1] - P[0], P[2] - P[1]));
}

__device__ __forceinline__ double ko_uniform(const double* __restrict__ F, const Nbr& n, const Coef& c, double f0) {
  return c.ko[0] * ko_bracket(F, n, f0);
}


// Inputs of the generated algebra at one point (layout documented in codegen/bssn.py).
template <class T>
__device__ __forceinline__ void gather(const double* __restrict__ U, const double* __restrict__ prim, const Nbr& n,
                                       const Coef& c, long fs, double* in) {
#pragma unroll
  for (int f = 0; f < T::NF; ++f) in[f] = ldg(U + (long)f * fs, n.c);
#pragma unroll
  for (int m = 0; m < T::ND1; ++m) {
    const double* F = U + (long)T::d1_field(m) * fs;
    in[T::NF + 3 * m + 0] = fd1<0>(F, n, c);
    in[T::NF + 3 * m + 1] = fd1<1>(F, n, c);
    in[T::NF + 3 * m + 2] = fd1<2>(F, n, c);
  }
#pragma unroll
  for (int m = 0; m < T::ND2; ++m) {
    const int f = T::d2_field(m);
    const double* F = U + (long)f * fs;
    const double f0 = in[f];
    const int b = T::NF + 3 * T::ND1 + 6 * m;
    in[b + 0] = fd2<0>(F, n, c, f0);
    in[b + 1] = fdmix<0, 1>(F, n, c.mix[0]);
    in[b + 2] = fdmix<0, 2>(F, n, c.mix[1]);
    in[b + 3] = fd2<1>(F, n, c, f0);
    in[b + 4] = fdmix<1, 2>(F, n, c.mix[2]);
    in[b + 5] = fd2<2>(F, n, c, f0);
  }
  if constexpr (T::FLUID) in[T::NIN - 1] = ldg(prim, n.c);
}

// ---------------------------------------------------------------------------
// Stage = derivative pass + algebra pass.
//
// Derivative pass (one BX x DBY tile of one z-plane per block): writes every
// finite difference the algebra needs, and the Kreiss-Oliger term of every
// non-fluid field, into D (layout: D[3 m + d] first derivative d of the m-th
// first-derivative field, D[3 ND1 + 6 m + p] second derivative p of the m-th
// second-derivative field, D[NDER0 + ko_slot(f)] KO term of field f, divided by
// c.ko[0] when the spacing is equal -- see Coef::ko_s).  For the
// second-derivative fields the first derivatives along y and z are computed
// once per tile point (with a 2-point halo) into shared memory, and the mixed
// derivatives are D_x(D_y f), D_x(D_z f), D_y(D_z f) of those values; along x
// the neighbour differences d_k = f(+-k) - f0 are shared by D1, D2 and KO.
// Optional restrictions (StageArgs): a field range f_lo .. f_hi, no KO slots
// (skip_ko, for the reverse mode), and for the algebra pass a plane range.
// Algebra pass (any point mapping): the generated pointwise algebra on the
// state values and D, KO and the fluid flux divergence, and the RK4 combine.
// ---------------------------------------------------------------------------
constexpr int TXH = BX + 4;  // tile width with the x halo

template <class T>
__device__ __forceinline__ int ko_slot(int f) {
  return (T::FLUID && f >= 28) ? f - 4 : f;
}

__device__ __forceinline__ long plane_off(const DevGrid& g, int x, int y, int k) {
  return ((long)wrap_index(k, g.nz) * g.ny + wrap_index(y, g.ny)) * g.pitch + wrap_index(x, g.nx);
}

}  // namespace cosmos

#include "stage_int.cuh"

namespace cosmos {

// Inputs of the algebra pass at one point, read from global memory where the
// generated code uses them (state values, then the derivative buffer, then the
// fluid density), so that no input has to stay live in a register.
template <class T>
struct AlgIn {
  const double* __restrict__ U;
  const double* __restrict__ D;
  const double* __restrict__ prim;
  long fs, c;
  __device__ __forceinline__ double operator[](int k) const {
    constexpr int NDER0 = 3 * T::ND1 + 6 * T::ND2;
    if (k < T::NF) return ldg(U + (long)k * fs, c);
    if (k < T::NF + NDER0) return ldg(D + (long)(k - T::NF) * fs, c);
    return ldg(prim, c);
  }
};

// The largest biased exponent of v over the warp's active lanes into *E (one
// atomic per warp): the next stage's reference exponent without a scan of the
// state (the exponent field of the stored value, as field_exponent_kernel reads).
__device__ __forceinline__ void record_exponent(unsigned* E, double v) {
  const unsigned e = (unsigned)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FFu);
  const unsigned mask = __activemask();
  const unsigned m = __reduce_max_sync(mask, e);
  unsigned lane;
  asm("mov.u32 %0, %%laneid;" : "=r"(lane));
  if (lane == (unsigned)(__ffs(mask) - 1)) atomicMax(E, m);
}

// Output side of the algebra pass: out[f] = r adds the Kreiss-Oliger term (or
// the fluid flux divergence) and applies the RK4 stage combine of MODE, as
// soon as the generated code has the value.
template <class T, int MODE>
struct AlgOut {
  const StageArgs& a;
  long fs, c;
  long cm[3];
  struct Slot {
    const AlgOut& o;
    int f;
    __device__ __forceinline__ void operator=(double r) const {
      const StageArgs& a = o.a;
      const long fs = o.fs, c = o.c;
      constexpr int NDER0 = 3 * T::ND1 + 6 * T::ND2;
      if (T::FLUID && f >= 24 && f < 28) {
        const double* H = a.flux + (long)(f - 24) * fs;  // direction d at H + 4 d fs
        r -= (ldg(H, c) - ldg(H, o.cm[0])) * a.c.ih[0];
        r -= (ldg(H + 4 * fs, c) - ldg(H + 4 * fs, o.cm[1])) * a.c.ih[1];
        r -= (ldg(H + 8 * fs, c) - ldg(H + 8 * fs, o.cm[2])) * a.c.ih[2];
      } else {
        r = fma(a.c.ko_s, ldg(a.D + (long)(NDER0 + ko_slot<T>(f)) * fs, c), r);  // see Coef::ko_s
      }
      const long ofs = (long)f * fs + c;
      if constexpr (MODE == MODE_RHS) {
        a.out[ofs] = r;
      } else if constexpr (MODE == MODE_S1) {
        const double v = fma(a.cdt, r, ldg(a.U0, ofs));
        a.out[ofs] = v;
        a.acc[ofs] = r;
        if (a.E_rec && !(T::FLUID && f >= 24 && f < 28)) record_exponent(a.E_rec + 32 * ko_slot<T>(f), v);
      } else if constexpr (MODE == MODE_S23) {
        const double v = fma(a.cdt, r, ldg(a.U0, ofs));
        a.out[ofs] = v;
        a.acc[ofs] = fma(a.bk, r, a.acc[ofs]);
        if (a.E_rec && !(T::FLUID && f >= 24 && f < 28)) record_exponent(a.E_rec + 32 * ko_slot<T>(f), v);
      } else {
        a.U0w[ofs] = fma(a.cdt, a.acc[ofs] + r, a.U0w[ofs]);
      }
    }
  };
  __device__ __forceinline__ Slot operator[](int f) const { return Slot{*this, f}; }
};

// Algebra pass at one grid point (i, j, k).
template <class T, int MODE>
__device__ __forceinline__ void alg_point(const StageArgs& a, const AlgebraParams& ap, int i, int j, int k) {
  const long fs = a.g.fstride;
  const long c = ((long)k * a.g.ny + j) * a.g.pitch + i;
  const AlgIn<T> in{a.U, a.D, a.prim, fs, c};
  AlgOut<T, MODE> out{a, fs, c, {0, 0, 0}};
  if constexpr (T::FLUID) {
    out.cm[0] = c - i + wrap_index(i - 1, a.g.nx);
    out.cm[1] = c + (long)(wrap_index(j - 1, a.g.ny) - j) * a.g.pitch;
    out.cm[2] = c + (long)(wrap_index(k - 1, a.g.nz) - k) * a.g.pitch * a.g.ny;
  }
  T::rhs(in, out, ap);
}

template <class T, int MODE>
__global__ void __launch_bounds__(BX* BY, COSMOS_STAGE_MIN_BLOCKS) stage_kernel(const StageArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z + a.k_lo;
  if (i >= a.g.nx || j >= a.g.ny) return;
  alg_point<T, MODE>(a, a.ap, i, j, k);
}

// Point (i, j, k) of work item `t` (thread `lane` of the block) of a batch:
// 2D tiles of blockDim.x x blockDim.y points in one z-plane, or runs of
// blockDim.x * blockDim.y consecutive points in memory order.  Returns false
// for a thread past the grid edge.
__device__ __forceinline__ bool batch_point(const BatchTile& t, const DevGrid& g, int mapping, int& i, int& j,
                                            int& k) {
  if (mapping == BATCH_MAP_TILE2D) {
    i = t.a * blockDim.x + threadIdx.x;
    j = t.b * blockDim.y + threadIdx.y;
    k = t.c;
    return i < g.nx && j < g.ny;
  }
  const long p = (long)t.a + threadIdx.y * blockDim.x + threadIdx.x;
  const long npts = (long)g.nx * g.ny * g.nz;
  if (p >= npts) return false;
  i = (int)(p % g.nx);
  j = (int)((p / g.nx) % g.ny);
  k = (int)(p / ((long)g.nx * g.ny));
  return true;
}

// Persistent batched algebra pass: blocks stride over the flat work list of
// all instances; instance `inst` uses args[inst] with K_ref taken from kref.
// The instance's arguments are copied to shared memory when the instance
// changes: read from there they cannot alias the pass's stores.
template <class T, int MODE>
__global__ void __launch_bounds__(BX* BY, COSMOS_STAGE_MIN_BLOCKS)
    batch_stage_kernel(const StageArgs* __restrict__ args, const BatchTile* __restrict__ tiles, long ntiles,
                       int mapping, const double* __restrict__ kref) {
  __shared__ StageArgs sa;
  static_assert(sizeof(StageArgs) % sizeof(long long) == 0, "StageArgs is copied in 8-byte words");
  constexpr int W = (int)(sizeof(StageArgs) / sizeof(long long));
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
  int inst = -1;
  for (long w = blockIdx.x; w < ntiles; w += gridDim.x) {
    const BatchTile t = tiles[w];
    if (t.inst != inst) {  // uniform across the block
      __syncthreads();     // every thread is done with the previous instance's arguments
      const long long* src = reinterpret_cast<const long long*>(args + t.inst);
      long long* dst = reinterpret_cast<long long*>(&sa);
      for (int q = tid; q < W; q += nthr) dst[q] = src[q];
      __syncthreads();
      inst = t.inst;
    }
    AlgebraParams ap = sa.ap;
    ap.Kref = kref[t.inst];
    int i, j, k;
    if (batch_point(t, sa.g, mapping, i, j, k)) alg_point<T, MODE>(sa, ap, i, j, k);
  }
}

// Constraints H, M^i per point plus per-block partial norms.
template <class T>
__global__ void __launch_bounds__(BX* BY, 2) constraint_kernel(const ConstraintArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const bool valid = (i < a.g.nx) && (j < a.g.ny);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (valid) {
    const Nbr n = make_nbr(a.g, i, j, k);
    const long fs = a.g.fstride;
    double in[T::NIN];
    gather<T>(a.U, a.prim, n, a.c, fs, in);
    T::constraints(in, v, a.ap);
    if (a.hm) {
#pragma unroll
      for (int m = 0; m < 4; ++m) a.hm[(long)m * fs + n.c] = v[m];
    }
  }
  double r[8];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    r[m] = v[m] * v[m];
    r[4 + m] = fabs(v[m]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      r[m] += __shfl_down_sync(0xffffffffu, r[m], off);
      r[4 + m] = fmax(r[4 + m], __shfl_down_sync(0xffffffffu, r[4 + m], off));
    }
  }
  __shared__ double red[BY][8];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < 8; ++m) red[threadIdx.y][m] = r[m];
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double s[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) s[m] = red[0][m];
    for (int w = 1; w < BY; ++w) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        s[m] += red[w][m];
        s[4 + m] = fmax(s[4 + m], red[w][4 + m]);
      }
    }
    const long b = ((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int m = 0; m < 8; ++m) a.partial[b * 8 + m] = s[m];
  }
}

#define COSMOS_DEFINE_VARIANT(NAME, IS_FLUID, IS_SCALAR)                                                          \
  struct T_##NAME {                                                                                             \
    static constexpr int NF = alg_##NAME::NF, ND1 = alg_##NAME::ND1, ND2 = alg_##NAME::ND2,                     \
                         NIN = alg_##NAME::NIN;                                                                 \
    static constexpr bool FLUID = IS_FLUID, SCALAR = IS_SCALAR;                                                 \
    __device__ static constexpr int d1_field(int m) { return alg_##NAME::d1_field(m); }                        \
    __device__ static constexpr int d2_field(int m) { return alg_##NAME::d2_field(m); }                        \
    __device__ static constexpr int d1_slot(int f) { return alg_##NAME::d1_slot(f); }                          \
    __device__ static constexpr int d2_slot(int f) { return alg_##NAME::d2_slot(f); }                          \
    template <class In, class Out>                                                                              \
    __device__ static __forceinline__ void rhs(const In& in, Out&& out, const AlgebraParams& p) {               \
      alg_##NAME::rhs(in, out, p);                                                                              \
    }                                                                                                           \
    __device__ static __forceinline__ void constraints(const double* in, double* out, const AlgebraParams& p) {  \
      alg_##NAME::constraints(in, out, p);                                                                      \
    }                                                                                                           \
  };                                                                                                            \
  cudaError_t launch_stage_##NAME(const StageArgs& a, int mode, cudaStream_t s) {                               \
    dim3 grid = point_grid(a.g), block(BX, BY);                                                                \
    if (a.k_cnt > 0) grid.z = a.k_cnt;                                                                          \
    if (mode < 0 || !(mode & 8)) {                                                                            \
      if (!a.L) return cudaErrorInvalidValue; /* the derivative pass reads the limb copy */                     \
      if (near_indices(a.g))                                                                                    \
        ideriv_kernel<T_##NAME, true><<<ideriv_grid(a.g), dim3(BX, DBY), 0, s>>>(a);                            \
      else                                                                                                      \
        ideriv_kernel<T_##NAME, false><<<ideriv_grid(a.g), dim3(BX, DBY), 0, s>>>(a);                           \
    }                                                                                                           \
    if (mode < 0) return cudaGetLastError();                                                                    \
    switch (mode & 7) {                                                                                             \
      case MODE_RHS: stage_kernel<T_##NAME, MODE_RHS><<<grid, block, 0, s>>>(a); break;                        \
      case MODE_S1: stage_kernel<T_##NAME, MODE_S1><<<grid, block, 0, s>>>(a); break;                          \
      case MODE_S23: stage_kernel<T_##NAME, MODE_S23><<<grid, block, 0, s>>>(a); break;                        \
      default: stage_kernel<T_##NAME, MODE_S4><<<grid, block, 0, s>>>(a); break;                               \
    }                                                                                                           \
    return cudaGetLastError();                                                                                  \
  }                                                                                                             \
  cudaError_t launch_batch_stage_##NAME(const StageArgs* args, const BatchTile* tiles, long ntiles, int mapping,  \
                                        const double* kref, int mode, dim3 grid, dim3 block, cudaStream_t s,      \
                                        const BatchTile* dtiles, long ndtiles, int ideriv_blocks,                 \
                                        bool ideriv_near) {                                                       \
    if (ideriv_blocks <= 0) return cudaErrorInvalidValue;                                                       \
    if (ideriv_near)                                                                                            \
      batch_ideriv_kernel<T_##NAME, true><<<ideriv_blocks, dim3(BX, DBY), 0, s>>>(args, dtiles, ndtiles);       \
    else                                                                                                        \
      batch_ideriv_kernel<T_##NAME, false><<<ideriv_blocks, dim3(BX, DBY), 0, s>>>(args, dtiles, ndtiles);      \
    switch (mode) {                                                                                             \
      case MODE_S1:                                                                                             \
        batch_stage_kernel<T_##NAME, MODE_S1><<<grid, block, 0, s>>>(args, tiles, ntiles, mapping, kref);       \
        break;                                                                                                  \
      case MODE_S23:                                                                                            \
        batch_stage_kernel<T_##NAME, MODE_S23><<<grid, block, 0, s>>>(args, tiles, ntiles, mapping, kref);      \
        break;                                                                                                  \
      default:                                                                                                  \
        batch_stage_kernel<T_##NAME, MODE_S4><<<grid, block, 0, s>>>(args, tiles, ntiles, mapping, kref);       \
        break;                                                                                                  \
    }                                                                                                           \
    return cudaGetLastError();                                                                                  \
  }                                                                                                             \
  cudaError_t launch_constraints_##NAME(const ConstraintArgs& a, cudaStream_t s) {                              \
    constraint_kernel<T_##NAME><<<point_grid(a.g), dim3(BX, BY), 0, s>>>(a);                                    \
    return cudaGetLastError();                                                                                  \
  }

}  // namespace cosmos

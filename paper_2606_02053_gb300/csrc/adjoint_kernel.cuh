// Reverse mode (vector-Jacobian product) of the right-hand side F(U):
//   v = (dF/dU)^T w
// F(U)(p) = A(inputs at p) + KO(U)(p) - sum_d (H_d(p) - H_d(p - e_d)) / h_d,
// the inputs being U(p) and finite differences of U around p.  On a periodic
// grid the centred stencils transpose to D_d^T = -D_d, D_dd^T = D_dd,
// (D_a D_b)^T = D_a D_b and KO^T = KO, so
//   v_f = abar_f - sum_d D_d(dbar_{f,d}) + sum_ab D_ab(ddbar_{f,ab}) + KO(w_f) + (fluid terms)
// with (abar, dbar, ddbar) the cotangents of the algebra inputs (pass 1, the
// generated reverse of the pointwise algebra) and the fluid terms from the
// reverse of the face fluxes and of the primitive recovery.
#pragma once

#include "stage_kernel.cuh"

namespace cosmos {

struct VjpArgs {
  DevGrid g;
  Coef c;
  AlgebraParams ap;
  FluidParams fp;
  const double* __restrict__ U;     // linearisation point
  const double* __restrict__ prim;  // primitives at U (fluid)
  const double* __restrict__ W;     // cotangent of F(U) (state layout)
  const double* __restrict__ D;     // derivative-pass output at U (KO slots unused)
  double* CB;                       // [NIN][pts] input cotangents (pass 1)
  double* FC;                       // [3][34][pts] face-input cotangents (fluid)
  double* VF;                       // [nf][pts] fluid contributions to v (fluid)
  // pass 2 outputs:  lam += v;  knext = a_lam * lam0 + a_v * v  (knext optional)
  const double* __restrict__ lam0;
  double* lam;
  double* knext;
  double a_lam, a_v;
};

// Inputs of the reverse algebra at one point: the forward inputs (state,
// derivative buffer, fluid density) followed by the cotangents W of the
// outputs, each read from global memory where the generated code uses it.
template <class T>
struct VjpIn {
  const VjpArgs& a;
  long fs, c;
  __device__ __forceinline__ double operator[](int k) const {
    constexpr int NDER0 = 3 * T::ND1 + 6 * T::ND2;
    if (k < T::NF) return ldg(a.U + (long)k * fs, c);
    if (k < T::NF + NDER0) return ldg(a.D + (long)(k - T::NF) * fs, c);
    if (k < T::NIN) return ldg(a.prim, c);
    return ldg(a.W + (long)(k - T::NIN) * fs, c);
  }
};

// Input cotangents, stored to CB as soon as the generated code has each one.
struct VjpOut {
  double* CB;
  long fs, c;
  struct Slot {
    double* p;
    __device__ __forceinline__ void operator=(double v) const { *p = v; }
  };
  __device__ __forceinline__ Slot operator[](int m) const { return Slot{CB + (long)m * fs + c}; }
};

#ifndef COSMOS_VJP_MIN_BLOCKS
#define COSMOS_VJP_MIN_BLOCKS 3  // reverse algebra: resident 128-thread blocks per SM the registers are sized for
#endif

template <class T>
__global__ void __launch_bounds__(BX* BY, COSMOS_VJP_MIN_BLOCKS) vjp_pass1_kernel(const VjpArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.g.nx || j >= a.g.ny) return;
  const long fs = a.g.fstride;
  const long c = ((long)k * a.g.ny + j) * a.g.pitch + i;
  const VjpIn<T> in{a, fs, c};
  VjpOut out{a.CB, fs, c};
  T::rhs_vjp(in, out, a.ap);
}

// Face-flux reverse: H_d(p) enters F at p (-1/h) and at p + e_d (+1/h).
template <int D>
__device__ __forceinline__ void face_vjp(const VjpArgs& a, const Nbr& n) {
  const long fs = a.g.fstride;
  double in[34 + 4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const long off = disp<D>(n, o - 1);
#pragma unroll
    for (int m = 0; m < 4; ++m) in[4 * o + m] = ldg(a.prim + m * fs, off);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const long off = disp<D>(n, s);
    double* q = in + 16 + 9 * s;
    q[0] = ldg(a.U, off);
    q[1] = ldg(a.U + 17 * fs, off);
    q[2] = ldg(a.U + (18 + D) * fs, off);
#pragma unroll
    for (int m = 0; m < 6; ++m) q[3 + m] = ldg(a.U + (1 + m) * fs, off);
  }
  const long up = disp<D>(n, 1);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const double* Wm = a.W + (long)(24 + m) * fs;
    in[34 + m] = (ldg(Wm, up) - ldg(Wm, n.c)) * a.c.ih[D];
  }
  double out[34];
  if (D == 0) fluid_face_flux_0_vjp(in, out, a.fp);
  if (D == 1) fluid_face_flux_1_vjp(in, out, a.fp);
  if (D == 2) fluid_face_flux_2_vjp(in, out, a.fp);
#pragma unroll
  for (int m = 0; m < 34; ++m) a.FC[(long)(34 * D + m) * fs + n.c] = out[m];
}

static __global__ void __launch_bounds__(BX* BY) vjp_face_kernel(const VjpArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.g.nx || j >= a.g.ny) return;
  const Nbr n = make_nbr(a.g, i, j, k);
  face_vjp<0>(a, n);
  face_vjp<1>(a, n);
  face_vjp<2>(a, n);
}

// Per cell: gather the face-input cotangents that refer to this cell, add the
// algebra's d/d rho, run the reverse of the primitive recovery, and store the
// fluid contributions to v (chi, gt, alpha, beta, tau, S) in VF.
template <int D>
__device__ __forceinline__ void gather_face_cot(const VjpArgs& a, const Nbr& n, double qb[4], double mb[9]) {
  const long fs = a.g.fstride;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const long off = disp<D>(n, 1 - o);  // face p = c - (o - 1) e_d sees cell c as its input o
#pragma unroll
    for (int m = 0; m < 4; ++m) qb[m] += ldg(a.FC + (long)(34 * D + 4 * o + m) * fs, off);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const long off = disp<D>(n, -s);  // face p = c - s e_d sees cell c as its metric side s
#pragma unroll
    for (int m = 0; m < 9; ++m) mb[m] += ldg(a.FC + (long)(34 * D + 16 + 9 * s + m) * fs, off);
  }
}

template <class T>
__global__ void __launch_bounds__(BX* BY) vjp_cell_kernel(const VjpArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.g.nx || j >= a.g.ny) return;
  const Nbr n = make_nbr(a.g, i, j, k);
  const long fs = a.g.fstride;
  double qb[4] = {ldg(a.CB + (long)(T::NIN - 1) * fs, n.c), 0.0, 0.0, 0.0};  // d/d rho from the algebra
  double mb[3][9];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int m = 0; m < 9; ++m) mb[d][m] = 0.0;
  gather_face_cot<0>(a, n, qb, mb[0]);
  gather_face_cot<1>(a, n, qb, mb[1]);
  gather_face_cot<2>(a, n, qb, mb[2]);
  double in[11 + 4];
  in[0] = ldg(a.U, n.c);
#pragma unroll
  for (int m = 0; m < 6; ++m) in[1 + m] = ldg(a.U + (1 + m) * fs, n.c);
#pragma unroll
  for (int m = 0; m < 4; ++m) in[7 + m] = ldg(a.U + (24 + m) * fs, n.c);
#pragma unroll
  for (int m = 0; m < 4; ++m) in[11 + m] = qb[m];
  double pb[11];
  fluid_prim_vjp(in, pb, a.fp);
  double vf[T::NF];
#pragma unroll
  for (int f = 0; f < T::NF; ++f) vf[f] = 0.0;
  vf[0] = pb[0] + mb[0][0] + mb[1][0] + mb[2][0];
#pragma unroll
  for (int m = 0; m < 6; ++m) vf[1 + m] = pb[1 + m] + mb[0][3 + m] + mb[1][3 + m] + mb[2][3 + m];
  vf[17] = mb[0][1] + mb[1][1] + mb[2][1];
#pragma unroll
  for (int d = 0; d < 3; ++d) vf[18 + d] = mb[d][2];
#pragma unroll
  for (int m = 0; m < 4; ++m) vf[24 + m] = pb[7 + m];
#pragma unroll
  for (int f = 0; f < T::NF; ++f) a.VF[(long)f * fs + n.c] = vf[f];
}

// Transposed stencils + RK4 reverse-sweep accumulation, one field at a time
// (each v_f depends on the cotangents of field f only).
template <class T>
__global__ void __launch_bounds__(BX* BY, 3) vjp_pass2_kernel(const VjpArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.g.nx || j >= a.g.ny) return;
  const Nbr n = make_nbr(a.g, i, j, k);
  const long fs = a.g.fstride;
  const bool ko_equal = a.c.ko[0] == a.c.ko[1] && a.c.ko[1] == a.c.ko[2];
#pragma unroll 1
  for (int f = 0; f < T::NF; ++f) {
    double v = ldg(a.CB + (long)f * fs, n.c);
    const int m = T::d1_slot(f);
    if (m >= 0) {
      const double* G = a.CB + (long)(T::NF + 3 * m) * fs;
      v -= fd1<0>(G, n, a.c) + fd1<1>(G + fs, n, a.c) + fd1<2>(G + 2 * fs, n, a.c);
    }
    const int m2 = T::d2_slot(f);
    if (m2 >= 0) {
      const double* G = a.CB + (long)(T::NF + 3 * T::ND1 + 6 * m2) * fs;
      double s = fd2<0>(G, n, a.c, ldg(G, n.c));
      s += fdmix<0, 1>(G + fs, n, a.c.mix[0]);
      s += fdmix<0, 2>(G + 2 * fs, n, a.c.mix[1]);
      s += fd2<1>(G + 3 * fs, n, a.c, ldg(G + 3 * fs, n.c));
      s += fdmix<1, 2>(G + 4 * fs, n, a.c.mix[2]);
      s += fd2<2>(G + 5 * fs, n, a.c, ldg(G + 5 * fs, n.c));
      v += s;
    }
    if (!(T::FLUID && f >= 24 && f < 28)) {  // KO is symmetric: KO^T w = KO w
      const double* Wf = a.W + (long)f * fs;
      v = ko_equal ? v + ko_uniform(Wf, n, a.c, ldg(Wf, n.c)) : ko_add(Wf, n, a.c, ldg(Wf, n.c), v);
    }
    if constexpr (T::FLUID) v += ldg(a.VF + (long)f * fs, n.c);
    const long o = (long)f * fs + n.c;
    a.lam[o] += v;
    if (a.knext) a.knext[o] = a.a_lam * ldg(a.lam0, o) + a.a_v * v;
  }
}

// Gather traits for the vacuum layout (used by the initial-data reverse).
struct T_vac_adj {
  static constexpr int NF = alg_vac::NF, ND1 = alg_vac::ND1, ND2 = alg_vac::ND2, NIN = alg_vac::NIN;
  static constexpr bool FLUID = false, SCALAR = false;
  __device__ static constexpr int d1_field(int m) { return alg_vac::d1_field(m); }
  __device__ static constexpr int d2_field(int m) { return alg_vac::d2_field(m); }
};

#define COSMOS_DEFINE_ADJOINT(NAME, IS_FLUID)                                                                     \
  struct A_##NAME {                                                                                             \
    static constexpr int NF = alg_##NAME::NF, ND1 = alg_##NAME::ND1, ND2 = alg_##NAME::ND2,                     \
                         NIN = alg_##NAME::NIN;                                                                 \
    static constexpr bool FLUID = IS_FLUID, SCALAR = false;                                                     \
    __device__ static constexpr int d1_field(int m) { return alg_##NAME::d1_field(m); }                        \
    __device__ static constexpr int d2_field(int m) { return alg_##NAME::d2_field(m); }                        \
    __device__ static constexpr int d1_slot(int f) { return alg_##NAME::d1_slot(f); }                          \
    __device__ static constexpr int d2_slot(int f) { return alg_##NAME::d2_slot(f); }                          \
    template <class In, class Out>                                                                              \
    __device__ static __forceinline__ void rhs_vjp(const In& in, Out&& out, const AlgebraParams& p) {           \
      alg_##NAME::rhs_vjp(in, out, p);                                                                          \
    }                                                                                                           \
  };                                                                                                            \
  cudaError_t launch_vjp_##NAME(const VjpArgs& a, cudaStream_t s) {                                             \
    const dim3 grid = point_grid(a.g), block(BX, BY);                                                          \
    vjp_pass1_kernel<A_##NAME><<<grid, block, 0, s>>>(a);                                                       \
    cudaError_t e = cudaGetLastError();                                                                         \
    if (e != cudaSuccess) return e;                                                                             \
    if (IS_FLUID) {                                                                                             \
      vjp_face_kernel<<<grid, block, 0, s>>>(a);                                                                \
      if ((e = cudaGetLastError()) != cudaSuccess) return e;                                                    \
      vjp_cell_kernel<A_##NAME><<<grid, block, 0, s>>>(a);                                                      \
      if ((e = cudaGetLastError()) != cudaSuccess) return e;                                                    \
    }                                                                                                           \
    vjp_pass2_kernel<A_##NAME><<<grid, block, 0, s>>>(a);                                                       \
    return cudaGetLastError();                                                                                  \
  }

}  // namespace cosmos

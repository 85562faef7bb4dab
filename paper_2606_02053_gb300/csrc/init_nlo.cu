// Initial data at the next-to-leading order of the gradient expansion (id
// kind 3; section "Physical system settings", initial-data paragraph: the
// growing mode of the long-wavelength expansion in eps = k/(aH), up to the
// next-leading order).  Constant-mean-curvature slicing, zero shift, flat FLRW
// background with P = w rho.  From the leading-order data (chi0 = a0^-2
// e^{-2 zeta}, gt = delta, K = -3 H0) and the Ricci tensor R_ij of their
// metric, with M_ij = R_ij - 1/3 delta_ij tr R and delta = chi0 tr R / (6 H0^2):
//   At_ij = 2 chi0 M_ij / ((5 + 3w) H0)
//   gt_ij = (delta_ij + h_ij) / det(delta + h)^{1/3},
//           h_ij = -4 chi0 M_ij / ((5 + 3w)(1 + 3w) H0^2)
//   alpha = 1 - (1 + 3w) delta / (3 (1 + w)),  chi = chi0 (1 + 2 delta / (3 (1 + w)))
// (the growing solution of the trace-free evolution, the lapse that keeps the
// mean curvature constant, the conformal factor that lapse gives), then
// Gt^i = gt^jk Gt^i_jk of the new gt, and the fluid's E and J_i from the
// discrete Hamiltonian and momentum constraints of the final metric.
// Differences are the 4th-order centred ones of the right-hand side.
#include <math.h>
#include <string.h>

#include "host.cuh"
#include "stage_kernel.cuh"

namespace cosmos {

namespace {

// gt, At, alpha of the next order in place (they are not read here) and the new
// chi into chi_new (chi0 at the neighbours is read by other threads).
__global__ void nlo_metric_kernel(const DevGrid g, const Coef c, double H0, double w, double* __restrict__ U,
                                  double* __restrict__ chi_new) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const Nbr n = make_nbr(g, i, j, k);
  const long fs = g.fstride;
  const double* X = U;  // chi0
  const double chi = ldg(X, n.c);
  const double d[3] = {fd1<0>(X, n, c), fd1<1>(X, n, c), fd1<2>(X, n, c)};
  double dd[3][3];
  dd[0][0] = fd2<0>(X, n, c, chi);
  dd[1][1] = fd2<1>(X, n, c, chi);
  dd[2][2] = fd2<2>(X, n, c, chi);
  dd[0][1] = dd[1][0] = fdmix<0, 1>(X, n, c.mix[0]);
  dd[0][2] = dd[2][0] = fdmix<0, 2>(X, n, c.mix[1]);
  dd[1][2] = dd[2][1] = fdmix<1, 2>(X, n, c.mix[2]);
  // Ricci tensor of the conformally flat metric delta_ij / chi (gt = delta, so
  // the conformal Christoffels vanish):
  //   R_ij = (d_i d_j chi + delta_ij lap chi)/(2 chi) - d_i chi d_j chi/(4 chi^2)
  //          - 3 delta_ij |d chi|^2/(4 chi^2)
  const double lap = dd[0][0] + dd[1][1] + dd[2][2];
  const double g2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double R[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const double e = a == b ? 1.0 : 0.0;
      R[a][b] = (dd[a][b] + e * lap) / (2.0 * chi) - d[a] * d[b] / (4.0 * chi * chi) - 3.0 * e * g2 / (4.0 * chi * chi);
    }
  const double trR = R[0][0] + R[1][1] + R[2][2];
  const double delta = chi * trR / (6.0 * H0 * H0);
  double gm[3][3], M[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      M[a][b] = R[a][b] - (a == b ? trR / 3.0 : 0.0);
      gm[a][b] = (a == b ? 1.0 : 0.0) - 4.0 * chi * M[a][b] / ((5.0 + 3.0 * w) * (1.0 + 3.0 * w) * H0 * H0);
    }
  const double det = gm[0][0] * (gm[1][1] * gm[2][2] - gm[1][2] * gm[2][1]) -
                     gm[0][1] * (gm[1][0] * gm[2][2] - gm[1][2] * gm[2][0]) +
                     gm[0][2] * (gm[1][0] * gm[2][1] - gm[1][1] * gm[2][0]);
  const double s = 1.0 / cbrt(det);
  const int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      U[(1 + sym[a][b]) * fs + n.c] = gm[a][b] * s;
      U[(8 + sym[a][b]) * fs + n.c] = 2.0 * chi * M[a][b] / ((5.0 + 3.0 * w) * H0);
    }
  U[17 * fs + n.c] = 1.0 - (1.0 + 3.0 * w) * delta / (3.0 * (1.0 + w));
  chi_new[n.c] = chi * (1.0 + 2.0 * delta / (3.0 * (1.0 + w)));
}

__global__ void copy_field_kernel(const DevGrid g, const double* __restrict__ src, double* __restrict__ dst) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long c = ((long)k * g.ny + j) * g.pitch + i;
  dst[c] = src[c];
}

// Gt^i = gt^jk gt^il Gt_ljk, Gt_ljk = 1/2 (d_j gt_lk + d_k gt_lj - d_l gt_jk).
__global__ void nlo_gamma_kernel(const DevGrid g, const Coef c, double* __restrict__ U) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const Nbr n = make_nbr(g, i, j, k);
  const long fs = g.fstride;
  const int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  double gt[3][3], dg[3][3][3];  // dg[d][a][b] = d_d gt_ab
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      const double* F = U + (long)(1 + sym[a][b]) * fs;
      gt[a][b] = gt[b][a] = ldg(F, n.c);
      const double v[3] = {fd1<0>(F, n, c), fd1<1>(F, n, c), fd1<2>(F, n, c)};
      for (int d = 0; d < 3; ++d) dg[d][a][b] = dg[d][b][a] = v[d];
    }
  double cf[3][3];
  cf[0][0] = gt[1][1] * gt[2][2] - gt[1][2] * gt[2][1];
  cf[0][1] = gt[1][2] * gt[2][0] - gt[1][0] * gt[2][2];
  cf[0][2] = gt[1][0] * gt[2][1] - gt[1][1] * gt[2][0];
  cf[1][1] = gt[0][0] * gt[2][2] - gt[0][2] * gt[2][0];
  cf[1][2] = gt[0][1] * gt[2][0] - gt[0][0] * gt[2][1];
  cf[2][2] = gt[0][0] * gt[1][1] - gt[0][1] * gt[1][0];
  const double det = gt[0][0] * cf[0][0] + gt[0][1] * cf[0][1] + gt[0][2] * cf[0][2];
  double gu[3][3];
  gu[0][0] = cf[0][0] / det;
  gu[0][1] = gu[1][0] = cf[0][1] / det;
  gu[0][2] = gu[2][0] = cf[0][2] / det;
  gu[1][1] = cf[1][1] / det;
  gu[1][2] = gu[2][1] = cf[1][2] / det;
  gu[2][2] = cf[2][2] / det;
  for (int a = 0; a < 3; ++a) {
    double s = 0.0;
    for (int l = 0; l < 3; ++l)
      for (int b = 0; b < 3; ++b)
        for (int e = 0; e < 3; ++e)
          s += gu[b][e] * gu[a][l] * 0.5 * (dg[b][l][e] + dg[e][l][b] - dg[l][b][e]);
    U[(14 + a) * fs + n.c] = s;
  }
}

// tau~ = E chi^{-3/2}, S~_a = J_a chi^{-3/2} with 16 pi E = H and 8 pi J_a =
// gt_ab M^b of the metric without matter (hm = the vacuum constraints).
__global__ void nlo_fluid_kernel(const DevGrid g, const double* __restrict__ hm, double* __restrict__ U) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long c = ((long)k * g.ny + j) * g.pitch + i;
  const long fs = g.fstride;
  const int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  const double chi = U[c];
  const double chi32 = chi * sqrt(chi);
  U[24 * fs + c] = hm[c] / (16.0 * PI) / chi32;
  for (int a = 0; a < 3; ++a) {
    double Ja = 0.0;
    for (int b = 0; b < 3; ++b) Ja += U[(1 + sym[a][b]) * fs + c] * hm[(1 + b) * fs + c];
    U[(25 + a) * fs + c] = Ja / (8.0 * PI) / chi32;
  }
}

}  // namespace

int init_nlo(const cosmos_grid* g, const cosmos_params* p, double* state, double* hm, double* partial,
             cudaStream_t s) {
  const DevGrid dg = make_devgrid(g);
  const Coef c = make_coef(g, 0.0);
  const dim3 grid = point_grid(dg), block(BX, BY);
  nlo_metric_kernel<<<grid, block, 0, s>>>(dg, c, p->H0, p->w, state, hm);
  copy_field_kernel<<<grid, block, 0, s>>>(dg, hm, state);
  nlo_gamma_kernel<<<grid, block, 0, s>>>(dg, c, state);
  if (cudaGetLastError() != cudaSuccess) return COSMOS_ECUDA;
  ConstraintArgs ca;
  memset(&ca, 0, sizeof(ca));
  ca.g = dg;
  ca.c = c;
  cosmos_params pv = *p;
  pv.fluid = 0;
  pv.scalar = 0;
  ca.ap = algebra_params(&pv, 0.0);
  ca.U = state;
  ca.hm = hm;
  ca.partial = partial;
  if (launch_constraints_vac(ca, s) != cudaSuccess) return COSMOS_ECUDA;
  nlo_fluid_kernel<<<grid, block, 0, s>>>(dg, hm, state);
  return cudaGetLastError() == cudaSuccess ? COSMOS_OK : COSMOS_ECUDA;
}

}  // namespace cosmos

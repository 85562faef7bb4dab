// Reverse-mode kernels for the vacuum variant, and the initial-data reverse
// (zeta -> chi, and the fluid energy fixed by the discrete Hamiltonian
// constraint, which depends on chi through its derivatives).
#include "adjoint_kernel.cuh"

namespace cosmos {
COSMOS_DEFINE_ADJOINT(vac, false)

// Pass 1 of the initial-data reverse: per point, the cotangent of
// H_vac(chi, d chi, dd chi) is Ebar/(16 pi) with Ebar = lam_tau chi^{-3/2}.
__global__ void __launch_bounds__(BX* BY) init_ham_vjp_kernel(const DevGrid g, const Coef c, const AlgebraParams ap,
                                                              const double* __restrict__ U,
                                                              const double* __restrict__ lam, double* __restrict__ CB10) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const Nbr n = make_nbr(g, i, j, k);
  const long fs = g.fstride;
  double in[alg_vac::NIN + 1];
  gather<T_vac_adj>(U, nullptr, n, c, fs, in);
  const double chi = in[0];
  const double Ebar = ldg(lam + 24 * fs, n.c) / (chi * sqrt(chi));
  in[alg_vac::NIN] = Ebar / (16.0 * PI);
  double out[10];
  alg_vac::ham_vjp_chi(in, out, ap);
#pragma unroll
  for (int m = 0; m < 10; ++m) CB10[(long)m * fs + n.c] = out[m];
}

// Pass 2: chi_bar = direct terms + transposed stencils of the chi-input
// cotangents; zeta_bar = chi_bar d chi / d zeta = -2 chi chi_bar.
__global__ void __launch_bounds__(BX* BY) init_zeta_vjp_kernel(const DevGrid g, const Coef c,
                                                               const double* __restrict__ U,
                                                               const double* __restrict__ lam,
                                                               const double* __restrict__ CB10, int fluid,
                                                               double* __restrict__ zbar) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const Nbr n = make_nbr(g, i, j, k);
  const long fs = g.fstride;
  const double chi = ldg(U, n.c);
  double cb = ldg(lam, n.c);
  if (fluid) {
    const double tau = ldg(U + 24 * fs, n.c);  // tau = E chi^{-3/2}:  d tau / d chi |_E = -3/2 tau / chi
    cb += ldg(lam + 24 * fs, n.c) * (-1.5 * tau / chi);
    cb += ldg(CB10, n.c);
    cb -= fd1<0>(CB10 + fs, n, c) + fd1<1>(CB10 + 2 * fs, n, c) + fd1<2>(CB10 + 3 * fs, n, c);
    const double* G = CB10 + 4 * fs;
    cb += fd2<0>(G, n, c, ldg(G, n.c)) + fdmix<0, 1>(G + fs, n, c.mix[0]) + fdmix<0, 2>(G + 2 * fs, n, c.mix[1]) +
          fd2<1>(G + 3 * fs, n, c, ldg(G + 3 * fs, n.c)) + fdmix<1, 2>(G + 4 * fs, n, c.mix[2]) +
          fd2<2>(G + 5 * fs, n, c, ldg(G + 5 * fs, n.c));
  }
  zbar[((long)k * g.ny + j) * g.pitch + i] = -2.0 * chi * cb;
}

cudaError_t launch_init_zeta_vjp(const DevGrid& g, const Coef& c, const AlgebraParams& ap, const double* U,
                                 const double* lam, double* CB10, int fluid, double* zbar, cudaStream_t s) {
  if (fluid) {
    init_ham_vjp_kernel<<<point_grid(g), dim3(BX, BY), 0, s>>>(g, c, ap, U, lam, CB10);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  init_zeta_vjp_kernel<<<point_grid(g), dim3(BX, BY), 0, s>>>(g, c, U, lam, CB10, fluid, zbar);
  return cudaGetLastError();
}
}  // namespace cosmos

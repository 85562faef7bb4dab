// Fluid passes of the right-hand side (Kurganov-Tadmor, section "Physical
// system settings"): cell-centred primitive recovery, then the numerical flux
// through the +x, +y, +z face of every cell.  The stage kernel adds
// -(H_d(c) - H_d(c - e_d)) / h_d, so each face flux is computed once.
#include "stage_kernel.cuh"

namespace cosmos {

__device__ __forceinline__ void prim_point(const DevGrid& g, const double* __restrict__ U, double* __restrict__ prim,
                                           const FluidParams& fp, int i, int j, int k) {
  const long c = ((long)k * g.ny + j) * g.pitch + i;
  const long fs = g.fstride;
  double in[11];
  in[0] = ldg(U, c);
#pragma unroll
  for (int m = 0; m < 6; ++m) in[1 + m] = ldg(U + (1 + m) * fs, c);
#pragma unroll
  for (int m = 0; m < 4; ++m) in[7 + m] = ldg(U + (24 + m) * fs, c);
  double out[4];
  fluid_prim(in, out, fp);
#pragma unroll
  for (int m = 0; m < 4; ++m) prim[m * fs + c] = out[m];
}

__global__ void __launch_bounds__(BX* BY) prim_kernel(const DevGrid g, const double* __restrict__ U,
                                                      double* __restrict__ prim, const FluidParams fp) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  prim_point(g, U, prim, fp, i, j, k);
}

template <int D>
__device__ __forceinline__ void face(const double* __restrict__ U, const double* __restrict__ prim, const Nbr& n,
                                     long fs, const FluidParams& fp, double* __restrict__ H) {
  double in[34];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const long off = disp<D>(n, o - 1);
#pragma unroll
    for (int m = 0; m < 4; ++m) in[4 * o + m] = ldg(prim + m * fs, off);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const long off = disp<D>(n, s);
    double* q = in + 16 + 9 * s;
    q[0] = ldg(U, off);                   // chi
    q[1] = ldg(U + 17 * fs, off);         // alpha
    q[2] = ldg(U + (18 + D) * fs, off);   // beta^D
#pragma unroll
    for (int m = 0; m < 6; ++m) q[3 + m] = ldg(U + (1 + m) * fs, off);
  }
  double out[4];
  if (D == 0) fluid_face_flux_0(in, out, fp);
  if (D == 1) fluid_face_flux_1(in, out, fp);
  if (D == 2) fluid_face_flux_2(in, out, fp);
#pragma unroll
  for (int m = 0; m < 4; ++m) H[(4 * D + m) * fs + n.c] = out[m];
}

__device__ __forceinline__ void flux_point(const DevGrid& g, const double* __restrict__ U,
                                           const double* __restrict__ prim, double* __restrict__ H,
                                           const FluidParams& fp, int i, int j, int k) {
  const Nbr n = make_nbr(g, i, j, k);
  face<0>(U, prim, n, g.fstride, fp, H);
  face<1>(U, prim, n, g.fstride, fp, H);
  face<2>(U, prim, n, g.fstride, fp, H);
}

__global__ void __launch_bounds__(BX* BY) flux_kernel(const DevGrid g, const double* __restrict__ U,
                                                      const double* __restrict__ prim, double* __restrict__ H,
                                                      const FluidParams fp) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  flux_point(g, U, prim, H, fp, i, j, k);
}

// Batched passes: blocks stride over the flat work list of every instance
// (stage input args[inst].U, outputs into that instance's prim / flux buffers).
__global__ void __launch_bounds__(BX* BY) batch_prim_kernel(const StageArgs* __restrict__ args,
                                                            const BatchTile* __restrict__ tiles, long ntiles,
                                                            int mapping, const FluidParams fp) {
  for (long w = blockIdx.x; w < ntiles; w += gridDim.x) {
    const BatchTile t = tiles[w];
    const StageArgs& a = args[t.inst];
    int i, j, k;
    if (batch_point(t, a.g, mapping, i, j, k)) prim_point(a.g, a.U, const_cast<double*>(a.prim), fp, i, j, k);
  }
}

__global__ void __launch_bounds__(BX* BY) batch_flux_kernel(const StageArgs* __restrict__ args,
                                                            const BatchTile* __restrict__ tiles, long ntiles,
                                                            int mapping, const FluidParams fp) {
  for (long w = blockIdx.x; w < ntiles; w += gridDim.x) {
    const BatchTile t = tiles[w];
    const StageArgs& a = args[t.inst];
    int i, j, k;
    if (batch_point(t, a.g, mapping, i, j, k)) flux_point(a.g, a.U, a.prim, const_cast<double*>(a.flux), fp, i, j, k);
  }
}

static FluidParams fluid_params(double w) {
  FluidParams fp;
  fp.w = w;
  fp.sqrt_w = sqrt(w);
  return fp;
}

cudaError_t launch_fluid_prim(const DevGrid& g, const double* U, double* prim, double w, cudaStream_t s) {
  prim_kernel<<<point_grid(g), dim3(BX, BY), 0, s>>>(g, U, prim, fluid_params(w));
  return cudaGetLastError();
}

cudaError_t launch_batch_fluid(const StageArgs* args, const BatchTile* tiles, long ntiles, int mapping, double w,
                               dim3 grid, dim3 block, cudaStream_t s) {
  batch_prim_kernel<<<grid, block, 0, s>>>(args, tiles, ntiles, mapping, fluid_params(w));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_flux_kernel<<<grid, block, 0, s>>>(args, tiles, ntiles, mapping, fluid_params(w));
  return cudaGetLastError();
}

cudaError_t launch_fluid_flux(const DevGrid& g, const double* U, const double* prim, double* flux, double w,
                              int /*nf_offset_fluid*/, cudaStream_t s) {
  flux_kernel<<<point_grid(g), dim3(BX, BY), 0, s>>>(g, U, prim, flux, fluid_params(w));
  return cudaGetLastError();
}

}  // namespace cosmos

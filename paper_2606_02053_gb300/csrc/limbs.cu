// Pre-pass of the integer derivative pass (stage_int.cuh): the reference
// exponent of every limb slot, then the limb copy of the stage state.
#include "stage_kernel.cuh"

namespace cosmos {

// E[s] = max over the grid of the biased exponent of slot s (E zeroed before).
// Blocks stride over the rows (j, k); padding columns are never read.
__global__ void field_exponent_kernel(const DevGrid g, const double* __restrict__ U, int s_lo, int fluid,
                                      int* __restrict__ E) {
  const int s = s_lo + blockIdx.y;
  const double* F = U + (long)limb_field(s, fluid) * g.fstride;
  const long rows = (long)g.ny * g.nz;
  unsigned m = 0;
  // four rows per iteration, so that four loads are in flight per thread
  for (long r0 = 4 * (long)blockIdx.x; r0 < rows; r0 += 4 * (long)gridDim.x)
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      unsigned long long b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = r0 + q < rows ? (unsigned long long)__double_as_longlong(__ldg(F + (r0 + q) * g.pitch + i)) : 0ull;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned e = (unsigned)((b[q] >> 52) & 0x7FF);
        m = e > m ? e : m;
      }
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned v = __shfl_down_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax((unsigned*)E + s, m);
}

__global__ void to_limbs_kernel(const DevGrid g, const double* __restrict__ U, int s_lo, int fluid,
                                const int* __restrict__ E, long long* __restrict__ L) {
  const int s = s_lo + blockIdx.y;
  const double* F = U + (long)limb_field(s, fluid) * g.fstride;
  long long* Ls = L + (long)s * g.fstride;
  const int e_ref = max(E[s], 1);
  const long rows = (long)g.ny * g.nz;
  for (long r = blockIdx.x; r < rows; r += gridDim.x) {
    const long o = r * g.pitch;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) Ls[o + i] = to_limbs(__ldg(F + o + i), e_ref);
  }
}

// Batched pre-pass: blockIdx.z = instance, blockIdx.y = slot; the arguments
// of instance i are args[i] (its stage input U, grid, limb copy and exponents).
__global__ void batch_field_exponent_kernel(const StageArgs* __restrict__ args, int fluid) {
  const StageArgs& a = args[blockIdx.z];
  const DevGrid g = a.g;
  const int s = blockIdx.y;
  const double* F = a.U + (long)limb_field(s, fluid) * g.fstride;
  unsigned m = 0;
  const long rows = (long)g.ny * g.nz;
  for (long r = blockIdx.x; r < rows; r += gridDim.x) {
    const double* R = F + r * g.pitch;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const unsigned e = (unsigned)(((unsigned long long)__double_as_longlong(__ldg(R + i)) >> 52) & 0x7FF);
      m = e > m ? e : m;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned v = __shfl_down_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax((unsigned*)a.E + s, m);
}

__global__ void batch_to_limbs_kernel(const StageArgs* __restrict__ args, int fluid) {
  const StageArgs& a = args[blockIdx.z];
  const DevGrid g = a.g;
  const int s = blockIdx.y;
  const double* F = a.U + (long)limb_field(s, fluid) * g.fstride;
  long long* Ls = const_cast<long long*>(a.L) + (long)s * g.fstride;
  const int e_ref = max(a.E[s], 1);
  const long rows = (long)g.ny * g.nz;
  for (long r = blockIdx.x; r < rows; r += gridDim.x) {
    const long o = r * g.pitch;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) Ls[o + i] = to_limbs(__ldg(F + o + i), e_ref);
  }
}

cudaError_t launch_batch_limbs(const StageArgs* args, int n, int nslot, int fluid, int* E_all, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(E_all, 0, sizeof(int) * (size_t)n * nslot, s);
  if (e != cudaSuccess) return e;
  const dim3 grid(32, (unsigned)nslot, (unsigned)n);
  batch_field_exponent_kernel<<<grid, 128, 0, s>>>(args, fluid);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  batch_to_limbs_kernel<<<grid, 128, 0, s>>>(args, fluid);
  return cudaGetLastError();
}

cudaError_t launch_limbs(const DevGrid& g, const double* U, int fluid, int s_lo, int s_hi, int* E, long long* L,
                         cudaStream_t s) {
  if (s_hi <= s_lo) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(E + s_lo, 0, sizeof(int) * (s_hi - s_lo), s);
  if (e != cudaSuccess) return e;
  const long rows = (long)g.ny * g.nz;
  const int threads = g.nx >= 256 ? 256 : (g.nx >= 128 ? 128 : 64);
  const dim3 grid((unsigned)(rows < 2048 ? rows : 2048), (unsigned)(s_hi - s_lo));
  field_exponent_kernel<<<grid, threads, 0, s>>>(g, U, s_lo, fluid, E);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  to_limbs_kernel<<<grid, threads, 0, s>>>(g, U, s_lo, fluid, E, L);
  return cudaGetLastError();
}

// The limb copy of slots s_lo .. s_hi - 1 with the reference exponents given
// in E (no scan).
cudaError_t launch_to_limbs(const DevGrid& g, const double* U, int fluid, int s_lo, int s_hi, const int* E,
                            long long* L, cudaStream_t s) {
  if (s_hi <= s_lo) return cudaSuccess;
  const long rows = (long)g.ny * g.nz;
  const int threads = g.nx >= 256 ? 256 : (g.nx >= 128 ? 128 : 64);
  const dim3 grid((unsigned)(rows < 2048 ? rows : 2048), (unsigned)(s_hi - s_lo));
  to_limbs_kernel<<<grid, threads, 0, s>>>(g, U, s_lo, fluid, E, L);
  return cudaGetLastError();
}

// Only the exponent scan of slots s_lo .. s_hi - 1 into E.
cudaError_t launch_field_exponents(const DevGrid& g, const double* U, int fluid, int s_lo, int s_hi, int* E,
                                   cudaStream_t s) {
  if (s_hi <= s_lo) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(E + s_lo, 0, sizeof(int) * (s_hi - s_lo), s);
  if (e != cudaSuccess) return e;
  const long rows = (long)g.ny * g.nz;
  const int threads = g.nx >= 256 ? 256 : (g.nx >= 128 ? 128 : 64);
  const dim3 grid((unsigned)(rows < 2048 ? rows : 2048), (unsigned)(s_hi - s_lo));
  field_exponent_kernel<<<grid, threads, 0, s>>>(g, U, s_lo, fluid, E);
  return cudaGetLastError();
}

__global__ void exponents_from_record_kernel(unsigned* __restrict__ rec, int* __restrict__ E, int nslot) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslot; s += gridDim.x * blockDim.x) {
    E[s] = (int)rec[32 * s];
    rec[32 * s] = 0u;
  }
}

cudaError_t launch_exponents_from_record(unsigned* rec, int* E, int nslot, cudaStream_t s) {
  exponents_from_record_kernel<<<(nslot + 255) / 256, 256, 0, s>>>(rec, E, nslot);
  return cudaGetLastError();
}

// The batched limb copy with the exponents already in args[i].E (no scan).
cudaError_t launch_batch_to_limbs(const StageArgs* args, int n, int nslot, int fluid, cudaStream_t s) {
  const dim3 grid(32, (unsigned)nslot, (unsigned)n);
  batch_to_limbs_kernel<<<grid, 128, 0, s>>>(args, fluid);
  return cudaGetLastError();
}

}  // namespace cosmos

// cosmos_constraints_noalloc: the constraint norms without any caller-provided
// workspace.  Its scratch (per-block partial norms, the final eight sums and,
// with the fluid on, the cell primitives) lives in one file-scope device array
// that the library image carries; every GPU that loads the library holds it
// until the process exits.
#include <mutex>
#include <string.h>

#include "common.cuh"

namespace cosmos {

// 2^21 doubles = 16 MiB.
constexpr size_t NOALLOC_SCRATCH_DOUBLES = size_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static double* g_scratch_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mutex;

// Device address of the static array for the current device.  The host-side
// name g_noalloc_scratch is only a stand-in; kernels must be given this
// address.  Resolved once per device, on the first call made with that
// device current.
static cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Fixed-order reduction of the per-block partials (sum of squares, max |.|).
__global__ void noalloc_reduce(const double* __restrict__ part, long nb, double* __restrict__ out) {
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

static size_t round256(size_t doubles) { return (doubles + 31) & ~(size_t)31; }

}  // namespace cosmos

using namespace cosmos;

extern "C" int cosmos_constraints_noalloc(const cosmos_grid* g, const cosmos_params* p, const double* state,
                                          double* ham_mom, double norms_host[8], void* stream) {
  // the same argument checks as cosmos_constraints, then the scratch size
  const int v = validate(g, p);
  if (v != COSMOS_OK) return v;
  if (!state || !norms_host) return COSMOS_EINVAL;
  if (((uintptr_t)state & 15u) || ((uintptr_t)ham_mom & 15u)) return COSMOS_EALIGN;

  const DevGrid dg = make_devgrid(g);
  const dim3 blocks = point_grid(dg);
  const long nb = (long)blocks.x * blocks.y * blocks.z;
  const size_t prim_doubles = p->fluid ? round256(4 * (size_t)dg.fstride) : 0;
  const size_t part_doubles = round256(8 * (size_t)nb);
  if (prim_doubles + part_doubles + 8 > NOALLOC_SCRATCH_DOUBLES) return COSMOS_EWORKSPACE;

  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return COSMOS_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  double* prim = p->fluid ? scratch : nullptr;
  double* partial = scratch + prim_doubles;
  double* fin = partial + part_doubles;

  ConstraintArgs c;
  memset(&c, 0, sizeof(c));
  c.g = dg;
  c.c = make_coef(g, 0.0);
  c.ap.w = p->w;
  c.U = state;
  c.prim = prim;
  c.hm = ham_mom;
  c.partial = partial;
  if (p->fluid && launch_fluid_prim(dg, state, prim, p->w, s) != cudaSuccess) return COSMOS_ECUDA;
  cudaError_t e;
  if (p->fluid && p->scalar)
    e = launch_constraints_fluid_scalar(c, s);
  else if (p->fluid)
    e = launch_constraints_fluid(c, s);
  else if (p->scalar)
    e = launch_constraints_scalar(c, s);
  else
    e = launch_constraints_vac(c, s);
  if (e != cudaSuccess) return COSMOS_ECUDA;
  noalloc_reduce<<<1, 256, 0, s>>>(partial, nb, fin);
  if (cudaGetLastError() != cudaSuccess) return COSMOS_ECUDA;
  double r[8];
  if (cudaMemcpyAsync(r, fin, sizeof(r), cudaMemcpyDeviceToHost, s) != cudaSuccess) return COSMOS_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return COSMOS_ECUDA;
  const double npts = (double)g->nx * g->ny * g->nz;
  for (int m = 0; m < 4; ++m) {
    norms_host[m] = sqrt(r[m] / npts);
    norms_host[4 + m] = r[4 + m];
  }
  return COSMOS_OK;
}

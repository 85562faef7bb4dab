// Stage / RHS / constraint kernels for the "fluid_scalar" matter variant.
#include "stage_kernel.cuh"

namespace cosmos {
COSMOS_DEFINE_VARIANT(fluid_scalar, true, true)
}  // namespace cosmos

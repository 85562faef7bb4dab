// Stage / RHS / constraint kernels for the "fluid" matter variant.
#include "stage_kernel.cuh"

namespace cosmos {
COSMOS_DEFINE_VARIANT(fluid, true, false)
}  // namespace cosmos

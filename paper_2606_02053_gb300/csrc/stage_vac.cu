// Stage / RHS / constraint kernels for the "vac" matter variant.
#include "stage_kernel.cuh"

namespace cosmos {
COSMOS_DEFINE_VARIANT(vac, false, false)
}  // namespace cosmos

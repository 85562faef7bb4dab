// Stage / RHS / constraint kernels for the "scalar" matter variant.
#include "stage_kernel.cuh"

namespace cosmos {
COSMOS_DEFINE_VARIANT(scalar, false, true)
}  // namespace cosmos

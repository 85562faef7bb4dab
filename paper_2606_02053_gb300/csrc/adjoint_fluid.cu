// Reverse-mode kernels for the fluid variant.
#include "adjoint_kernel.cuh"

namespace cosmos {
COSMOS_DEFINE_ADJOINT(fluid, true)
}  // namespace cosmos

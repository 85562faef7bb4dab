// Reverse-mode kernels for the fluid + scalar variant.
#include "adjoint_kernel.cuh"

namespace cosmos {
COSMOS_DEFINE_ADJOINT(fluid_scalar, true)
}  // namespace cosmos

// Reverse-mode kernels for the scalar variant.
#include "adjoint_kernel.cuh"

namespace cosmos {
COSMOS_DEFINE_ADJOINT(scalar, false)
}  // namespace cosmos

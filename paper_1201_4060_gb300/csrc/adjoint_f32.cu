// Instantiations of the adjoint particle kernels (f32 coefficients, orders 2-8).
#include "adjoint.cuh"

namespace bs {
BS_ADJOINT_INSTANTIATE(2, float, float)
BS_ADJOINT_INSTANTIATE(3, float, float)
BS_ADJOINT_INSTANTIATE(4, float, float)
BS_ADJOINT_INSTANTIATE(5, float, float)
BS_ADJOINT_INSTANTIATE(6, float, float)
BS_ADJOINT_INSTANTIATE(7, float, float)
BS_ADJOINT_INSTANTIATE(8, float, float)
}  // namespace bs

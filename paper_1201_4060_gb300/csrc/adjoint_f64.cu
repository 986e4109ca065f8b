// Instantiations of the adjoint particle kernels (f64 coefficients, orders 2-8).
#include "adjoint.cuh"

namespace bs {
BS_ADJOINT_INSTANTIATE(2, double, double)
BS_ADJOINT_INSTANTIATE(3, double, double)
BS_ADJOINT_INSTANTIATE(4, double, double)
BS_ADJOINT_INSTANTIATE(5, double, double)
BS_ADJOINT_INSTANTIATE(6, double, double)
BS_ADJOINT_INSTANTIATE(7, double, double)
BS_ADJOINT_INSTANTIATE(8, double, double)
}  // namespace bs

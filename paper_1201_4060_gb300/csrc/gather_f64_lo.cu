// Instantiations of the gather kernel (f64 coefficients, orders 2, 3, 4, 5).
#include "particles.cuh"

namespace bs {
BS_GATHER_INSTANTIATE(2, double, double, double)
BS_GATHER_INSTANTIATE(3, double, double, double)
BS_GATHER_INSTANTIATE(4, double, double, double)
BS_GATHER_INSTANTIATE(5, double, double, double)
}  // namespace bs

// Instantiations of the gather kernel (f64 coefficients, orders 6, 7, 8).
#include "particles.cuh"

namespace bs {
BS_GATHER_INSTANTIATE(6, double, double, double)
BS_GATHER_INSTANTIATE(7, double, double, double)
BS_GATHER_INSTANTIATE(8, double, double, double)
}  // namespace bs

// Instantiations of the gather kernel (f32 coefficients, orders 6, 7, 8).
#include "particles.cuh"

namespace bs {
BS_GATHER_INSTANTIATE(6, float, float, float)
BS_GATHER_INSTANTIATE(7, float, float, float)
BS_GATHER_INSTANTIATE(8, float, float, float)
}  // namespace bs

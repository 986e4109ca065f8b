// Instantiations of the gather kernel (f32 coefficients, orders 2, 3, 4, 5).
#include "particles.cuh"

namespace bs {
BS_GATHER_INSTANTIATE(2, float, float, float)
BS_GATHER_INSTANTIATE(3, float, float, float)
BS_GATHER_INSTANTIATE(4, float, float, float)
BS_GATHER_INSTANTIATE(5, float, float, float)
}  // namespace bs

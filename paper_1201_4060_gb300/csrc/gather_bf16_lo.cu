// Instantiations of the gather kernel (bf16 coefficients, orders 2, 3, 4, 5).
#include "particles.cuh"

namespace bs {
BS_GATHER_INSTANTIATE(2, __nv_bfloat16, float, float)
BS_GATHER_INSTANTIATE(3, __nv_bfloat16, float, float)
BS_GATHER_INSTANTIATE(4, __nv_bfloat16, float, float)
BS_GATHER_INSTANTIATE(5, __nv_bfloat16, float, float)
}  // namespace bs

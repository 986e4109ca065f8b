// Instantiations of the gather kernel (bf16 coefficients, orders 6, 7, 8).
#include "particles.cuh"

namespace bs {
BS_GATHER_INSTANTIATE(6, __nv_bfloat16, float, float)
BS_GATHER_INSTANTIATE(7, __nv_bfloat16, float, float)
BS_GATHER_INSTANTIATE(8, __nv_bfloat16, float, float)
}  // namespace bs

// Instantiations of the adjoint particle kernels (bf16 coefficients, orders 2-8).
#include "adjoint.cuh"

namespace bs {
BS_ADJOINT_INSTANTIATE(2, __nv_bfloat16, float)
BS_ADJOINT_INSTANTIATE(3, __nv_bfloat16, float)
BS_ADJOINT_INSTANTIATE(4, __nv_bfloat16, float)
BS_ADJOINT_INSTANTIATE(5, __nv_bfloat16, float)
BS_ADJOINT_INSTANTIATE(6, __nv_bfloat16, float)
BS_ADJOINT_INSTANTIATE(7, __nv_bfloat16, float)
BS_ADJOINT_INSTANTIATE(8, __nv_bfloat16, float)
}  // namespace bs

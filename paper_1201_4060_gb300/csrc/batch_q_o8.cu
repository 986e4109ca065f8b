// Persistent batch kernel (u and grad u, FP32 coefficients) of order 8, every brick y extent.
#include "batch_queue.cuh"

namespace bs {
namespace batch_impl {
int launch_batch_queue_o8(int by, const Queue& q, int sms, cudaStream_t stream) {
    return dispatch_brick_y<8>(by, q, sms, stream);
}
}  // namespace batch_impl
}  // namespace bs

// bspline_interp_noalloc: particle evaluation without any device allocation.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph
// capture owned by another framework (allocation is not a capturable
// operation), code that must never stall the device (cudaMalloc and
// cudaFree can synchronise), and processes whose device memory is owned by
// a different allocator with a fixed budget.  For them this entry point
// takes the grid parameters directly instead of a plan and keeps all of its
// scratch (particle bins, sort buffers and the status word) in one fixed
// array compiled into the library, sized for at most BSPLINE_NOALLOC_MAX_N^3
// grids and BSPLINE_NOALLOC_MAX_PARTICLES particles.
//
// Host code cannot use the array's name as a device address, so its device
// address is looked up once per device with cudaGetSymbolAddress (while that
// device is current) and cached.  That look-up happens on the first call on a
// device, which is why the first call should come before any stream capture.
// Every call uses the same array: the per-brick counters and the status word
// are cleared at the start of each call, and calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;      // 16 MiB on every GPU that loads the library
constexpr size_t kStatusBytes = 256;                      // status words, kept apart from the workspace
static_assert(sizeof(unsigned long long) * bs::kStatusWords <= kStatusBytes, "status words fit");
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
int scratch_for_device(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return BSPLINE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return bs::set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return BSPLINE_OK;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

}  // namespace

extern "C" int bspline_interp_noalloc(const void* coeffs, int N, int order, bspline_dtype dtype, double L,
                                      const double* x, int64_t P, void* out_u, void* out_grad, int flags,
                                      void* stream) {
    if (dtype != BSPLINE_F64 && dtype != BSPLINE_F32 && dtype != BSPLINE_BF16) return BSPLINE_ERR_INVALID_ARG;
    if (!bs::supported_grid(N)) return BSPLINE_ERR_UNSUPPORTED_N;
    if (order < 2 || order > 8) return BSPLINE_ERR_UNSUPPORTED_ORDER;
    if (!(L > 0.0) || !(L < 1e300)) return BSPLINE_ERR_INVALID_ARG;
    if (flags & ~BSPLINE_INTERP_NO_GRAD) return BSPLINE_ERR_INVALID_ARG;
    if (P < 0) return BSPLINE_ERR_INVALID_ARG;
    if (N > BSPLINE_NOALLOC_MAX_N || P > BSPLINE_NOALLOC_MAX_PARTICLES) return BSPLINE_ERR_TOO_LARGE;
    if (P == 0) return BSPLINE_OK;
    if (!coeffs || !x || !out_u) return BSPLINE_ERR_INVALID_ARG;
    if (!(flags & BSPLINE_INTERP_NO_GRAD) && !out_grad) return BSPLINE_ERR_INVALID_ARG;
    const size_t ob = dtype == BSPLINE_F64 ? 8 : 4;
    if (!aligned(coeffs, 16) || !aligned(x, 8) || !aligned(out_u, ob) || (out_grad && !aligned(out_grad, ob)))
        return BSPLINE_ERR_INVALID_ARG;

    // A plan on the stack: only the fields the launch sequence reads; it owns nothing.
    bspline_plan_s p;
    p.N = N;
    p.order = order;
    p.dtype = dtype;
    p.L = L;
    p.stream = (cudaStream_t)stream;
    if (bs::interp_workspace_bytes(&p, P) + kStatusBytes > kScratchBytes) return BSPLINE_ERR_TOO_LARGE;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bs::set_cuda_error(e);
    p.device = dev;
    void* base = nullptr;
    int rc = scratch_for_device(dev, &base);
    if (rc == BSPLINE_OK) {
        auto* status = reinterpret_cast<unsigned long long*>(base);
        p.d_status = status;                       // words 0-2 are cleared by every call (non-finite, tile wait, bounds)
        void* ws = static_cast<unsigned char*>(base) + kStatusBytes;
        rc = bs::launch_interp_ws(&p, ws, status, coeffs, x, P, out_u, out_grad, flags);
    }
    return rc;
}

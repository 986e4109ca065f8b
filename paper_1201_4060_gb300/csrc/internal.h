// Internal declarations of the B-spline interpolation library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include <vector>

#include "../../include/bspline.h"

namespace bs {

// Bricks of the particle sort: particles are binned by the brick that holds
// the first node of their stencil, and one CTA stages one brick (plus the
// order-1 halo) of coefficients in shared memory.  FP64: 8^3 cells.
// FP32/BF16: 16 x BY x 16 cells with BY = 12 up to order 6 and 8 above, so
// that the FP32 tile, its z rows padded to a multiple of 16 bytes for 16-byte
// copies, still fits two CTAs per SM (order 6: 3 x 21 x 17 x 24 floats).
constexpr int brick_x(int dtype) { return dtype == BSPLINE_F64 ? 8 : 16; }
constexpr int brick_y(int dtype, int order) { return dtype == BSPLINE_F64 ? 8 : (order <= 6 ? 12 : 8); }
constexpr int brick_z(int dtype) { return brick_x(dtype); }

// Bricks per axis (partial bricks at the high end count) and their total.
struct BrickGrid {
    int nbx, nby, nbz;
    int by;            // brick edge along y (x and z: brick_x)
    int bshift;        // log2 of the x and z edge
    unsigned NB;
};
inline BrickGrid brick_grid(int N, int dtype, int order) {
    BrickGrid g;
    const int bx = brick_x(dtype), by = brick_y(dtype, order);
    g.nbx = (N + bx - 1) / bx;
    g.nby = (N + by - 1) / by;
    g.nbz = g.nbx;
    g.by = by;
    g.bshift = bx == 16 ? 4 : 3;
    g.NB = (unsigned)g.nbx * g.nby * g.nbz;
    return g;
}

// Grid sizes with compiled transforms: powers of two 8..1024, and 3 * 2^k
// from 48 to 768 (radix-3 stage; multiples of the 16-cell brick).
inline bool supported_grid(int N) {
    if (N < 8 || N > 1024) return false;
    if ((N & (N - 1)) == 0) return true;
    const int q = N / 3;
    return N % 3 == 0 && (q & (q - 1)) == 0 && N % 16 == 0;
}

// Device status words of a plan, read by bspline_status.  Particle calls
// (interp, eval, the adjoint's particle side) clear words 0-2 when they start,
// the transform clears word 3.
constexpr int kStatusNonfinite = 0;          // non-finite positions of the last particle call
constexpr int kStatusParticleTimeout = 1;    // a tile wait of the last particle call ran out
constexpr int kStatusBounds = 2;             // index checks that failed (BSPLINE_CHECKS builds)
constexpr int kStatusTransformTimeout = 3;   // a wait of the last transform ran out
constexpr int kStatusWords = 4;
constexpr int kStatusParticleWords = 3;      // the words a particle call clears

// Index checks of a BSPLINE_CHECKS=1 build (compiled with -DBSPLINE_CHECKS=1):
// BS_CHECK_OK(cond, word) is true when cond holds; when it does not, the
// failure is counted in *word (a device status word) and the caller skips the
// access the condition guards.  In other builds it is the constant true and
// cond is not evaluated.
#ifndef BSPLINE_CHECKS
#define BSPLINE_CHECKS 0
#endif
#ifdef __CUDACC__
__device__ __forceinline__ bool bs_check_count(bool ok, unsigned long long* word) {
    if (!ok) atomicAdd(word, 1ULL);
    return ok;
}
#endif
#define BS_CHECK_OK(cond, word) (!BSPLINE_CHECKS || bs_check_count((cond), (word)))

struct PendingTiming {
    int stage;
    cudaEvent_t start, stop;
};

struct DeviceBuffer {
    void* ptr = nullptr;
    size_t bytes = 0;
    int grow(size_t need);      // cudaMalloc on first use / growth (synchronises)
    void release();
};

}  // namespace bs

struct bspline_plan_s {
    int N = 0;
    int order = 0;
    int dtype = 0;
    int prefilter = BSPLINE_PREFILTER_INTERP;
    double L = 0.0;
    int device = 0;
    cudaStream_t stream = nullptr;

    // Prefilter c(k), k = 0..N-1 (index k <-> signed wavenumber k mod N), in
    // FP64 and rounded to FP32; twiddles exp(+2 pi i m / N), m = 0..N-1.
    double* d_c64 = nullptr;
    float* d_c32 = nullptr;
    double2* d_tw64 = nullptr;
    float2* d_tw32 = nullptr;

    // Transform workspace: complex [3][N][N][N/2+1].
    bs::DeviceBuffer work;
    // Particle workspace (binning, sort, sorted particle records).
    bs::DeviceBuffer pws;
    // Device status words (bs::kStatus*): non-finite count and wait time-outs.
    unsigned long long* d_status = nullptr;
    int sms = 1;            // streaming multiprocessors of the plan's device
    int test_hooks = 0;     // BSPLINE_TEST_* flags
    unsigned direct_below = BSPLINE_GATHER_SPLIT_AUTO;   // gather split (bspline_plan_set_gather_split)
    int deterministic = 0;  // bspline_plan_set_deterministic: fixed-point spread of the adjoint
    int band = 0;           // bspline_plan_set_band: modes beyond |k_i| <= band taken as zero (0: none)
    bs::DeviceBuffer det;   // its accumulator [3][N][N][N] int64 and the cotangent bound
    bs::DeviceBuffer cot;   // adjoint, FP32 types: the cotangents in sorted order, [P][16] floats
    // Buffers, second stream and events of bspline_run_host (and the second
    // stream of bspline_eval); the copy stream and its events feed the
    // host-to-device copies of bspline_run_host.
    bs::DeviceBuffer host_uhat, host_coef, host_x, host_u, host_grad;
    cudaStream_t aux_stream = nullptr, copy_stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_sorted = nullptr;
    cudaEvent_t ev_copied[4] = {};      // positions, then the three u_hat components, arrived
    // Per-kernel timing (bspline_plan_set_timing): event pairs recorded on the
    // plan's stream around each launch, resolved by bspline_stage_times.
    bool timing = false;
    std::vector<bs::PendingTiming> pending;
    std::vector<cudaEvent_t> free_events;
};

namespace bs {

int set_cuda_error(cudaError_t e);

// Bracket a kernel launch with timing events when the plan's timing is on.
struct StageTimer {
    bspline_plan_s* p;
    int stage;
    cudaEvent_t start = nullptr;
    StageTimer(bspline_plan_s* plan, int s);
    ~StageTimer();
};

// Transform: u_hat -> coefficients (prefilter fused into the first pass).
int launch_coeffs(bspline_plan_s* p, const void* u_hat, void* coeffs);

// Transform of components c0..c1-1 only (launch_coeffs = 0..3).
int launch_coeffs_range(bspline_plan_s* p, const void* u_hat, void* coeffs, int c0, int c1);

// Transform of F fields with p's grid size, order, dtype and prefilter, one launch per kernel:
// in_fields / out_fields are device arrays of F u_hat / coefficient pointers, work holds
// coeffs_fields_workspace_bytes(p, F) bytes; a wait that runs out sets *error.
size_t coeffs_fields_workspace_bytes(const bspline_plan_s* p, int F);
int launch_coeffs_fields(const bspline_plan_s* p, int F, const void* const* in_fields, void* const* out_fields,
                         void* work, unsigned* error, cudaStream_t st);

// Particles: bin, sort and evaluate u and grad u.
size_t interp_workspace_bytes(const bspline_plan_s* p, int64_t P);
int launch_interp(bspline_plan_s* p, const void* coeffs, const double* x, int64_t P, void* out_u,
                  void* out_grad, int flags);
// The same, with the sort on sort_stream (recording `sorted` there) and the
// gather on the plan's stream once `sorted` has been reached.
int launch_interp_split(bspline_plan_s* p, const void* coeffs, const double* x, int64_t P, void* out_u,
                        void* out_grad, int flags, cudaStream_t sort_stream, cudaEvent_t sorted);
// The same sequence on a caller-supplied workspace (interp_workspace_bytes bytes) and status word.
int launch_interp_ws(bspline_plan_s* p, void* ws, unsigned long long* status, const void* coeffs,
                     const double* x, int64_t P, void* out_u, void* out_grad, int flags);

// Brick order of P positions: perm[i] = original index of the i-th particle in
// the order the gather evaluates them (bricks in key order, invalid positions last).
int launch_sort_order(bspline_plan_s* p, const double* x, int64_t P, int* perm);

// Adjoint: bin/sort, then spread cotangents into g_coef (accumulate; skipped
// if NULL) and write position gradients g_x (skipped if NULL).
int launch_adjoint_particles(bspline_plan_s* p, const void* coeffs, const double* x, int64_t P, const void* g_u,
                             const void* g_grad, void* g_coef, double* g_x);
// Adjoint of launch_coeffs: g_u_hat (half spectrum) from g_coef, through the
// transform workspace (grown by the caller).
int launch_adjoint_transform(bspline_plan_s* p, const void* g_coef, void* g_u_hat);
size_t coeffs_workspace_bytes(const bspline_plan_s* p);

}  // namespace bs

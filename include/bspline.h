/*
 * bspline.h -- C ABI of the GB300 (sm_103a) B-spline interpolation library
 * for pseudo-spectral fields.
 *
 * The method (van Hinsberg, ten Thije Boonkkamp, Toschi, Clercx, "On the
 * efficiency and accuracy of interpolation methods for spectral codes"):
 *   1. prefilter every Fourier mode by c(kx) c(ky) c(kz), c(k) = 1/F_D[B_D](k)
 *      (Section 7, Eqs. B_spline_multiplication, B_spline_multiplication_3d);
 *   2. one inverse real 3D FFT gives the B-spline coefficients u_B
 *      (Section 7, coefficient transform);
 *   3. evaluate the order-n tensor-product B-spline and its first derivatives
 *      at off-grid points (Sections 3-4, Eqs. interpolation, interpolation2,
 *      Table 1; stencil nodes by Eq. alg-int-6).
 *
 * Conventions shared by every entry point
 *   - Domain [0, L)^3, default L = 2 pi, N grid points per axis.
 *   - Field u(x) = sum_k u_hat_k exp(i (2 pi / L) k . x): u_hat holds
 *     Fourier-series coefficients (not N^3-scaled DFT output).
 *   - u_hat layout: half spectrum [3][N][N][N/2+1] of interleaved complex
 *     (re, im), index (component, kx, ky, kz), signed wavenumber k stored at
 *     index k mod N, kz >= 0 only, kz fastest.  Real-to-complex semantics:
 *     the imaginary part of self-conjugate modes (kz = 0 or N/2 planes) is
 *     ignored, as by any inverse real FFT.
 *   - Coefficient layout: real [3][N][N][N], z fastest, element type of the
 *     plan's dtype (double, float or bfloat16).
 *   - Positions x: double [P][3], any real values; wrapped periodically.
 *   - Outputs: out_u [P][3] and out_grad [P][3][3] with
 *     out_grad[p][i][j] = d u_i / d x_j in physical units; element type
 *     double for BSPLINE_F64 plans, float otherwise.
 *   - All pointers passed to the compute calls are device pointers unless the
 *     name says host.  The caller owns every buffer it passes; the plan owns
 *     its tables and workspace and frees them in bspline_destroy.
 *   - Calls are asynchronous on the plan's stream (default: the legacy
 *     default stream).  Device-side status (non-finite input count) is read
 *     with bspline_status after synchronising that stream.
 *   - Every function returns 0 (BSPLINE_OK) or a negative status code and
 *     never aborts or throws; a failed call leaves the outputs unspecified.
 *   - A plan holds mutable state (workspace, streams, timers): calls on one
 *     plan must not run concurrently from several host threads.  Distinct
 *     plans are independent and may be used from different threads.
 */
#ifndef BSPLINE_H
#define BSPLINE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bspline_plan_s* bspline_plan_t;

/* Coefficient storage type.  F64: FP64 everywhere.  F32: FP32 transform,
 * FP32 coefficients, FP32 weights and accumulation.  BF16: FP32 transform,
 * coefficients rounded to bfloat16 on store, FP32 weights and accumulation.
 * Position-to-cell index and local offset are computed in FP64 for all. */
typedef enum { BSPLINE_F64 = 0, BSPLINE_F32 = 1, BSPLINE_BF16 = 2 } bspline_dtype;

/* Prefilter choice (Section 7): INTERP is c(k) = 1/F_D[B_D](k), which makes
 * the interpolant reproduce the grid values; L2 is the L2-optimal
 * c(k) = F[B](kappa) / sum_i F[B](kappa + i)^2 of Eq. B_spline_coeff. */
typedef enum { BSPLINE_PREFILTER_INTERP = 0, BSPLINE_PREFILTER_L2 = 1 } bspline_prefilter;

enum {
    BSPLINE_OK = 0,
    BSPLINE_ERR_INVALID_ARG = -1,       /* null/misaligned pointer, P < 0, bad flag, bad plan */
    BSPLINE_ERR_UNSUPPORTED_N = -2,     /* N not a supported transform length */
    BSPLINE_ERR_UNSUPPORTED_ORDER = -3, /* order outside [2, 8] */
    BSPLINE_ERR_CUDA = -4,              /* a CUDA runtime call failed */
    BSPLINE_ERR_NONFINITE_INPUT = -5,   /* returned by bspline_status when positions were NaN/Inf */
    BSPLINE_ERR_TIMEOUT = -6,           /* a bounded device-side wait gave up */
    BSPLINE_ERR_NOT_IMPLEMENTED = -7,
    BSPLINE_ERR_OUT_OF_MEMORY = -8,     /* workspace allocation failed */
    BSPLINE_ERR_TOO_LARGE = -9,         /* beyond the fixed scratch of bspline_interp_noalloc */
    BSPLINE_ERR_BOUNDS = -10            /* returned by bspline_status: an index check of a
                                           BSPLINE_CHECKS build failed (the access was skipped) */
};

/* Flags of bspline_interp and bspline_eval. */
#define BSPLINE_INTERP_NO_GRAD 0x1      /* out_grad may be NULL; only u is evaluated */
/* BSPLINE_INTERP_SORTED: the positions are already grouped by the plan's
 * brick (the order bspline_sort_order gives, or any order with the same
 * brick sequence): the count pass writes each particle's located record in
 * place, so the placement pass of the sort is skipped, and each particle's
 * outputs are written at its own index within its brick's range (Section 5:
 * the stencil nodes of Eq. alg-int-6 pick the brick).  The count pass checks
 * the promise: if the order is broken anywhere, the call sorts as without
 * the flag (same results, the time of an unsorted call).  Bricks are never
 * split off to the direct gather under this flag. */
#define BSPLINE_INTERP_SORTED 0x2

/* Create a plan for an N^3 periodic grid, B-spline order `order` (the
 * paper's N: stencil width, degree order-1), coefficient type `dtype`.
 * N: a power of two from 8 to 1024, or 3 * 2^k from 48 to 768 (the
 * transforms add a radix-3 stage).  order: 2..8.  L = 2 pi.
 * Allocates device tables on the current CUDA device.  On success *out
 * receives the plan; on failure *out is set to NULL. */
int bspline_plan(bspline_plan_t* out, int N, int order, bspline_dtype dtype);

/* Domain length L > 0 (finite). */
int bspline_plan_set_length(bspline_plan_t plan, double L);

/* Prefilter choice (default BSPLINE_PREFILTER_INTERP). */
int bspline_plan_set_prefilter(bspline_plan_t plan, bspline_prefilter kind);

/* Band-limited input (no counterpart in the paper, which transforms the full
 * spectrum; pseudo-spectral fields are dealiased, e.g. by the 2/3 rule, and
 * hold no mode beyond a known wavenumber).  kmax > 0 declares that every mode
 * of u_hat with |kx| > kmax, |ky| > kmax or kz > kmax (signed wavenumbers,
 * kz >= 0 in the half spectrum) is zero: bspline_coeffs, bspline_eval and
 * bspline_run_host then neither read those modes nor transform the lines that
 * hold nothing else, and bspline_run_host copies only the box |kx|, |ky|, kz <=
 * kmax from the host.  The coefficients are bit for bit those of the full
 * transform of u_hat with those modes zero (whatever u_hat holds there).
 * kmax = 0 (the default) turns it off.  Errors: INVALID_ARG for kmax < 0 or
 * 2 kmax >= N (the band must leave out the Nyquist planes).  Since the forward
 * path then ignores the modes outside the box, their gradient is zero: the
 * g_u_hat of bspline_spread_adjoint holds zeros there and, inside the box,
 * the full adjoint's bits (the transposed transform skips the ky lines beyond
 * the band). */
int bspline_plan_set_band(bspline_plan_t plan, int kmax);

/* The prefilter c(k) that a plan of this N, order and kind applies along each
 * axis (Section 7: Eq. B_spline_multiplication for INTERP, Eq. B_spline_coeff
 * for L2), computed on the host in FP64 exactly as bspline_plan computes it.
 * out: host array of N doubles, out[k] for the signed wavenumber k mod N.
 * No CUDA call and no plan needed.  Errors: INVALID_ARG (out NULL, bad kind),
 * UNSUPPORTED_N, UNSUPPORTED_ORDER. */
int bspline_prefilter_values(int N, int order, bspline_prefilter kind, double* out);

/* Bind the plan to a cudaStream_t (passed as void*; NULL = legacy stream). */
int bspline_plan_set_stream(bspline_plan_t plan, void* stream);

/* Gather split.  Particles are sorted by brick; a brick holding fewer than
 * direct_below particles is evaluated by the direct gather (each particle's
 * stencil read from global memory, a thread per particle), the others by the
 * staged gather (the brick's coefficient tile staged in shared memory, a CTA
 * per up to 2048 of its particles).  Both give the same results bit for bit;
 * only the time differs: a staged brick carries a fixed cost of a few
 * microseconds of dependent latency, which a handful of particles does not
 * repay.  0 stages every brick.  FP32 and BF16 plans (FP64 plans always
 * stage).  BSPLINE_GATHER_SPLIT_AUTO (the default) takes 32 for a call with
 * fewer than 12 particles per brick on average and 0 otherwise;
 * bspline_plan_autotune picks the split by timing. */
#define BSPLINE_GATHER_SPLIT_AUTO 0xfffffffeu
int bspline_plan_set_gather_split(bspline_plan_t plan, unsigned direct_below);

/* Autotuner of the gather split: times bspline_interp of these P particles
 * (device buffers as for bspline_interp, out_grad NULL for u only) with the
 * split at 0, 8, 32, 128, 512 and "every brick direct", sets the fastest on
 * the plan and returns it in *split_out and its time per call in *ms_out
 * (either may be NULL).  out_u and out_grad are scratch: on return they
 * hold the result of the last timed call.  If the environment variable
 * BSPLINE_AUTOTUNE_CACHE names a file, a choice recorded there for the same
 * (GPU name, N, order, dtype, ceil(log2 P)) is applied without timing
 * (*ms_out = 0), and a new choice is appended to it as one JSON line.
 * Synchronises the plan's stream. */
int bspline_plan_autotune(bspline_plan_t plan, const void* coeffs, const double* x, int64_t P, void* out_u,
                          void* out_grad, unsigned* split_out, double* ms_out);

/* Size in bytes of the coefficient buffer (3 N^3 elements of the dtype). */
int bspline_coeffs_bytes(bspline_plan_t plan, size_t* bytes);

/* Size in bytes of the u_hat buffer (3 N^2 (N/2+1) complex of the dtype's
 * transform type: complex double for F64, complex float otherwise). */
int bspline_uhat_bytes(bspline_plan_t plan, size_t* bytes);

/* Steps 1-2: coeffs = inverse real FFT of c(kx)c(ky)c(kz) u_hat
 * (Section 7, Eqs. B_spline_multiplication_3d and the coefficient transform).
 * u_hat: device, layout above, complex double (F64 plan) or complex float
 * (F32/BF16 plans), 16-byte aligned, not modified.  coeffs: device,
 * bspline_coeffs_bytes() bytes, 16-byte aligned; must not alias u_hat. */
int bspline_coeffs(bspline_plan_t plan, const void* u_hat, void* coeffs);

/* Step 3: evaluate u and grad u at P positions (Sections 3-4, Table 1).
 * coeffs: device, as written by bspline_coeffs.  x: device double [P][3].
 * out_u: device [P][3]; out_grad: device [P][3][3] or NULL with
 * BSPLINE_INTERP_NO_GRAD.  P = 0 is a no-op.  Positions that are NaN or Inf
 * give NaN outputs and are counted in the plan's status word.  Uses plan
 * workspace sized for P (grown on demand; growth synchronises the device). */
int bspline_interp(bspline_plan_t plan, const void* coeffs, const double* x, int64_t P,
                   void* out_u, void* out_grad, int flags);

/* The order in which a plan evaluates particles (Section 5, Eq. alg-int-6:
 * each particle belongs to the brick of cells holding its first stencil
 * node; bricks of 16 x 12 x 16 cells, 16 x 8 x 16 above order 6, 8^3 for
 * FP64 plans, in x-major key order): perm (device int32 [P]) receives the
 * original index of the particle that comes i-th, bricks in key order and
 * non-finite positions last; the order within a brick is arbitrary.  A caller
 * that permutes its positions (and whatever it carries per particle) by perm
 * can then pass BSPLINE_INTERP_SORTED until particles change bricks.  x:
 * device double [P][3].  Uses the plan's particle workspace; asynchronous on
 * the plan's stream. */
int bspline_sort_order(bspline_plan_t plan, const double* x, int64_t P, int32_t* perm);

/* Steps 1-3 in one call on device buffers: bspline_coeffs(u_hat -> coeffs)
 * then bspline_interp(coeffs, x -> out_u, out_grad), arguments and checks as
 * those two.  The particle sort needs only x, so it runs on a second stream
 * of the plan (created on first use at the device's greatest stream
 * priority), concurrently with the coefficient transform, and the
 * evaluation starts once both are done; the call returns after queueing and
 * everything it queued is ordered after earlier work on the plan's stream
 * and before later work on it.  Same results as the two calls. */
int bspline_eval(bspline_plan_t plan, const void* u_hat, void* coeffs, const double* x, int64_t P,
                 void* out_u, void* out_grad, int flags);

/* Adjoint (reverse-mode derivative) of bspline_coeffs + bspline_interp for
 * the loss  sum_p g_u[p] . u(x_p) + sum_p g_grad[p] : grad u(x_p).  The paper
 * has no adjoint; this is the transpose of the maps of Sections 3-4 and 7.
 *   g_u     device [P][3] of the output type, or NULL (= zero);
 *   g_grad  device [P][3][3] of the output type, or NULL (= zero);
 *   g_coeffs device [3][N][N][N] of the OUTPUT type (double for F64 plans,
 *           float otherwise), 16-byte aligned, or NULL: the spread of the
 *           cotangents onto the coefficients is ADDED to it (callers zero it
 *           for a fresh gradient);
 *   g_u_hat device half spectrum [3][N][N][N/2+1], complex double (F64) or
 *           complex float, or NULL: overwritten with the adjoint of the
 *           coefficient transform applied to g_coeffs (after the spread),
 *           c(kx) c(ky) c(kz) m(kz) sum_x g_coeffs(x) exp(-2 pi i k.x / N),
 *           m = 1 for kz = 0 and N/2, else 2 (gradient convention dL/dRe + i dL/dIm);
 *           requires g_coeffs;
 *   g_x     device double [P][3], or NULL: overwritten with dL/dx (second
 *           derivatives of the interpolant enter through g_grad); requires
 *           coeffs (as written by bspline_coeffs); NaN for non-finite positions.
 * x is required when P > 0 and g_coeffs or g_x is given.  Non-finite positions
 * contribute nothing to g_coeffs and are counted in the status word.
 * FP32 and BF16 plans sum each work item's contributions exactly in
 * two-word fixed point at scales taken from the item's largest cotangent
 * (each contribution rounded once, about 40 bits below that bound), convert
 * each node's sum to FP32 once and add the items into g_coeffs with FP32
 * atomics: the order of those additions, and so the last bits, vary between
 * calls, unless bspline_plan_set_deterministic turned on exact sums over all
 * items.  Items holding a non-finite cotangent are summed with FP32 atomics,
 * so NaN and infinities reach the nodes of those particles' stencils.
 * FP64 plans sum with FP64 atomics.  FP32 and BF16 plans keep a copy of the
 * cotangents in the particles' sorted order (64 bytes a particle, grown on
 * first use), which the spread and the position gradients read instead of
 * gathering them from the original indices.  Uses the plan's particle and transform
 * workspaces.  BSPLINE_ERR_INVALID_ARG for a missing required pointer, a bad
 * alignment or P outside [0, 2^31). */
int bspline_spread_adjoint(bspline_plan_t plan, const void* coeffs, const double* x, int64_t P,
                           const void* g_u, const void* g_grad, void* g_coeffs, void* g_u_hat,
                           double* g_x);

/* Deterministic adjoint (FP32 and BF16 plans; FP64 plans: NOT_IMPLEMENTED).
 * By default bspline_spread_adjoint adds the work items' sums to g_coeffs
 * with floating-point atomics, so the order of the additions, and the last
 * bits of g_coeffs and g_u_hat, vary between calls.  With enable = 1 each
 * contribution is computed in FP32 as before and rounded once to an integer
 * at the scale 2^e, one scale for the whole call:
 * e = min(36 - ceil(log2 Gb), 61 - ceil(log2(P Gb)), 118) with
 * Gb = G (1 + 3 N/L) (Gb = G without g_grad) and G the largest |g_u| or
 * |g_grad| over the particles, so that no node's sum can leave the 64-bit
 * range; the integers are summed exactly (integer atomics into a 64-bit
 * accumulator) and converted back once per node: the result is
 * bit-identical from call to call, and each contribution carries an
 * absolute rounding of at most 2^-(e+1).  Costs a [3][N][N][N] int64
 * accumulator in the plan (allocated on first use), a pass over the
 * cotangents and a pass over the accumulator.  A non-finite cotangent makes
 * the call fall back to FP32 atomics (not bit-identical then).  Position
 * gradients and the transform are deterministic in both modes. */
int bspline_plan_set_deterministic(bspline_plan_t plan, int enable);

/* Device workspace bspline_interp needs for P positions. */
int bspline_workspace_bytes(bspline_plan_t plan, int64_t P, size_t* bytes);

/* Synchronise the plan's stream and report the device status words.  Two
 * groups of words: the transform's (cleared when bspline_coeffs, bspline_eval
 * or the transform half of bspline_run_host starts) and the particle side's
 * (cleared when bspline_interp, bspline_eval, bspline_run_host or the particle
 * half of bspline_spread_adjoint starts); each holds until its next start.
 * Returns BSPLINE_ERR_TIMEOUT if a bounded device wait of either ran out: in
 * the transform the coefficients are then unspecified; in the evaluation (a
 * coefficient tile that never arrived) the particles of the abandoned tile get
 * NaN outputs (NaN position gradients in the adjoint).  Else
 * BSPLINE_ERR_BOUNDS if an index check of a BSPLINE_CHECKS build failed, else
 * BSPLINE_ERR_NONFINITE_INPUT if the last particle call met non-finite
 * positions, else BSPLINE_OK.  *nonfinite (may be NULL) receives that count
 * of non-finite positions. */
int bspline_status(bspline_plan_t plan, int64_t* nonfinite);

/* Whole path with HOST buffers: copies u_hat_host and x_host to plan-owned
 * device buffers, runs bspline_coeffs and bspline_interp, copies the results
 * to u_host and grad_host (grad_host may be NULL), and synchronises the
 * plan's stream.  Host buffers should be page-locked for full copy speed. */
int bspline_run_host(bspline_plan_t plan, const void* u_hat_host, const double* x_host, int64_t P,
                     void* u_host, void* grad_host);

/* bspline_run_host without its final synchronisation: returns once the
 * copies and kernels are queued on the plan's streams.  The host buffers
 * must stay valid, the inputs unchanged and the outputs unread until
 * bspline_wait(plan) returns; errors of the queued work are reported there.
 * Calls on one plan run in order (each starts after everything the previous
 * one queued); calls on plans with different streams overlap, so a caller
 * that alternates two plans streams steps with one step's result copy to the
 * host running while the next step's inputs are copied in. */
int bspline_run_host_async(bspline_plan_t plan, const void* u_hat_host, const double* x_host, int64_t P,
                           void* u_host, void* grad_host);

/* Wait for all work queued on the plan (all of its streams); the first CUDA
 * error of that work, else BSPLINE_OK. */
int bspline_wait(bspline_plan_t plan);

/* Free the plan, its tables and workspace.  NULL is accepted. */
int bspline_destroy(bspline_plan_t plan);

/* Static string for a status code. */
const char* bspline_status_string(int status);

/* Library version string. */
const char* bspline_version(void);

/* Per-kernel device timing, for profiling.  When enabled, every kernel the
 * plan launches is bracketed by CUDA events recorded on the plan's stream;
 * bspline_stage_times synchronises the stream and adds the elapsed times
 * (milliseconds) and launch counts of all calls since the last reset into
 * ms[i] and launches[i], i < BSPLINE_NSTAGES (either pointer may be NULL),
 * then clears the record.  Disabled by default; enabling or disabling clears
 * the record.  The stage index identifies the kernel: */
enum {
    BSPLINE_STAGE_FFT_X = 0,    /* prefilter + c2c along kx */
    BSPLINE_STAGE_FFT_YZ = 1,   /* c2c along ky and c2r along kz, store coefficients */
    BSPLINE_STAGE_BIN = 2,      /* locate + brick histogram */
    BSPLINE_STAGE_SCAN = 3,     /* brick offsets */
    BSPLINE_STAGE_SCATTER = 4,  /* counting-sort scatter */
    BSPLINE_STAGE_GATHER = 5,   /* weights + stencil contraction */
    BSPLINE_STAGE_SPREAD = 6,   /* adjoint: cotangents spread onto coefficients */
    BSPLINE_STAGE_GRAD_X = 7,   /* adjoint: position gradients */
    BSPLINE_STAGE_ADJ_FFT = 8,  /* adjoint: forward real transform + prefilter */
    BSPLINE_STAGE_GATHER_DIRECT = 9,   /* gather of the sparse bricks from global memory */
    BSPLINE_NSTAGES = 10
};
int bspline_plan_set_timing(bspline_plan_t plan, int enable);
int bspline_stage_times(bspline_plan_t plan, double* ms, int64_t* launches);

/* Test hooks.  BSPLINE_TEST_DROP_TRANSFORM_SIGNALS makes the ky-transform
 * items of bspline_coeffs skip their completion signals, so the waits that
 * depend on them run out after about a second: the kernel then stops, leaves
 * the coefficients unspecified, and bspline_status reports
 * BSPLINE_ERR_TIMEOUT.  It exists to test that error path.
 * BSPLINE_TEST_NO_TMA stages every brick of the FP32 gather and of the FP32
 * position gradient with cp.async instead of TMA tensor copies (same tile,
 * same results), to compare the two paths.  0 clears. */
#define BSPLINE_TEST_DROP_TRANSFORM_SIGNALS 0x1
#define BSPLINE_TEST_NO_TMA 0x2
/* BSPLINE_TEST_SKIP_TMA_ISSUE: FP32 tiles that would come by TMA arm their
 * shared-memory barrier for the tile's bytes but issue no copy, so the tile
 * wait runs out after about a second with nothing in flight: those items are
 * abandoned with NaN outputs and bspline_status reports BSPLINE_ERR_TIMEOUT.
 * It exists to test that error path. */
#define BSPLINE_TEST_SKIP_TMA_ISSUE 0x4
int bspline_plan_set_test_hooks(bspline_plan_t plan, int hooks);

/* Allocation-free evaluation of u and grad u (no counterpart in the paper: it
 * serves callers, not the method).  Some callers cannot allocate device
 * memory: code running inside a CUDA graph capture that another framework
 * owns (allocation cannot be captured), code that must never stall the GPU
 * (cudaMalloc and cudaFree may synchronise the device), and processes whose
 * device memory belongs to another allocator with a fixed budget.  This entry
 * point needs no plan and calls no allocator: it does what bspline_interp
 * does on a plan with the same N, order, dtype and L, with all scratch in one
 * fixed 16 MiB device array inside the library (present on every GPU that
 * loads the library until the process exits).
 * Arguments as bspline_interp, plus: N, order, dtype, L (domain length; the
 * coefficients come from bspline_coeffs of such a plan) and stream (a
 * cudaStream_t as void*, NULL = legacy stream).
 * Limits: N <= BSPLINE_NOALLOC_MAX_N and P <= BSPLINE_NOALLOC_MAX_PARTICLES,
 * else BSPLINE_ERR_TOO_LARGE is returned before any device work.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture.  All calls share the one array, whose contents persist between
 * calls; each call clears the parts that must start at zero.  Calls that
 * overlap on the GPU (concurrent streams or host threads) race on the array,
 * so serialise them.  Non-finite positions give NaN outputs; their count is
 * not reported (there is no plan to hold a status word).  A coefficient tile
 * whose copy never completes (a bounded wait of about a second runs out)
 * leaves NaN outputs for the particles of that tile; this is not reported
 * otherwise either.  The cached address belongs to the device's primary
 * context: after cudaDeviceReset the library must be reloaded before this
 * entry point is used again. */
#define BSPLINE_NOALLOC_MAX_N 256
#define BSPLINE_NOALLOC_MAX_PARTICLES 131072
int bspline_interp_noalloc(const void* coeffs, int N, int order, bspline_dtype dtype, double L,
                           const double* x, int64_t P, void* out_u, void* out_grad, int flags,
                           void* stream);

/* ---- Batches of independent fields.  No counterpart in the paper: a launch
 * structure for many small fields (grid size, order and dtype may differ per
 * field), whose short kernels would otherwise leave the GPU idle.
 * When every field has an FP32 plan of one order and u and grad u are wanted
 * for every field with particles, the fields of one grid size and prefilter
 * are transformed together (one launch of each transform kernel per group, in
 * workspace the batch owns), and the particle side of all fields runs as one
 * persistent kernel after the transforms: a device work queue of count, scan,
 * placement and gather tasks (the steps of bspline_interp; Section 5 locate,
 * Sections 3-4 evaluation), taken in order by every CTA, each task waiting
 * (bounded, about a second) for the tasks of its field that it needs; it
 * stages bricks of 16 x brick_y x 16 cells and gathers up to item_particles
 * particles of a brick per task (both tuned by bspline_batch_autotune).
 * Other batches record each field's bspline_interp after its transform.
 * bspline_batch_create: nfields >= 1 plans (all on one device; one plan may
 * serve several fields, which then run one after another).  The batch keeps
 * the plan handles, not ownership: destroy it before its plans.
 * bspline_batch_capture: records bspline_coeffs(u_hat[i] -> coeffs[i]) and
 * bspline_interp(coeffs[i], x[i], P[i] -> out_u[i], out_grad[i]) for every
 * field into one CUDA graph, the fields spread round-robin over `streams`
 * concurrent streams by plan.  Arrays of nfields device pointers (host arrays
 * of pointers; out_grad may be NULL for u only, or hold NULL entries); the
 * same argument rules as the single-field calls; plan workspaces are grown
 * here, outside the graph.  Nothing runs until a launch.
 * bspline_batch_launch: replays the graph with one launch on `stream`
 * (cudaStream_t, NULL = legacy stream); every launch rereads u_hat and x and
 * rewrites coeffs and the outputs named at capture.  Status words of the
 * plans are read with bspline_status as usual.
 * bspline_batch_autotune: captures with 1, 2, 4, 8, 16 streams (up to the
 * number of distinct plans), times three graph launches of each on `stream`,
 * keeps the fastest graph; best_streams and best_ms (mean time of one launch)
 * may be NULL.  Requires an earlier capture (its arguments are reused).
 * Errors: BSPLINE_ERR_INVALID_ARG for bad arguments or a launch before a
 * capture; BSPLINE_ERR_CUDA / OUT_OF_MEMORY from the runtime. */
typedef struct bspline_batch_s* bspline_batch_t;
int bspline_batch_create(bspline_batch_t* out, int nfields, const bspline_plan_t* plans);
int bspline_batch_capture(bspline_batch_t batch, int streams, const void* const* u_hat, void* const* coeffs,
                          const double* const* x, const int64_t* P, void* const* out_u, void* const* out_grad);
int bspline_batch_launch(bspline_batch_t batch, void* stream);
int bspline_batch_autotune(bspline_batch_t batch, void* stream, int* best_streams, double* best_ms);
int bspline_batch_destroy(bspline_batch_t batch);

/* bspline_batch_autotune (continued): for a batch that runs the queue it then
 * times brick_y in {8, 12, 16} (12 up to order 6) and item_particles in {512,
 * 1024, 2048} at the best stream count and keeps the fastest.  If the
 * environment variable BSPLINE_AUTOTUNE_CACHE names a file, a choice recorded
 * there for the same GPU, order, dtype and fields (grids, particle counts,
 * grad) is recaptured without timing (*best_ms = 0), and a new choice is
 * appended as one JSON line.
 * bspline_batch_set_layout: queue = -1 (use the queue when the fields allow
 * it, the default), 0 (never), 1 (required: BSPLINE_ERR_NOT_IMPLEMENTED if
 * the fields do not allow it); brick_y_cells 0 (the plans' default), 8, 12 or
 * 16 (8 or 16 above order 6); item_particles 32..2048.  Recaptures if
 * arguments were captured before.
 * bspline_batch_config: the current graph's choices; queue = 1 if it runs the
 * queue kernel; kernel_nodes = kernel launches in one replay of the graph.
 * Any output pointer may be NULL.
 * bspline_batch_status: synchronises the stream of the last launch and reads
 * the queue's status: BSPLINE_ERR_TIMEOUT if a wait of that launch ran out
 * (the outputs of that launch are then unspecified), else
 * BSPLINE_ERR_NONFINITE_INPUT with the count of non-finite positions over all
 * fields in *nonfinite, else BSPLINE_OK (also for a batch without the queue,
 * whose plans report through bspline_status).
 * bspline_batch_set_test_hooks: BSPLINE_TEST_DROP_QUEUE_SIGNAL makes the
 * first count task of field 0 skip its completion signal, so the scan of
 * field 0 waits until its bounded wait runs out; it exists to test that
 * error path.  0 clears.  Recaptures if arguments were captured before. */
#define BSPLINE_TEST_DROP_QUEUE_SIGNAL 0x8
int bspline_batch_set_layout(bspline_batch_t batch, int queue, int brick_y_cells, int item_particles);
int bspline_batch_config(bspline_batch_t batch, int* queue, int* streams, int* brick_y_cells, int* item_particles,
                         int* kernel_nodes);
int bspline_batch_status(bspline_batch_t batch, int64_t* nonfinite);
int bspline_batch_set_test_hooks(bspline_batch_t batch, int hooks);

#ifdef __cplusplus
}
#endif

#endif /* BSPLINE_H */

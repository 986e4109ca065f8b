// C ABI of the library: plan life cycle, argument checks, host-side tables.
//
// Tables are computed on the host in FP64 when a plan is made:
//   * node values B_(n)(d) of the centred B-spline by the Cox-de Boor
//     recurrence of the cardinal B-spline M_n (B_(n)(y) = M_n(y + n/2));
//   * prefilter c(k) = 1 / sum_d B_(n)(d) cos(2 pi k d / N) (Section 7,
//     Eq. B_spline_multiplication: F_D[B_D] is real because B is even), or
//     the L2-optimal c(k) = sinc(kappa)^n / sum_d B_(2n)(d) cos(2 pi kappa d)
//     (Eq. B_spline_coeff; its alias sum of sinc^(2n) is the cosine series of
//     the node values of B_(2n) by Poisson summation);
//   * twiddles exp(+2 pi i m / N) with quadrant reduction of the angle.
// The FP64 values are rounded to FP32 once for the FP32/BF16 plans.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace bs {

int set_cuda_error(cudaError_t e) {
    if (e == cudaSuccess) return BSPLINE_OK;
    if (e == cudaErrorMemoryAllocation) return BSPLINE_ERR_OUT_OF_MEMORY;
    return BSPLINE_ERR_CUDA;
}

int DeviceBuffer::grow(size_t need) {
    if (need <= bytes && ptr) return BSPLINE_OK;
    release();
    if (need == 0) return BSPLINE_OK;
    cudaError_t e = cudaMalloc(&ptr, need);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        cudaGetLastError();
        return set_cuda_error(e);
    }
    bytes = need;
    return BSPLINE_OK;
}

static cudaEvent_t take_event(bspline_plan_s* p) {
    if (!p->free_events.empty()) {
        cudaEvent_t e = p->free_events.back();
        p->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

StageTimer::StageTimer(bspline_plan_s* plan, int s) : p(plan), stage(s) {
    if (!p->timing) return;
    start = take_event(p);
    if (start) cudaEventRecord(start, p->stream);
}

StageTimer::~StageTimer() {
    if (!p->timing || !start) return;
    cudaEvent_t stop = take_event(p);
    if (!stop) {
        p->free_events.push_back(start);
        return;
    }
    cudaEventRecord(stop, p->stream);
    p->pending.push_back(PendingTiming{stage, start, stop});
}

void DeviceBuffer::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

namespace {

const double kPi = 3.14159265358979323846264338327950288;

// Cardinal B-spline of order k (support [0, k)) by the Cox-de Boor recurrence.
double cardinal(int k, double x) {
    if (k == 1) return (x >= 0.0 && x < 1.0) ? 1.0 : 0.0;
    return (x * cardinal(k - 1, x) + (k - x) * cardinal(k - 1, x - 1.0)) / (k - 1);
}

// Node values B_(n)(d), d = -h..h with h = n/2 + 1 (zero outside the support).
std::vector<double> node_values(int n) {
    const int h = n / 2 + 1;
    std::vector<double> b(2 * h + 1);
    for (int d = -h; d <= h; ++d) b[d + h] = cardinal(n, d + 0.5 * n);
    return b;
}

// exp(2 pi i m / N) for N divisible by 4, angle reduced to the first octant.
void twiddle(int m, int N, double* re, double* im) {
    m = ((m % N) + N) % N;
    const int q = (4 * m) / N;
    const int r = m - q * (N / 4);
    double c, s;
    if (8 * r <= N) {
        c = std::cos(2.0 * kPi * r / N);
        s = std::sin(2.0 * kPi * r / N);
    } else {
        const int rr = N / 4 - r;
        c = std::sin(2.0 * kPi * rr / N);
        s = std::cos(2.0 * kPi * rr / N);
    }
    switch (q) {
        case 0: *re = c; *im = s; break;
        case 1: *re = -s; *im = c; break;
        case 2: *re = -c; *im = -s; break;
        default: *re = s; *im = -c; break;
    }
}

// The prefilter c(k), k = 0..N-1, of an order-n plan of the given kind, in FP64.
std::vector<double> prefilter_table(int N, int n, int kind) {
    const std::vector<double> b = node_values(n);
    const std::vector<double> b2 = node_values(2 * n);
    const int h = n / 2 + 1, h2 = n + 1;
    std::vector<double> c(N);
    for (int k = 0; k < N; ++k) {
        const int ks = (k < N / 2) ? k : k - N;
        double v;
        if (kind == BSPLINE_PREFILTER_INTERP) {
            // F_D[B_D](k) = sum_d B(d) cos(2 pi k d / N), phase k d reduced mod N exactly
            double s = 0.0;
            for (int d = -h; d <= h; ++d) {
                if (b[d + h] == 0.0) continue;
                double re, im;
                twiddle((int)(((long long)k * d) % N), N, &re, &im);
                s += b[d + h] * re;
            }
            v = 1.0 / s;
        } else {
            const double x = kPi * ks / N;
            const double sinc = (ks == 0) ? 1.0 : std::sin(x) / x;
            double s = 0.0;
            for (int d = -h2; d <= h2; ++d) {
                if (b2[d + h2] == 0.0) continue;
                double re, im;
                twiddle((int)(((long long)k * d) % N), N, &re, &im);
                s += b2[d + h2] * re;
            }
            v = std::pow(sinc, n) / s;
        }
        c[k] = v;
    }
    return c;
}

int upload_prefilter(bspline_plan_s* p) {
    const int N = p->N;
    const std::vector<double> c = prefilter_table(N, p->order, p->prefilter);
    std::vector<float> cf(N);
    for (int k = 0; k < N; ++k) cf[k] = (float)c[k];
    cudaError_t e = cudaMemcpy(p->d_c64, c.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_c32, cf.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
    return set_cuda_error(e);
}

int upload_twiddles(bspline_plan_s* p) {
    const int N = p->N;
    std::vector<double2> t(N);
    std::vector<float2> tf(N);
    for (int m = 0; m < N; ++m) {
        double re, im;
        twiddle(m, N, &re, &im);
        t[m] = make_double2(re, im);
        tf[m] = make_float2((float)re, (float)im);
    }
    cudaError_t e = cudaMemcpy(p->d_tw64, t.data(), sizeof(double2) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw32, tf.data(), sizeof(float2) * N, cudaMemcpyHostToDevice);
    return set_cuda_error(e);
}

bool valid_plan(bspline_plan_t p) { return p != nullptr && p->N > 0; }

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// Makes the plan's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; cudaGetLastError(); return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) { ok = false; cudaGetLastError(); }
    }
    ~DeviceGuard() {
        int cur;
        if (ok && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t elem_bytes(int dtype) {
    return dtype == BSPLINE_F64 ? 8 : (dtype == BSPLINE_F32 ? 4 : 2);
}

size_t out_bytes(int dtype) { return dtype == BSPLINE_F64 ? 8 : 4; }

size_t uhat_bytes_of(const bspline_plan_s* p) {
    return (p->dtype == BSPLINE_F64 ? 16 : 8) * 3 * (size_t)p->N * p->N * (p->N / 2 + 1);
}

size_t coef_bytes_of(const bspline_plan_s* p) { return elem_bytes(p->dtype) * 3 * (size_t)p->N * p->N * p->N; }

void clear_timing(bspline_plan_s* p) {
    for (auto& t : p->pending) {
        p->free_events.push_back(t.start);
        p->free_events.push_back(t.stop);
    }
    p->pending.clear();
}

void free_plan(bspline_plan_s* p) {
    clear_timing(p);
    for (cudaEvent_t e : p->free_events) cudaEventDestroy(e);
    p->free_events.clear();
    if (p->d_c64) cudaFree(p->d_c64);
    if (p->d_c32) cudaFree(p->d_c32);
    if (p->d_tw64) cudaFree(p->d_tw64);
    if (p->d_tw32) cudaFree(p->d_tw32);
    if (p->d_status) cudaFree(p->d_status);
    p->work.release();
    p->pws.release();
    p->det.release();
    p->cot.release();
    if (p->aux_stream) cudaStreamDestroy(p->aux_stream);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->ev_sorted) cudaEventDestroy(p->ev_sorted);
    for (cudaEvent_t ev : p->ev_copied)
        if (ev) cudaEventDestroy(ev);
    p->host_uhat.release();
    p->host_coef.release();
    p->host_x.release();
    p->host_u.release();
    p->host_grad.release();
    p->N = 0;
    delete p;
}

// The plan's second stream and its two events, created on first use.
int ensure_aux(bspline_plan_s* plan) {
    cudaError_t e = cudaSuccess;
    // the sort is short and gates the gather: at the greatest priority its blocks are dispatched ahead of the
    // transform's waiting blocks, so it runs alongside the transform instead of after it
    if (!plan->aux_stream) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&plan->aux_stream, cudaStreamNonBlocking, greatest);
    }
    if (e == cudaSuccess && !plan->ev_start) e = cudaEventCreateWithFlags(&plan->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess && !plan->ev_sorted) e = cudaEventCreateWithFlags(&plan->ev_sorted, cudaEventDisableTiming);
    return set_cuda_error(e);
}

// The copy stream and its events, created on first use.
int ensure_copy(bspline_plan_s* plan) {
    cudaError_t e = cudaSuccess;
    if (!plan->copy_stream) e = cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking);
    for (cudaEvent_t& ev : plan->ev_copied)
        if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    return set_cuda_error(e);
}

}  // namespace
}  // namespace bs

using namespace bs;

extern "C" {

int bspline_plan(bspline_plan_t* out, int N, int order, bspline_dtype dtype) {
    if (!out) return BSPLINE_ERR_INVALID_ARG;
    *out = nullptr;
    if (dtype != BSPLINE_F64 && dtype != BSPLINE_F32 && dtype != BSPLINE_BF16) return BSPLINE_ERR_INVALID_ARG;
    if (!bs::supported_grid(N)) return BSPLINE_ERR_UNSUPPORTED_N;
    if (order < 2 || order > 8) return BSPLINE_ERR_UNSUPPORTED_ORDER;
    bspline_plan_s* p = new (std::nothrow) bspline_plan_s();
    if (!p) return BSPLINE_ERR_OUT_OF_MEMORY;
    p->N = N;
    p->order = order;
    p->dtype = dtype;
    p->L = 2.0 * kPi;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_c64, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_c32, sizeof(float) * N);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tw64, sizeof(double2) * N);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tw32, sizeof(float2) * N);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(unsigned long long) * kStatusWords);
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(unsigned long long) * kStatusWords);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return set_cuda_error(e);
    }
    int rc = upload_prefilter(p);
    if (!rc) rc = upload_twiddles(p);
    if (rc) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return BSPLINE_OK;
}

int bspline_prefilter_values(int N, int order, bspline_prefilter kind, double* out) {
    if (!out) return BSPLINE_ERR_INVALID_ARG;
    if (kind != BSPLINE_PREFILTER_INTERP && kind != BSPLINE_PREFILTER_L2) return BSPLINE_ERR_INVALID_ARG;
    if (!bs::supported_grid(N)) return BSPLINE_ERR_UNSUPPORTED_N;
    if (order < 2 || order > 8) return BSPLINE_ERR_UNSUPPORTED_ORDER;
    const std::vector<double> c = prefilter_table(N, order, kind);
    std::memcpy(out, c.data(), sizeof(double) * N);
    return BSPLINE_OK;
}

int bspline_plan_set_length(bspline_plan_t plan, double L) {
    if (!valid_plan(plan) || !(L > 0.0) || !std::isfinite(L)) return BSPLINE_ERR_INVALID_ARG;
    plan->L = L;
    return BSPLINE_OK;
}

int bspline_plan_set_prefilter(bspline_plan_t plan, bspline_prefilter kind) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    if (kind != BSPLINE_PREFILTER_INTERP && kind != BSPLINE_PREFILTER_L2) return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    plan->prefilter = kind;
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) return set_cuda_error(e);
    return upload_prefilter(plan);
}

int bspline_plan_set_band(bspline_plan_t plan, int kmax) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    if (kmax < 0 || (kmax > 0 && 2 * kmax >= plan->N)) return BSPLINE_ERR_INVALID_ARG;
    plan->band = kmax;
    return BSPLINE_OK;
}

int bspline_plan_set_stream(bspline_plan_t plan, void* stream) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    plan->stream = (cudaStream_t)stream;
    return BSPLINE_OK;
}

int bspline_coeffs_bytes(bspline_plan_t plan, size_t* bytes) {
    if (!valid_plan(plan) || !bytes) return BSPLINE_ERR_INVALID_ARG;
    *bytes = coef_bytes_of(plan);
    return BSPLINE_OK;
}

int bspline_uhat_bytes(bspline_plan_t plan, size_t* bytes) {
    if (!valid_plan(plan) || !bytes) return BSPLINE_ERR_INVALID_ARG;
    *bytes = uhat_bytes_of(plan);
    return BSPLINE_OK;
}

int bspline_coeffs(bspline_plan_t plan, const void* u_hat, void* coeffs) {
    if (!valid_plan(plan) || !u_hat || !coeffs) return BSPLINE_ERR_INVALID_ARG;
    if (!aligned(u_hat, 16) || !aligned(coeffs, 16)) return BSPLINE_ERR_INVALID_ARG;
    const char* a = (const char*)u_hat;
    const char* b = (const char*)coeffs;
    if (a < b + coef_bytes_of(plan) && b < a + uhat_bytes_of(plan)) return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    return launch_coeffs(plan, u_hat, coeffs);
}

int bspline_interp(bspline_plan_t plan, const void* coeffs, const double* x, int64_t P, void* out_u,
                   void* out_grad, int flags) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    if (flags & ~(BSPLINE_INTERP_NO_GRAD | BSPLINE_INTERP_SORTED)) return BSPLINE_ERR_INVALID_ARG;
    if (P < 0 || P > 0x7fffffffLL) return BSPLINE_ERR_INVALID_ARG;
    if (P == 0) return BSPLINE_OK;
    if (!coeffs || !x || !out_u) return BSPLINE_ERR_INVALID_ARG;
    if (!(flags & BSPLINE_INTERP_NO_GRAD) && !out_grad) return BSPLINE_ERR_INVALID_ARG;
    const size_t ob = out_bytes(plan->dtype);
    if (!aligned(coeffs, 16) || !aligned(x, 8) || !aligned(out_u, ob) || (out_grad && !aligned(out_grad, ob)))
        return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    return launch_interp(plan, coeffs, x, P, out_u, out_grad, flags);
}

int bspline_eval(bspline_plan_t plan, const void* u_hat, void* coeffs, const double* x, int64_t P, void* out_u,
                 void* out_grad, int flags) {
    if (!valid_plan(plan) || !u_hat || !coeffs) return BSPLINE_ERR_INVALID_ARG;
    if (!aligned(u_hat, 16) || !aligned(coeffs, 16)) return BSPLINE_ERR_INVALID_ARG;
    const char* a = (const char*)u_hat;
    const char* b = (const char*)coeffs;
    if (a < b + coef_bytes_of(plan) && b < a + uhat_bytes_of(plan)) return BSPLINE_ERR_INVALID_ARG;
    if (flags & ~(BSPLINE_INTERP_NO_GRAD | BSPLINE_INTERP_SORTED)) return BSPLINE_ERR_INVALID_ARG;
    if (P < 0 || P > 0x7fffffffLL) return BSPLINE_ERR_INVALID_ARG;
    if (P > 0) {
        if (!x || !out_u) return BSPLINE_ERR_INVALID_ARG;
        if (!(flags & BSPLINE_INTERP_NO_GRAD) && !out_grad) return BSPLINE_ERR_INVALID_ARG;
        const size_t ob = out_bytes(plan->dtype);
        if (!aligned(x, 8) || !aligned(out_u, ob) || (out_grad && !aligned(out_grad, ob)))
            return BSPLINE_ERR_INVALID_ARG;
    }
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    int rc;
    if (P == 0) return launch_coeffs(plan, u_hat, coeffs);
    if ((rc = ensure_aux(plan))) return rc;
    // the second stream starts after everything already queued on the plan's stream
    cudaError_t e = cudaEventRecord(plan->ev_start, plan->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->aux_stream, plan->ev_start, 0);
    if (e != cudaSuccess) return set_cuda_error(e);
    if ((rc = launch_coeffs(plan, u_hat, coeffs))) return rc;
    return launch_interp_split(plan, coeffs, x, P, out_u, out_grad, flags, plan->aux_stream, plan->ev_sorted);
}

int bspline_sort_order(bspline_plan_t plan, const double* x, int64_t P, int32_t* perm) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    if (P < 0 || P > 0x7fffffffLL) return BSPLINE_ERR_INVALID_ARG;
    if (P == 0) return BSPLINE_OK;
    if (!x || !perm || !aligned(x, 8) || !aligned(perm, 4)) return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    return launch_sort_order(plan, x, P, perm);
}

int bspline_spread_adjoint(bspline_plan_t plan, const void* coeffs, const double* x, int64_t P, const void* g_u,
                           const void* g_grad, void* g_coeffs, void* g_u_hat, double* g_x) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    if (P < 0 || P > 0x7fffffffLL) return BSPLINE_ERR_INVALID_ARG;
    if (g_u_hat && !g_coeffs) return BSPLINE_ERR_INVALID_ARG;
    const bool particles = P > 0 && (g_coeffs || g_x);
    if (particles && !x) return BSPLINE_ERR_INVALID_ARG;
    if (P > 0 && g_x && !coeffs) return BSPLINE_ERR_INVALID_ARG;
    const size_t ob = out_bytes(plan->dtype);
    if (!aligned(coeffs, 16) || !aligned(x, 8) || !aligned(g_u, ob) || !aligned(g_grad, ob) ||
        !aligned(g_coeffs, 16) || !aligned(g_u_hat, 16) || !aligned(g_x, 8))
        return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    int rc;
    if (particles && (rc = launch_adjoint_particles(plan, coeffs, x, P, g_u, g_grad, g_coeffs, g_x)))
        return rc;
    if (g_u_hat) {
        if ((rc = plan->work.grow(coeffs_workspace_bytes(plan)))) return rc;
        if ((rc = launch_adjoint_transform(plan, g_coeffs, g_u_hat))) return rc;
    }
    return BSPLINE_OK;
}

int bspline_workspace_bytes(bspline_plan_t plan, int64_t P, size_t* bytes) {
    if (!valid_plan(plan) || !bytes || P < 0 || P > 0x7fffffffLL) return BSPLINE_ERR_INVALID_ARG;
    *bytes = interp_workspace_bytes(plan, P);
    return BSPLINE_OK;
}

int bspline_status(bspline_plan_t plan, int64_t* nonfinite) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    unsigned long long h[kStatusWords] = {};
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    if (e == cudaSuccess) e = cudaMemcpy(h, plan->d_status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (nonfinite) *nonfinite = (int64_t)h[kStatusNonfinite];
    if (h[kStatusParticleTimeout] || h[kStatusTransformTimeout]) return BSPLINE_ERR_TIMEOUT;
    if (h[kStatusBounds]) return BSPLINE_ERR_BOUNDS;
    return h[kStatusNonfinite] ? BSPLINE_ERR_NONFINITE_INPUT : BSPLINE_OK;
}

int bspline_plan_set_deterministic(bspline_plan_t plan, int enable) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    if (enable && plan->dtype == BSPLINE_F64) return BSPLINE_ERR_NOT_IMPLEMENTED;
    plan->deterministic = enable ? 1 : 0;
    return BSPLINE_OK;
}

int bspline_plan_set_gather_split(bspline_plan_t plan, unsigned direct_below) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    plan->direct_below = direct_below;
    return BSPLINE_OK;
}

int bspline_plan_autotune(bspline_plan_t plan, const void* coeffs, const double* x, int64_t P, void* out_u,
                          void* out_grad, unsigned* split_out, double* ms_out) {
    if (!valid_plan(plan) || P <= 0 || P > 0x7fffffffLL || !coeffs || !x || !out_u) return BSPLINE_ERR_INVALID_ARG;
    const size_t ob = out_bytes(plan->dtype);
    if (!aligned(coeffs, 16) || !aligned(x, 8) || !aligned(out_u, ob) || (out_grad && !aligned(out_grad, ob)))
        return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    const int flags = out_grad ? 0 : BSPLINE_INTERP_NO_GRAD;
    // cache key: GPU name, grid, order, dtype, particle count rounded up to a power of two
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, plan->device);
    if (e != cudaSuccess) return set_cuda_error(e);
    int plog2 = 0;
    while (plog2 < 62 && (1LL << plog2) < (long long)P) ++plog2;
    static const char* kDtype[] = {"f64", "f32", "bf16"};
    char key[384];
    std::snprintf(key, sizeof key, "%s|N%d|o%d|%s|p2^%d", prop.name, plan->N, plan->order, kDtype[plan->dtype], plog2);
    const char* path = std::getenv("BSPLINE_AUTOTUNE_CACHE");
    if (path && *path) {
        if (FILE* f = std::fopen(path, "r")) {
            char line[1024];
            char want[448];
            std::snprintf(want, sizeof want, "\"key\": \"%s\"", key);
            bool found = false;
            unsigned split = 0;
            while (std::fgets(line, sizeof line, f)) {
                const char* k = std::strstr(line, want);
                const char* s = std::strstr(line, "\"direct_below\": ");
                if (k && s && std::sscanf(s + 16, "%u", &split) == 1) found = true;   // the last match wins
            }
            std::fclose(f);
            if (found) {
                plan->direct_below = split;
                if (split_out) *split_out = split;
                if (ms_out) *ms_out = 0.0;
                return BSPLINE_OK;
            }
        }
    }
    static const unsigned kSplits[] = {0u, 8u, 32u, 128u, 512u, 0xffffffffu};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int rc = set_cuda_error(e);
    unsigned best = plan->direct_below;
    float best_ms = -1.f;
    for (unsigned split : kSplits) {
        if (rc) break;
        plan->direct_below = split;
        if ((rc = launch_interp(plan, coeffs, x, P, out_u, out_grad, flags))) break;     // warm-up
        if ((e = cudaEventRecord(e0, plan->stream)) != cudaSuccess) { rc = set_cuda_error(e); break; }
        for (int r = 0; r < 3 && rc == BSPLINE_OK; ++r) rc = launch_interp(plan, coeffs, x, P, out_u, out_grad, flags);
        if (rc) break;
        float ms = 0.f;
        e = cudaEventRecord(e1, plan->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if ((rc = set_cuda_error(e))) break;
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = split;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    plan->direct_below = best;
    if (rc) return rc;
    if (split_out) *split_out = best;
    if (ms_out) *ms_out = best_ms / 3.0;
    if (path && *path) {
        if (FILE* f = std::fopen(path, "a")) {
            std::fprintf(f, "{\"key\": \"%s\", \"direct_below\": %u, \"ms\": %.4f}\n", key, best, best_ms / 3.0);
            std::fclose(f);
        }
    }
    return BSPLINE_OK;
}

int bspline_plan_set_test_hooks(bspline_plan_t plan, int hooks) {
    if (!valid_plan(plan) ||
        (hooks & ~(BSPLINE_TEST_DROP_TRANSFORM_SIGNALS | BSPLINE_TEST_NO_TMA | BSPLINE_TEST_SKIP_TMA_ISSUE)))
        return BSPLINE_ERR_INVALID_ARG;
    plan->test_hooks = hooks;
    return BSPLINE_OK;
}

// Copies and compute overlap on three streams: the copy stream brings the
// positions and then the three u_hat components in back to back, so the
// host-to-device link never waits for a kernel; the second stream sorts the
// positions as soon as they have arrived, and the plan's stream transforms
// each component as soon as it has arrived; the gather waits for the sort
// and the last component, then the results are copied back on the plan's
// stream.  Returns once all of it is queued.
// With a band (bspline_plan_set_band) only the box |kx|, |ky|, kz <= band of each
// component crosses the host link: four pitched 3D copies (kx and ky each in
// [0, band] and [N - band, N)), rows of band + 1 modes; the transform reads
// nothing else.
static cudaError_t copy_band_h2d(const bspline_plan_s* p, void* dst, const void* src, int comp, size_t elem,
                                 cudaStream_t s) {
    const int N = p->N, H = N / 2 + 1, K = p->band;
    const int first[2] = {0, N - K}, count[2] = {K + 1, K};
    for (int a = 0; a < 2; ++a) {                       // kx range
        for (int b = 0; b < 2; ++b) {                   // ky range
            cudaMemcpy3DParms m = {};
            m.srcPtr = make_cudaPitchedPtr(const_cast<void*>(src), H * elem, H * elem, (size_t)N);
            m.dstPtr = make_cudaPitchedPtr(dst, H * elem, H * elem, (size_t)N);
            m.srcPos = make_cudaPos(0, (size_t)first[b], (size_t)comp * N + (size_t)first[a]);
            m.dstPos = m.srcPos;
            m.extent = make_cudaExtent((size_t)(K + 1) * elem, (size_t)count[b], (size_t)count[a]);
            m.kind = cudaMemcpyHostToDevice;
            const cudaError_t e = cudaMemcpy3DAsync(&m, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

int bspline_run_host_async(bspline_plan_t plan, const void* u_hat_host, const double* x_host, int64_t P,
                           void* u_host, void* grad_host) {
    if (!valid_plan(plan) || !u_hat_host || !u_host || (P > 0 && !x_host)) return BSPLINE_ERR_INVALID_ARG;
    if (P < 0 || P > 0x7fffffffLL) return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    const size_t ob = out_bytes(plan->dtype);
    int rc;
    if ((rc = plan->host_uhat.grow(uhat_bytes_of(plan)))) return rc;
    if ((rc = plan->host_coef.grow(coef_bytes_of(plan)))) return rc;
    if ((rc = plan->host_x.grow(sizeof(double) * 3 * (size_t)(P ? P : 1)))) return rc;
    if ((rc = plan->host_u.grow(ob * 3 * (size_t)(P ? P : 1)))) return rc;
    if ((rc = plan->host_grad.grow(ob * 9 * (size_t)(P ? P : 1)))) return rc;
    if ((rc = ensure_aux(plan)) || (rc = ensure_copy(plan))) return rc;
    cudaStream_t st = plan->stream, aux = plan->aux_stream, cp = plan->copy_stream;
    // the other streams start after everything already queued on the plan's stream (which ends
    // with the previous call's result copies, after every reader of the device buffers)
    cudaError_t e = cudaEventRecord(plan->ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, plan->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cp, plan->ev_start, 0);
    if (e == cudaSuccess && P)
        e = cudaMemcpyAsync(plan->host_x.ptr, x_host, sizeof(double) * 3 * P, cudaMemcpyHostToDevice, cp);
    if (e == cudaSuccess) e = cudaEventRecord(plan->ev_copied[0], cp);
    const size_t comp = uhat_bytes_of(plan) / 3;
    const size_t elem = plan->dtype == BSPLINE_F64 ? 16 : 8;   // one complex mode
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
        if (plan->band) e = copy_band_h2d(plan, plan->host_uhat.ptr, u_hat_host, c, elem, cp);
        else e = cudaMemcpyAsync((char*)plan->host_uhat.ptr + c * comp, (const char*)u_hat_host + c * comp, comp,
                                 cudaMemcpyHostToDevice, cp);
        if (e == cudaSuccess) e = cudaEventRecord(plan->ev_copied[1 + c], cp);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, plan->ev_copied[0], 0);
    if (e != cudaSuccess) return set_cuda_error(e);
    for (int c = 0; c < 3; ++c) {
        if ((e = cudaStreamWaitEvent(st, plan->ev_copied[1 + c], 0)) != cudaSuccess) return set_cuda_error(e);
        if ((rc = launch_coeffs_range(plan, plan->host_uhat.ptr, plan->host_coef.ptr, c, c + 1))) return rc;
    }
    if (P) {
        const int flags = grad_host ? 0 : BSPLINE_INTERP_NO_GRAD;
        if ((rc = launch_interp_split(plan, plan->host_coef.ptr, (const double*)plan->host_x.ptr, P, plan->host_u.ptr,
                                      plan->host_grad.ptr, flags, aux, plan->ev_sorted)))
            return rc;
        e = cudaMemcpyAsync(u_host, plan->host_u.ptr, ob * 3 * P, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && grad_host)
            e = cudaMemcpyAsync(grad_host, plan->host_grad.ptr, ob * 9 * P, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return BSPLINE_OK;
}

int bspline_wait(bspline_plan_t plan) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    if (e == cudaSuccess && plan->aux_stream) e = cudaStreamSynchronize(plan->aux_stream);
    if (e == cudaSuccess && plan->copy_stream) e = cudaStreamSynchronize(plan->copy_stream);
    return set_cuda_error(e);
}

int bspline_run_host(bspline_plan_t plan, const void* u_hat_host, const double* x_host, int64_t P, void* u_host,
                     void* grad_host) {
    int rc = bspline_run_host_async(plan, u_hat_host, x_host, P, u_host, grad_host);
    if (rc != BSPLINE_OK) {
        if (valid_plan(plan)) bspline_wait(plan);       // let whatever was queued finish before reporting
        return rc;
    }
    return bspline_wait(plan);
}

int bspline_destroy(bspline_plan_t plan) {
    if (!plan) return BSPLINE_OK;
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    {
        DeviceGuard g(plan->device);
        cudaStreamSynchronize(plan->stream);
        free_plan(plan);
    }
    return BSPLINE_OK;
}

const char* bspline_status_string(int status) {
    switch (status) {
        case BSPLINE_OK: return "ok";
        case BSPLINE_ERR_INVALID_ARG: return "invalid argument";
        case BSPLINE_ERR_UNSUPPORTED_N: return "unsupported grid size N";
        case BSPLINE_ERR_UNSUPPORTED_ORDER: return "unsupported B-spline order";
        case BSPLINE_ERR_CUDA: return "CUDA runtime error";
        case BSPLINE_ERR_NONFINITE_INPUT: return "non-finite positions";
        case BSPLINE_ERR_TIMEOUT: return "device wait timed out";
        case BSPLINE_ERR_NOT_IMPLEMENTED: return "not implemented";
        case BSPLINE_ERR_OUT_OF_MEMORY: return "out of device memory";
        case BSPLINE_ERR_TOO_LARGE: return "size beyond the fixed scratch of bspline_interp_noalloc";
        case BSPLINE_ERR_BOUNDS: return "an index check of a BSPLINE_CHECKS build failed";
    }
    return "unknown status";
}

const char* bspline_version(void) { return "bspline-gb300 0.1.0"; }

int bspline_plan_set_timing(bspline_plan_t plan, int enable) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    clear_timing(plan);
    plan->timing = enable != 0;
    return set_cuda_error(e);
}

int bspline_stage_times(bspline_plan_t plan, double* ms, int64_t* launches) {
    if (!valid_plan(plan)) return BSPLINE_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    for (auto& t : plan->pending) {
        float dt = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&dt, t.start, t.stop);
        if (t.stage >= 0 && t.stage < BSPLINE_NSTAGES) {
            if (ms) ms[t.stage] += dt;
            if (launches) launches[t.stage] += 1;
        }
    }
    clear_timing(plan);
    return set_cuda_error(e);
}

}  // extern "C"

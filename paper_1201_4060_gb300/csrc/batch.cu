// Batches of independent fields replayed as one CUDA graph.
//
// The paper evaluates one field at a time; many small fields (different grid
// sizes and particle counts) leave most of the GPU idle between the short
// kernels of each.  A batch records the coefficient transform and the
// evaluation of every field into one graph: fields go round-robin over K
// concurrent streams (a plan's fields stay on one stream, since they share
// its workspace), and the graph is replayed with one launch.  K is chosen by
// timing the captured graph for K = 1, 2, 4, ... (bspline_batch_autotune).
#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "internal.h"

struct bspline_batch_s {
    int n = 0;
    int device = 0;
    std::vector<bspline_plan_t> plans;
    // arguments of the last capture
    std::vector<const void*> u_hat;
    std::vector<void*> coeffs;
    std::vector<const double*> x;
    std::vector<int64_t> P;
    std::vector<void*> out_u, out_grad;
    bool have_args = false;
    int streams = 0;                    // streams of the instantiated graph (0: none)
    cudaStream_t origin = nullptr;      // capture origin
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

using namespace bs;

void drop_graph(bspline_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->streams = 0;
}

int ensure_streams(bspline_batch_s* b, int k) {
    cudaError_t e = cudaSuccess;
    if (!b->origin) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    if (e == cudaSuccess && !b->fork) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    while (e == cudaSuccess && (int)b->side.size() < k) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (s) b->side.push_back(s);
        if (ev) b->join.push_back(ev);
    }
    return set_cuda_error(e);
}

// Record every field into a new graph on k streams.
int capture(bspline_batch_s* b, int k) {
    drop_graph(b);
    std::map<bspline_plan_t, int> lane;             // plan -> stream
    for (int i = 0; i < b->n; ++i) {
        if (lane.count(b->plans[i])) continue;
        const int next = (int)(lane.size() % (size_t)k);
        lane[b->plans[i]] = next;
    }
    k = std::min<int>(k, (int)lane.size());
    int rc = ensure_streams(b, k);
    if (rc) return rc;
    // workspaces are allocated now: no allocation may happen inside the capture
    for (int i = 0; i < b->n; ++i) {
        bspline_plan_t p = b->plans[i];
        if ((rc = p->work.grow(coeffs_workspace_bytes(p)))) return rc;
        if ((rc = p->pws.grow(interp_workspace_bytes(p, b->P[i])))) return rc;
    }
    std::vector<cudaStream_t> saved(b->n);
    std::vector<bool> timing(b->n);
    for (int i = 0; i < b->n; ++i) {
        saved[i] = b->plans[i]->stream;
        timing[i] = b->plans[i]->timing;
        b->plans[i]->timing = false;
    }
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->origin);
    for (int s = 0; s < k && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->side[s], b->fork, 0);
    rc = set_cuda_error(e);
    for (int i = 0; i < b->n && rc == BSPLINE_OK; ++i) {
        bspline_plan_t p = b->plans[i];
        p->stream = b->side[lane[p] % k];
        rc = bspline_coeffs(p, b->u_hat[i], b->coeffs[i]);
        if (rc == BSPLINE_OK)
            rc = bspline_interp(p, b->coeffs[i], b->x[i], b->P[i], b->out_u[i], b->out_grad[i],
                                b->out_grad[i] ? 0 : BSPLINE_INTERP_NO_GRAD);
    }
    for (int s = 0; s < k; ++s) {
        cudaEventRecord(b->join[s], b->side[s]);
        cudaStreamWaitEvent(b->origin, b->join[s], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->origin, &g);
    for (int i = 0; i < b->n; ++i) {
        b->plans[i]->stream = saved[i];
        b->plans[i]->timing = timing[i];
    }
    if (rc == BSPLINE_OK && e != cudaSuccess) rc = set_cuda_error(e);
    if (rc != BSPLINE_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc;
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        drop_graph(b);
        return set_cuda_error(e);
    }
    b->streams = k;
    return BSPLINE_OK;
}

// Device guard for the batch's device.
struct Guard {
    int prev = -1;
    bool ok = true;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess || (prev != dev && cudaSetDevice(dev) != cudaSuccess)) {
            ok = false;
            cudaGetLastError();
        }
    }
    ~Guard() {
        int cur;
        if (ok && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int bspline_batch_create(bspline_batch_t* out, int nfields, const bspline_plan_t* plans) {
    if (!out) return BSPLINE_ERR_INVALID_ARG;
    *out = nullptr;
    if (nfields <= 0 || !plans) return BSPLINE_ERR_INVALID_ARG;
    for (int i = 0; i < nfields; ++i)
        if (!plans[i] || plans[i]->N <= 0 || plans[i]->device != plans[0]->device) return BSPLINE_ERR_INVALID_ARG;
    bspline_batch_s* b = new (std::nothrow) bspline_batch_s;
    if (!b) return BSPLINE_ERR_OUT_OF_MEMORY;
    b->n = nfields;
    b->device = plans[0]->device;
    b->plans.assign(plans, plans + nfields);
    *out = b;
    return BSPLINE_OK;
}

int bspline_batch_capture(bspline_batch_t b, int streams, const void* const* u_hat, void* const* coeffs,
                          const double* const* x, const int64_t* P, void* const* out_u, void* const* out_grad) {
    if (!b || streams < 1 || !u_hat || !coeffs || !x || !P || !out_u) return BSPLINE_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i)
        if (P[i] < 0 || P[i] > 0x7fffffffLL || !u_hat[i] || !coeffs[i] || (P[i] > 0 && (!x[i] || !out_u[i])))
            return BSPLINE_ERR_INVALID_ARG;
    Guard g(b->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    b->u_hat.assign(u_hat, u_hat + b->n);
    b->coeffs.assign(coeffs, coeffs + b->n);
    b->x.assign(x, x + b->n);
    b->P.assign(P, P + b->n);
    b->out_u.assign(out_u, out_u + b->n);
    if (out_grad) b->out_grad.assign(out_grad, out_grad + b->n);
    else b->out_grad.assign(b->n, nullptr);
    b->have_args = true;
    return capture(b, streams);
}

int bspline_batch_launch(bspline_batch_t b, void* stream) {
    if (!b || !b->exec) return BSPLINE_ERR_INVALID_ARG;
    Guard g(b->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    return set_cuda_error(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

int bspline_batch_autotune(bspline_batch_t b, void* stream, int* best_streams, double* best_ms) {
    if (!b || !b->have_args) return BSPLINE_ERR_INVALID_ARG;
    Guard g(b->device);
    if (!g.ok) return BSPLINE_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int rc = set_cuda_error(e);
    int best_k = 1, prev = 0;
    float best = 0.f;
    for (int k = 1; k <= 16 && rc == BSPLINE_OK; k *= 2) {
        if ((rc = capture(b, k))) break;
        if (b->streams == prev) break;             // fewer distinct plans than streams: nothing new to try
        prev = b->streams;
        for (int w = 0; w < 2 && rc == BSPLINE_OK; ++w) rc = set_cuda_error(cudaGraphLaunch(b->exec, st));
        if (rc) break;
        e = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = cudaGraphLaunch(b->exec, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if ((rc = set_cuda_error(e))) break;
        if (k == 1 || ms < best) {
            best = ms;
            best_k = b->streams;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = capture(b, best_k))) return rc;
    if (best_streams) *best_streams = best_k;
    if (best_ms) *best_ms = best / 3.0;
    return BSPLINE_OK;
}

int bspline_batch_destroy(bspline_batch_t b) {
    if (!b) return BSPLINE_OK;
    Guard g(b->device);
    drop_graph(b);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
    return BSPLINE_OK;
}

}  // extern "C"

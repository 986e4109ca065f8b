// Persistent particle kernel of a batch of fields: one launch counts, scans,
// places and evaluates the particles of every field through a device work
// queue (no counterpart in the paper, which treats one field at a time).
//
// Tickets are taken in order from one counter.  The queue holds, in this
// order: every field's count tasks (a range of its particles each), one scan
// task per field, every field's placement tasks (the same ranges), then every
// field's gather items (a brick's coefficient tile and up to chunk_len of its
// particles, as in the single-field gather).  A scan waits until its field's
// count tasks have all signalled, a placement task until its field's scan
// has, a gather item until its field's placement tasks have.  Every wait is
// for tasks with smaller tickets, taken by CTAs that are already running and
// wait only for smaller tickets still, so the waits end; each is nonetheless
// bounded (about a second of polls): when one runs out it sets the batch's
// time-out word, its task is skipped, and every later wait that is not yet
// satisfied gives up at once, so the launch ends.  Completion is a release
// reduction by thread 0 after a CTA barrier; a wait is an acquire load by
// thread 0 followed by a CTA barrier.
#pragma once
#include "particles.cuh"

namespace bs {
namespace batch_impl {

using gather_impl::Rec;
using gather_impl::Ws;

// One field of a batch (device copy, written at capture).
struct FieldDesc {
    const float* coef;           // [3][N][N][N] FP32 coefficients
    const double* x;             // [P][3]
    float* out_u;                // [P][3]
    float* out_grad;             // [P][3][3] (the batch evaluates grad u for every field or for none)
    long long P;
    int N;
    double scale;                // N / L
    float dscale;                // N / L for the derivatives
    BrickGrid bg;
    Ws<float> w;                 // the field's sort workspace, carved from the batch's buffer
};

// Queue of one launch.  ctr (zeroed before every launch): [0] ticket counter,
// [1] time-out word, then per field the finished count tasks, the finished
// scan, and the finished placement tasks.  status (zeroed before every
// launch; laid out as a plan's status words): [0] non-finite positions of all
// fields, [1] a wait ran out, [2] index checks that failed (checks builds).
struct Queue {
    const FieldDesc* fields;
    const unsigned* task_pre;    // [F + 1] prefix over fields of the count (= placement) tasks
    const unsigned* item_pre;    // [F + 1] prefix over fields of the gather items (upper bounds)
    unsigned* ctr;
    unsigned long long* status;
    int F;
    unsigned part_per_task;      // particles of one count / placement task
    unsigned chunk_len;          // particles of one gather item (<= kChunk)
    int drop_first_signal;       // test hook: the first count task of field 0 does not signal
};

constexpr long long kQueueWaitLimit = 1LL << 22;

__device__ __forceinline__ unsigned q_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void q_signal(unsigned* p) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

// Thread 0: bounded wait for *flag >= target.  False if it ran out (the
// time-out words are then set) or if another wait of the launch already had.
__device__ __forceinline__ bool q_wait(const unsigned* flag, unsigned target, unsigned* err,
                                       unsigned long long* status) {
    long long it = 0;
    while (q_ld_acquire(flag) < target) {
        if (q_ld_acquire(err) != 0u) return false;
        if (++it > kQueueWaitLimit) {
            atomicExch(err, 1u);
            atomicOr(&status[kStatusParticleTimeout], 1ULL);
            return false;
        }
        __nanosleep(200);
    }
    return true;
}

// Largest f with pre[f] <= t (pre nondecreasing, pre[0] = 0 <= t < pre[F]).
__device__ __forceinline__ int q_field_of(const unsigned* pre, int F, unsigned t) {
    int lo = 0, hi = F;                                  // pre[lo] <= t < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned q_warp_inclusive(unsigned v, unsigned lane) {
#pragma unroll
    for (unsigned d = 1; d < 32; d <<= 1) {
        const unsigned a = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += a;
    }
    return v;
}

// Count task: locate particles [p0, p1) of a field and count them per brick
// (the single-field count pass, warp-aggregated increments).
template <int ORD>
__device__ __forceinline__ void q_count(const FieldDesc& f, long long p0, long long p1, unsigned long long* status) {
    const unsigned NB = f.bg.NB;
    const int lane = threadIdx.x & 31;
    for (long long pw = p0 + (threadIdx.x & ~31u); pw < p1; pw += blockDim.x) {
        const long long p = pw + lane;
        const bool valid = p < p1;
        unsigned k = 0;
        if (valid) {
            Rec<float> r;
            k = gather_impl::locate_particle<float>(f.x, p, f.N, f.scale, ORD, f.bg, &r);
            if (k == NB) atomicAdd(&status[kStatusNonfinite], 1ULL);
        }
        const unsigned active = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const unsigned peers = __match_any_sync(active, k);
            const unsigned leader = __ffs(peers) - 1;
            if ((unsigned)lane == leader) atomicAdd(&f.w.count[k], (unsigned)__popc(peers));
        }
    }
}

// Placement task: locate again and write each record to its brick's next slot; NaN outputs for
// non-finite positions.
template <int ORD, bool GRAD>
__device__ __forceinline__ void q_place(const FieldDesc& f, long long p0, long long p1,
                                        unsigned long long* status) {
    const unsigned NB = f.bg.NB;
    const int lane = threadIdx.x & 31;
    for (long long pw = p0 + (threadIdx.x & ~31u); pw < p1; pw += blockDim.x) {
        const long long p = pw + lane;
        Rec<float> r;
        unsigned k = NB;
        if (p < p1) k = gather_impl::locate_particle<float>(f.x, p, f.N, f.scale, ORD, f.bg, &r);
        if (p < p1 && k >= NB) {
#pragma unroll
            for (int i = 0; i < 3; ++i) f.out_u[3 * p + i] = NAN;
            if (GRAD) {
#pragma unroll
                for (int i = 0; i < 9; ++i) f.out_grad[9 * p + i] = NAN;
            }
        }
        const bool place = p < p1 && k < NB;
        const unsigned active = __ballot_sync(0xffffffffu, place);
        if (place) {
            const unsigned peers = __match_any_sync(active, k);
            const unsigned leader = __ffs(peers) - 1;
            unsigned base = 0;
            if ((unsigned)lane == leader) base = atomicAdd(&f.w.cursor[k], (unsigned)__popc(peers));
            base = __shfl_sync(peers, base, leader);
            const unsigned d = base + (unsigned)__popc(peers & ((1u << lane) - 1u));
            r.idx = (unsigned)p;
            r.pad[0] = r.pad[1] = r.pad[2] = 0u;
            if (BS_CHECK_OK(d < f.w.offset[k] + f.w.count[k], status + kStatusBounds)) f.w.s_rec[d] = r;
        }
    }
}

// Scan task: the field's brick offsets, cursors, item prefix and item -> brick
// map (every brick staged), by one CTA of any multiple of 32 threads.
__device__ __forceinline__ void q_scan(const FieldDesc& f, unsigned chunk_len) {
    __shared__ unsigned wd[32], wc[32];
    const Ws<float>& w = f.w;
    const unsigned NB = f.bg.NB;
    const unsigned t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    unsigned cd = 0, cc = 0;
    for (unsigned b0 = 0; b0 < NB; b0 += blockDim.x) {
        const unsigned i = b0 + t;
        const unsigned ci = i < NB ? w.count[i] : 0u;
        const unsigned nc = (ci + chunk_len - 1) / chunk_len;
        const unsigned vd = q_warp_inclusive(ci, lane), vc = q_warp_inclusive(nc, lane);
        if (lane == 31) {
            wd[warp] = vd;
            wc[warp] = vc;
        }
        __syncthreads();
        if (warp == 0) {
            const unsigned a = q_warp_inclusive(lane < nw ? wd[lane] : 0u, lane);
            const unsigned c = q_warp_inclusive(lane < nw ? wc[lane] : 0u, lane);
            wd[lane] = a;
            wc[lane] = c;
        }
        __syncthreads();
        const unsigned exd = cd + (warp ? wd[warp - 1] : 0u) + vd - ci;
        const unsigned exc = cc + (warp ? wc[warp - 1] : 0u) + vc - nc;
        if (i < NB) {
            w.offset[i] = exd;
            w.cursor[i] = exd;
            w.chunk[i] = exc;
            for (unsigned k = 0; k < nc; ++k) w.item[exc + k] = i;
        }
        cd += wd[nw - 1];
        cc += wc[nw - 1];
        __syncthreads();                                 // the totals are read before the next tile
    }
    if (t == 0) {
        w.offset[NB] = cd;
        w.cursor[NB] = cd;
        w.offset[NB + 1] = cd + w.count[NB];
        w.offset[NB + 2] = cd;
        w.chunk[NB] = cc;
    }
}

template <int ORD, int BYO, bool GRAD>
__global__ void __launch_bounds__(gather_impl::kGatherThreads, 2) batch_queue_kernel(Queue q) {
    __shared__ int s_task[4];                            // phase (-1: skip, 4: done), field, index, spare
    const int F = q.F;
    const unsigned Tc = q.task_pre[F];                   // count tasks (and placement tasks)
    const unsigned Ts = Tc + (unsigned)F;                // + scans
    const unsigned Tp = Ts + Tc;                         // + placements
    const unsigned total = Tp + q.item_pre[F];           // + gather items
    unsigned* err = &q.ctr[1];
    unsigned* done_count = q.ctr + 2;
    unsigned* done_scan = done_count + F;
    unsigned* done_place = done_scan + F;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned t = atomicAdd(&q.ctr[0], 1u);
            int phase = 4, fi = 0;
            unsigned j = 0;
            if (t < Tc) {
                phase = 0;
                fi = q_field_of(q.task_pre, F, t);
                j = t - q.task_pre[fi];
            } else if (t < Ts) {
                phase = 1;
                fi = (int)(t - Tc);
                if (!q_wait(&done_count[fi], q.task_pre[fi + 1] - q.task_pre[fi], err, q.status)) phase = -1;
            } else if (t < Tp) {
                phase = 2;
                fi = q_field_of(q.task_pre, F, t - Ts);
                j = t - Ts - q.task_pre[fi];
                if (!q_wait(&done_scan[fi], 1u, err, q.status)) phase = -1;
            } else if (t < total) {
                phase = 3;
                fi = q_field_of(q.item_pre, F, t - Tp);
                j = t - Tp - q.item_pre[fi];
                if (!q_wait(&done_place[fi], q.task_pre[fi + 1] - q.task_pre[fi], err, q.status)) phase = -1;
            }
            s_task[0] = phase;
            s_task[1] = fi;
            s_task[2] = (int)j;
        }
        __syncthreads();
        const int phase = s_task[0], fi = s_task[1];
        const unsigned j = (unsigned)s_task[2];
        __syncthreads();                                 // s_task is rewritten by the next claim
        if (phase == 4) return;
        if (phase < 0) continue;
        const FieldDesc& f = q.fields[fi];
        if (phase == 0 || phase == 2) {
            const long long p0 = (long long)j * q.part_per_task;
            const long long p1 = min(f.P, p0 + (long long)q.part_per_task);
            if (phase == 0) q_count<ORD>(f, p0, p1, q.status);
            else q_place<ORD, GRAD>(f, p0, p1, q.status);
            __syncthreads();
            if (threadIdx.x == 0 && !(phase == 0 && q.drop_first_signal && fi == 0 && j == 0))
                q_signal(phase == 0 ? &done_count[fi] : &done_place[fi]);
        } else if (phase == 1) {
            q_scan(f, q.chunk_len);
            __syncthreads();
            if (threadIdx.x == 0) q_signal(&done_scan[fi]);
        } else {
            if (j < f.w.chunk[f.bg.NB])
                gather_impl::gather_f32_item<ORD, float, float, GRAD, BYO>(
                    j, q.chunk_len, f.coef, f.N, f.bg, f.w, f.out_u, GRAD ? f.out_grad : nullptr, f.dscale,
                    nullptr, 0, q.status);
            __syncthreads();                             // the tile and the order are reused by the next item
        }
    }
}

// Launch of one configuration (order, brick y extent, grad) on `stream`:
// persistent grid of the resident CTAs of every SM.
template <int ORD, int BYO, bool GRAD>
int launch_batch_queue(const Queue& q, int sms, cudaStream_t stream) {
    auto k = batch_queue_kernel<ORD, BYO, GRAD>;
    const size_t sm = gather_impl::tile_bytes<ORD, float, BYO>() + 128;
    int rc = gather_impl::set_smem(k, sm);
    if (rc) return rc;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, gather_impl::kGatherThreads, sm);
    if (e != cudaSuccess) return set_cuda_error(e);
    k<<<(unsigned)(std::max(per_sm, 1) * sms), gather_impl::kGatherThreads, sm, stream>>>(q);
    return set_cuda_error(cudaGetLastError());
}

// The brick y extents a batch can take (orders 7 and 8: 8 and 16 only).
inline bool queue_brick_y_ok(int order, int by) { return by == 8 || by == 16 || (by == 12 && order <= 6); }

// Launch for one order (u and grad u); one translation unit per order.
template <int ORD> int dispatch_brick_y(int by, const Queue& q, int sms, cudaStream_t stream) {
    switch (by) {
        case 8: return launch_batch_queue<ORD, 8, true>(q, sms, stream);
        case 16: return launch_batch_queue<ORD, 16, true>(q, sms, stream);
        case 12:
            if constexpr (ORD <= 6) return launch_batch_queue<ORD, 12, true>(q, sms, stream);
            break;
    }
    return BSPLINE_ERR_INVALID_ARG;
}
int launch_batch_queue_o2(int by, const Queue& q, int sms, cudaStream_t stream);
int launch_batch_queue_o3(int by, const Queue& q, int sms, cudaStream_t stream);
int launch_batch_queue_o4(int by, const Queue& q, int sms, cudaStream_t stream);
int launch_batch_queue_o5(int by, const Queue& q, int sms, cudaStream_t stream);
int launch_batch_queue_o6(int by, const Queue& q, int sms, cudaStream_t stream);
int launch_batch_queue_o7(int by, const Queue& q, int sms, cudaStream_t stream);
int launch_batch_queue_o8(int by, const Queue& q, int sms, cudaStream_t stream);

}  // namespace batch_impl
}  // namespace bs

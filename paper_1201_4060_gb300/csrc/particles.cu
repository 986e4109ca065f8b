// Particle side of the path: locate, bin/sort, and evaluate u and grad u.
//
// Locate (Eq. alg-int-6): s = x N / L in FP64; the stencil nodes are
// floor(s - n/2) + j, j = 1..n; the local variable is t = (s - n/2) - floor(s - n/2).
// The first node (the "anchor") picks a brick of 16^3 (FP64: 8^3) cells; particles are
// counting-sorted by brick so that one CTA stages the brick's coefficients
// (plus the n-1 halo) in shared memory once and evaluates all of its particles.
//
// Weights: per axis, the n node weights B(t + n/2 - j) and their derivatives
// come from the Cox-de Boor recurrence of the cardinal B-spline
// (M_k(x) = (x M_{k-1}(x) + (k - x) M_{k-1}(x - 1)) / (k - 1)), in registers.
// They equal the columns of M x_bar and M^(1) x_bar of Section 4.
//
// Contraction (Table 1, reordered to contract the contiguous z axis first):
// per component, Z0 = sum_z w_z a, Z1 = sum_z w'_z a (2 n^3), then
// Y00 = sum_y w_y Z0, Y10 = sum_y w'_y Z0, Y01 = sum_y w_y Z1 (3 n^2), then
// u = sum_x w_x Y00, du/dx = sum_x w'_x Y00, du/dy = sum_x w_x Y10,
// du/dz = sum_x w_x Y01 (4 n), derivatives scaled by N / L.
#include "adjoint.cuh"

namespace bs {

#define BS_ORDERS(M, CT, AT, TR) M(2, CT, AT, TR) M(3, CT, AT, TR) M(4, CT, AT, TR) M(5, CT, AT, TR) \
    M(6, CT, AT, TR) M(7, CT, AT, TR) M(8, CT, AT, TR)
BS_ORDERS(BS_GATHER_EXTERN, double, double, double)
BS_ORDERS(BS_GATHER_EXTERN, float, float, float)
BS_ORDERS(BS_GATHER_EXTERN, __nv_bfloat16, float, float)
#define BS_ADJ_ORDERS(M, CT, TR) M(2, CT, TR) M(3, CT, TR) M(4, CT, TR) M(5, CT, TR) M(6, CT, TR) M(7, CT, TR) \
    M(8, CT, TR)
BS_ADJ_ORDERS(BS_ADJOINT_EXTERN, double, double)
BS_ADJ_ORDERS(BS_ADJOINT_EXTERN, float, float)
BS_ADJ_ORDERS(BS_ADJOINT_EXTERN, __nv_bfloat16, float)

namespace gather_impl {

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

int encode_coef_tmap(CUtensorMap* map, const void* coef, int N, int box_z, int box_y, int box_x, int elem_bytes) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return BSPLINE_ERR_CUDA;
    const cuuint64_t n = (cuuint64_t)N, eb = (cuuint64_t)elem_bytes;
    const cuuint64_t dims[4] = {n, n, n, 3};                               // z, y, x, component
    const cuuint64_t strides[3] = {n * eb, n * n * eb, n * n * n * eb};  // bytes, dims 1..3
    const cuuint32_t box[4] = {(cuuint32_t)box_z, (cuuint32_t)box_y, (cuuint32_t)box_x, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType t = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUresult r = fn(map, t, 4, const_cast<void*>(coef), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? BSPLINE_OK : BSPLINE_ERR_CUDA;
}

}  // namespace gather_impl

namespace {
using namespace gather_impl;

// ------------------------------------------------------------------ bin
// Below this many bricks, particles of one warp often share a brick: aggregate their counter updates.
constexpr unsigned kAggregateBricks = 4096;

// Warp-aggregated increment of counter[key] for the lanes of `active`: one
// atomic per distinct key in the warp (few bricks, many particles: small
// grids); returns this lane's slot (old value + its rank among equal keys).
__device__ __forceinline__ unsigned warp_increment(unsigned* counter, unsigned key, unsigned active, bool need_old) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned peers = __match_any_sync(active, key);
    const unsigned leader = __ffs(peers) - 1;
    unsigned base = 0;
    if (lane == leader) base = need_old ? atomicAdd(&counter[key], (unsigned)__popc(peers))
                                        : (atomicAdd(&counter[key], (unsigned)__popc(peers)), 0u);
    base = __shfl_sync(peers, base, leader);
    return base + (unsigned)__popc(peers & ((1u << lane) - 1u));
}

// Counting sort, pass 1: particles per brick (slot NB: invalid positions, also
// counted in the status word).  The grid-stride loop runs warp-uniformly so that
// lanes can aggregate their increments (aggregate = few bricks).  SORTED: the
// caller passed the positions grouped by brick, so position p is also the
// particle's sorted slot: its record is written there (coalesced, its own
// index as the original one), each key is checked against its predecessor's
// (the lane below, or located again at a warp's first lane) and *w.unsorted is
// set if the order is broken anywhere, in which case the placement pass
// rewrites every record; invalid positions get their NaN outputs here.
template <typename TR, bool SORTED, typename OT>
__global__ void bin_kernel(const double* __restrict__ x, long long P, int N, double scale, int order,
                           BrickGrid g, Ws<TR> w, unsigned long long* __restrict__ status, int aggregate,
                           OT* __restrict__ out_u, OT* __restrict__ out_grad) {
    const unsigned NB = g.NB;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long lane = threadIdx.x & 31;
    for (long long pw = (long long)blockIdx.x * blockDim.x + threadIdx.x - lane; pw < P; pw += stride) {
        const long long p = pw + lane;
        const bool valid = p < P;
        unsigned k = 0;
        if (valid) {
            Rec<TR> r;
            k = locate_particle<TR>(x, p, N, scale, order, g, &r);
            if (k == NB) atomicAdd(status, 1ULL);
            if (SORTED && k < NB) {
                r.idx = (unsigned)p;
                if constexpr (sizeof(TR) == 4) r.pad[0] = r.pad[1] = r.pad[2] = 0u;
                w.s_rec[p] = r;
            }
        }
        if constexpr (SORTED) {
            unsigned prev = __shfl_up_sync(0xffffffffu, k, 1);
            if (lane == 0 && valid && p > 0) {
                Rec<TR> r;
                prev = locate_particle<TR>(x, p - 1, N, scale, order, g, &r);
            }
            const bool broken = valid && p > 0 && prev > k;
            if (__any_sync(0xffffffffu, broken) && lane == 0) atomicOr(w.unsorted, 1u);
            if (valid && k == NB) {
                const OT nan = (OT)NAN;
                if (out_u) {
#pragma unroll
                    for (int i = 0; i < 3; ++i) out_u[3 * p + i] = nan;
                }
                if (out_grad) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) out_grad[9 * p + i] = nan;
                }
            }
        }
        if (aggregate) {
            const unsigned active = __ballot_sync(0xffffffffu, valid);
            if (valid) warp_increment(w.count, k, active, false);
        } else if (valid) {
            atomicAdd(&w.count[k], 1u);
        }
    }
}

// ------------------------------------------------------------------ scan (single CTA)
// Places the bricks' segments in the sorted order and counts the staged
// gather's work items.  Bricks holding at least `below` particles ("dense":
// every brick when below = 0) come first, in brick order; the bricks below
// it ("sparse", evaluated by the direct gather) follow, in brick order, so
// the direct gather runs flat over one contiguous range; the invalid bin NB
// comes last.  Writes offset[b] (and its copy cursor[b] for the placement
// pass), offset[NB] = the end of the valid particles, offset[NB + 1] = the
// end of all, offset[NB + 2] = the start of the sparse range; chunk[] (dense
// bricks only) the exclusive prefix sum of the work items, ceil(count /
// kChunk), chunk[NB] their total, and item[] each item's brick.
__device__ __forceinline__ unsigned warp_inclusive(unsigned v, unsigned lane) {
#pragma unroll
    for (unsigned d = 1; d < 32; d <<= 1) {
        const unsigned a = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += a;
    }
    return v;
}

// SPLIT = false (below = 0: every brick dense) skips the sparse bookkeeping.
template <bool SPLIT>
__global__ void __launch_bounds__(1024) scan_kernel(const unsigned* __restrict__ count, unsigned* __restrict__ offset,
                                                    unsigned* __restrict__ cursor, unsigned* __restrict__ chunk,
                                                    unsigned* __restrict__ item, unsigned NB, unsigned below) {
    __shared__ unsigned wd[32], wsp[32], wc[32], s_total;
    const unsigned t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // total of the dense bricks (the start of the sparse range)
    unsigned D = 0;
    if constexpr (SPLIT) {
        unsigned dsum = 0;
        for (unsigned i = t; i < NB; i += 1024) {
            const unsigned ci = count[i];
            if (ci >= below) dsum += ci;
        }
        dsum = __reduce_add_sync(0xffffffffu, dsum);
        if (lane == 0) wd[warp] = dsum;
        __syncthreads();
        if (warp == 0) {
            const unsigned v = __reduce_add_sync(0xffffffffu, wd[lane]);
            if (lane == 0) s_total = v;
        }
        __syncthreads();
        D = s_total;
    }
    unsigned cd = 0, cs = 0, cc = 0;                      // carries: dense, sparse, items
    // tiles of 1024 consecutive bricks, one per thread: warp scans, then a scan of the 32 warp totals
    for (unsigned b0 = 0; b0 < NB; b0 += 1024) {
        const unsigned i = b0 + t;
        const unsigned ci = i < NB ? count[i] : 0u;
        const bool dense = !SPLIT || ci >= below;
        const unsigned vd0 = dense ? ci : 0u, vs0 = dense ? 0u : ci;
        const unsigned nc = dense ? (ci + kChunk - 1) / kChunk : 0u;
        const unsigned vd = warp_inclusive(vd0, lane), vc = warp_inclusive(nc, lane);
        const unsigned vs = SPLIT ? warp_inclusive(vs0, lane) : 0u;
        if (lane == 31) {
            wd[warp] = vd;
            wsp[warp] = vs;
            wc[warp] = vc;
        }
        __syncthreads();
        if (warp == 0) {
            wd[lane] = warp_inclusive(wd[lane], lane);
            if (SPLIT) wsp[lane] = warp_inclusive(wsp[lane], lane);
            wc[lane] = warp_inclusive(wc[lane], lane);
        }
        __syncthreads();
        const unsigned exd = cd + (warp ? wd[warp - 1] : 0u) + vd - vd0;          // exclusive
        const unsigned exs = cs + (warp ? wsp[warp - 1] : 0u) + vs - vs0;
        const unsigned exc = cc + (warp ? wc[warp - 1] : 0u) + vc - nc;
        if (i < NB) {
            const unsigned o = dense ? exd : D + exs;
            offset[i] = o;
            cursor[i] = o;
            chunk[i] = exc;
            for (unsigned k = 0; k < nc; ++k) item[exc + k] = i;
        }
        cd += wd[31];
        cs += wsp[31];
        cc += wc[31];
        __syncthreads();                                  // the totals are read before the next tile
    }
    if (t == 0) {
        offset[NB] = cd + cs;                             // the invalid bin
        cursor[NB] = cd + cs;
        offset[NB + 1] = cd + cs + count[NB];
        offset[NB + 2] = SPLIT ? D : cd;
        chunk[NB] = cc;
    }
}

// ------------------------------------------------------------------ place
// Counting sort, pass 2: locate again (cheaper than storing and re-reading the
// records) and write each record and its original index to the next free slot
// of its brick.  Invalid positions get NaN outputs.  SORTED: nothing to do
// unless the count pass found the order broken.  PERM (bspline_sort_order):
// every particle, invalid ones included (bin NB, last), gets a slot, and only
// its original index is written there, to perm.  cot (the adjoint of FP32
// types): each placed particle's cotangents g_u (or zeros) and g_grad (or
// zeros) also go to its slot, 16 floats (64 bytes: two whole sectors) a slot,
// so that the adjoint kernels read them in sorted order; a warp reads its 32
// particles' cotangents as whole lines into 12 * 32 floats of dynamic shared
// memory (the launch gives 12 * 32 * 4 bytes per warp).
template <typename TR, typename OT, bool SORTED = false, bool PERM = false>
__global__ void scatter_kernel(const double* __restrict__ x, long long P, int N, double scale, int order,
                               BrickGrid g, Ws<TR> w, OT* __restrict__ out_u, OT* __restrict__ out_grad,
                               int aggregate, unsigned long long* __restrict__ status, int* __restrict__ perm = nullptr,
                               const float* __restrict__ cu = nullptr, const float* __restrict__ cg = nullptr,
                               float4* __restrict__ cot = nullptr) {
    const unsigned NB = g.NB;
    if constexpr (SORTED) {
        if (*w.unsorted == 0u) return;
    }
    if constexpr (PERM) {
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
            Rec<TR> r;
            const unsigned k = locate_particle<TR>(x, p, N, scale, order, g, &r);
            const unsigned d = atomicAdd(&w.cursor[k], 1u);
            if (BS_CHECK_OK(d < (unsigned)P, status + kStatusBounds)) perm[d] = (int)p;
        }
        return;
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long lane = threadIdx.x & 31;
    extern __shared__ float s_cot_stage[];
    float* sw = s_cot_stage + (threadIdx.x >> 5) * (12 * 32);
    for (long long pw = (long long)blockIdx.x * blockDim.x + threadIdx.x - lane; pw < P; pw += stride) {
        const long long p = pw + lane;
        Rec<TR> r;
        unsigned k = NB;
        if (p < P) k = locate_particle<TR>(x, p, N, scale, order, g, &r);
        if (p < P && k >= NB) {
            const OT nan = (OT)NAN;
            if (out_u) {
#pragma unroll
                for (int i = 0; i < 3; ++i) out_u[3 * p + i] = nan;
            }
            if (out_grad) {
#pragma unroll
                for (int i = 0; i < 9; ++i) out_grad[9 * p + i] = nan;
            }
        }
        const bool place = p < P && k < NB;
        if (cot) {                                      // the warp's cotangents, coalesced
            const int nq = (int)min(32LL, P - pw);
            __syncwarp();                               // the previous iteration's reads are done
            for (int i = (int)lane; i < 3 * nq; i += 32) sw[i] = cu ? cu[3 * pw + i] : 0.f;
            for (int i = (int)lane; i < 9 * nq; i += 32) sw[96 + i] = cg ? cg[9 * pw + i] : 0.f;
            __syncwarp();
        }
        unsigned d = 0;
        if (aggregate) {
            const unsigned active = __ballot_sync(0xffffffffu, place);
            if (place) d = warp_increment(w.cursor, k, active, true);
        } else if (place) {
            d = atomicAdd(&w.cursor[k], 1u);
        }
        if (place && BS_CHECK_OK(d < w.offset[k] + w.count[k], status + kStatusBounds)) {
            r.idx = (unsigned)p;
            if constexpr (sizeof(TR) == 4) r.pad[0] = r.pad[1] = r.pad[2] = 0u;
            w.s_rec[d] = r;                             // one whole 32-byte sector
            if (cot) {
                float v[12];
#pragma unroll
                for (int i = 0; i < 3; ++i) v[i] = sw[3 * lane + i];
#pragma unroll
                for (int i = 0; i < 9; ++i) v[3 + i] = sw[96 + 9 * lane + i];
                float4* dst = cot + 4 * (size_t)d;
                dst[0] = make_float4(v[0], v[1], v[2], v[3]);
                dst[1] = make_float4(v[4], v[5], v[6], v[7]);
                dst[2] = make_float4(v[8], v[9], v[10], v[11]);
                dst[3] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
}

template <typename CT, typename AT, typename TR>
int dispatch_order(bspline_plan_s* p, const void* coeffs, Ws<TR> w, BrickGrid g, void* out_u,
                   void* out_grad, bool grad) {
    switch (p->order) {
        case 2: return run_gather<2, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad);
        case 3: return run_gather<3, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad);
        case 4: return run_gather<4, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad);
        case 5: return run_gather<5, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad);
        case 6: return run_gather<6, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad);
        case 7: return run_gather<7, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad);
        case 8: return run_gather<8, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad);
    }
    return BSPLINE_ERR_UNSUPPORTED_ORDER;
}

template <typename CT, typename AT, typename TR>
int dispatch_direct(bspline_plan_s* p, const void* coeffs, Ws<TR> w, BrickGrid g, void* out_u, void* out_grad,
                    bool grad, unsigned below) {
    switch (p->order) {
        case 2: return run_gather_direct<2, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad, below);
        case 3: return run_gather_direct<3, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad, below);
        case 4: return run_gather_direct<4, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad, below);
        case 5: return run_gather_direct<5, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad, below);
        case 6: return run_gather_direct<6, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad, below);
        case 7: return run_gather_direct<7, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad, below);
        case 8: return run_gather_direct<8, CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad, below);
    }
    return BSPLINE_ERR_UNSUPPORTED_ORDER;
}

inline unsigned grid_for(long long P, int threads) {
    long long g = (P + threads - 1) / threads;
    if (g > (1LL << 30)) g = 1LL << 30;
    return (unsigned)(g < 1 ? 1 : g);
}

// The sort (bin, scan, scatter) runs on sort_stream when one is given (it
// needs only the positions) and the gather on the plan's stream after `sorted`.
template <typename CT, typename AT, typename TR>
int run_interp(bspline_plan_s* p, const void* coeffs, const double* x, int64_t P, void* out_u, void* out_grad,
               int flags, cudaStream_t sort_stream, cudaEvent_t sorted) {
    const BrickGrid g = brick_grid(p->N, p->dtype, p->order);
    const unsigned NB = g.NB;
    Ws<TR> w;
    const size_t need = carve<TR>(&w, nullptr, NB, P);
    int rc = p->pws.grow(need);
    if (rc) return rc;
    carve<TR>(&w, p->pws.ptr, NB, P);
    const cudaStream_t main_stream = p->stream;
    cudaStream_t st = sort_stream ? sort_stream : main_stream;
    p->stream = st;                                     // stage timers follow the sort's stream
    struct Restore {
        bspline_plan_s* p;
        cudaStream_t s;
        ~Restore() { p->stream = s; }
    } restore{p, main_stream};
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.count, 0, sizeof(unsigned) * (NB + 2), st)) != cudaSuccess) return set_cuda_error(e);
    if ((e = cudaMemsetAsync(p->d_status, 0, sizeof(unsigned long long) * kStatusParticleWords, st)) != cudaSuccess)
        return set_cuda_error(e);                       // non-finite count, tile-wait flag, checks
    const bool grad = !(flags & BSPLINE_INTERP_NO_GRAD);
    const bool presorted = (flags & BSPLINE_INTERP_SORTED) != 0;
    const double scale = (double)p->N / p->L;
    AT* ou = (AT*)out_u;
    AT* og = grad ? (AT*)out_grad : nullptr;
    // Beside the transform (sort_stream given), the locate passes run as a small grid-stride grid, two
    // 256-thread CTAs per SM: they then share the SMs with the transform's CTAs instead of taking them in
    // turn, and use the HBM bandwidth the transform leaves (512^3, 2^24 particles: 5.33 -> 5.04 ms per
    // step; one CTA per SM or more than three were slower).  Alone, the full grid is faster.
    unsigned sort_grid = grid_for(P, 256);
    if (sort_stream && 2LL * p->sms < (long long)sort_grid) sort_grid = (unsigned)(2 * p->sms);
    // bricks with fewer particles than this go to the direct gather (FP32 accumulation only)
    unsigned below = p->direct_below;
    if (below == BSPLINE_GATHER_SPLIT_AUTO) below = P < 12LL * NB ? 32u : 0u;
    if (sizeof(AT) == 8 || presorted) below = 0u;       // sorted input: bricks stay in input order
    const int agg = NB < kAggregateBricks || presorted;  // sorted input: a warp's particles share bricks
    {
        StageTimer tm(p, BSPLINE_STAGE_BIN);
        if (presorted) bin_kernel<TR, true, AT><<<sort_grid, 256, 0, st>>>(x, P, p->N, scale, p->order, g, w, p->d_status, agg, ou, og);
        else bin_kernel<TR, false, AT><<<sort_grid, 256, 0, st>>>(x, P, p->N, scale, p->order, g, w, p->d_status, agg, ou, og);
    }
    {
        StageTimer tm(p, BSPLINE_STAGE_SCAN);
        if (below > 0) scan_kernel<true><<<1, 1024, 0, st>>>(w.count, w.offset, w.cursor, w.chunk, w.item, NB, below);
        else scan_kernel<false><<<1, 1024, 0, st>>>(w.count, w.offset, w.cursor, w.chunk, w.item, NB, 0u);
    }
    {
        StageTimer tm(p, BSPLINE_STAGE_SCATTER);
        if (presorted)
            scatter_kernel<TR, AT, true><<<sort_grid, 256, 0, st>>>(x, P, p->N, scale, p->order, g, w, ou, og, agg,
                                                                    p->d_status);
        else
            scatter_kernel<TR, AT><<<sort_grid, 256, 0, st>>>(x, P, p->N, scale, p->order, g, w, ou, og, agg, p->d_status);
    }
    if (sort_stream) {
        if ((e = cudaEventRecord(sorted, sort_stream)) != cudaSuccess) return set_cuda_error(e);
        if ((e = cudaStreamWaitEvent(main_stream, sorted, 0)) != cudaSuccess) return set_cuda_error(e);
    }
    p->stream = main_stream;
    {
        StageTimer tm(p, BSPLINE_STAGE_GATHER);
        rc = dispatch_order<CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad);
    }
    if (rc) return rc;
    if (below > 0) {
        StageTimer tm(p, BSPLINE_STAGE_GATHER_DIRECT);
        rc = dispatch_direct<CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad, below);
    }
    if (rc) return rc;
    return set_cuda_error(cudaGetLastError());
}

// Same launch sequence as run_interp, with the workspace and the status word
// supplied by the caller instead of the plan.
template <typename CT, typename AT, typename TR>
int run_interp_ws(bspline_plan_s* p, void* ws, unsigned long long* status, const void* coeffs, const double* x,
                  int64_t P, void* out_u, void* out_grad, int flags) {
    const BrickGrid g = brick_grid(p->N, p->dtype, p->order);
    const unsigned NB = g.NB;
    Ws<TR> w;
    carve<TR>(&w, ws, NB, P);
    cudaStream_t st = p->stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.count, 0, sizeof(unsigned) * (NB + 2), st)) != cudaSuccess) return set_cuda_error(e);
    if ((e = cudaMemsetAsync(status, 0, sizeof(unsigned long long) * kStatusParticleWords, st)) != cudaSuccess)
        return set_cuda_error(e);                       // non-finite count, tile-wait flag, checks
    const bool grad = !(flags & BSPLINE_INTERP_NO_GRAD);
    bin_kernel<TR, false, AT><<<grid_for(P, 256), 256, 0, st>>>(x, P, p->N, (double)p->N / p->L, p->order, g, w, status,
                                                               NB < kAggregateBricks, (AT*)nullptr, (AT*)nullptr);
    scan_kernel<false><<<1, 1024, 0, st>>>(w.count, w.offset, w.cursor, w.chunk, w.item, NB, 0u);
    scatter_kernel<TR, AT><<<grid_for(P, 256), 256, 0, st>>>(x, P, p->N, (double)p->N / p->L, p->order, g, w, (AT*)out_u, grad ? (AT*)out_grad : nullptr,
                                                             NB < kAggregateBricks, status);
    int rc = dispatch_order<CT, AT, TR>(p, coeffs, w, g, out_u, out_grad, grad);
    if (rc) return rc;
    return set_cuda_error(cudaGetLastError());
}

template <typename CT, typename TR>
int adjoint_order(bspline_plan_s* p, const void* coeffs, Ws<TR> w, BrickGrid g, long long items,
                  const void* g_u, const void* g_grad, void* g_coef, double* g_x, const float4* cot) {
    using adjoint_impl::run_adjoint;
    switch (p->order) {
        case 2: return run_adjoint<2, CT, TR>(p, coeffs, w, g, items, g_u, g_grad, g_coef, g_x, cot);
        case 3: return run_adjoint<3, CT, TR>(p, coeffs, w, g, items, g_u, g_grad, g_coef, g_x, cot);
        case 4: return run_adjoint<4, CT, TR>(p, coeffs, w, g, items, g_u, g_grad, g_coef, g_x, cot);
        case 5: return run_adjoint<5, CT, TR>(p, coeffs, w, g, items, g_u, g_grad, g_coef, g_x, cot);
        case 6: return run_adjoint<6, CT, TR>(p, coeffs, w, g, items, g_u, g_grad, g_coef, g_x, cot);
        case 7: return run_adjoint<7, CT, TR>(p, coeffs, w, g, items, g_u, g_grad, g_coef, g_x, cot);
        case 8: return run_adjoint<8, CT, TR>(p, coeffs, w, g, items, g_u, g_grad, g_coef, g_x, cot);
    }
    return BSPLINE_ERR_UNSUPPORTED_ORDER;
}

// Adjoint of the particle side: the same bin / scan / scatter as run_interp,
// then the spread into g_coef and the position gradient g_x (either may be
// skipped).  Non-finite positions contribute nothing and get NaN in g_x.
template <typename CT, typename TR>
int run_adjoint_particles(bspline_plan_s* p, const void* coeffs, const double* x, int64_t P, const void* g_u,
                          const void* g_grad, void* g_coef, double* g_x) {
    const BrickGrid g = brick_grid(p->N, p->dtype, p->order);
    const unsigned NB = g.NB;
    Ws<TR> w;
    const size_t need = carve<TR>(&w, nullptr, NB, P);
    int rc = p->pws.grow(need);
    if (rc) return rc;
    carve<TR>(&w, p->pws.ptr, NB, P);
    // FP32 types: the placement pass also copies each particle's cotangents to its sorted slot, which the
    // spread and the position gradients then read in order instead of gathering them from random indices
    float4* cot = nullptr;
    if (sizeof(TR) == 4 && (g_u || g_grad) && (g_coef || g_x)) {
        if ((rc = p->cot.grow(sizeof(float4) * 4 * (size_t)P))) return rc;
        cot = reinterpret_cast<float4*>(p->cot.ptr);
    }
    cudaStream_t st = p->stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.count, 0, sizeof(unsigned) * (NB + 2), st)) != cudaSuccess) return set_cuda_error(e);
    if ((e = cudaMemsetAsync(p->d_status, 0, sizeof(unsigned long long) * kStatusParticleWords, st)) != cudaSuccess)
        return set_cuda_error(e);                       // non-finite count, tile-wait flag, checks
    {
        StageTimer tm(p, BSPLINE_STAGE_BIN);
        bin_kernel<TR, false, double><<<grid_for(P, 256), 256, 0, st>>>(x, P, p->N, (double)p->N / p->L, p->order, g, w,
                                                                        p->d_status, NB < kAggregateBricks,
                                                                        (double*)nullptr, (double*)nullptr);
    }
    {
        StageTimer tm(p, BSPLINE_STAGE_SCAN);
        scan_kernel<false><<<1, 1024, 0, st>>>(w.count, w.offset, w.cursor, w.chunk, w.item, NB, 0u);
    }
    {
        StageTimer tm(p, BSPLINE_STAGE_SCATTER);
        const size_t cot_smem = cot ? sizeof(float) * 12 * 256 : 0;   // 12 * 32 floats per warp
        scatter_kernel<TR, double><<<grid_for(P, 256), 256, cot_smem, st>>>(x, P, p->N, (double)p->N / p->L, p->order, g, w, g_x, nullptr, NB < kAggregateBricks,
                                                                     p->d_status, nullptr, (const float*)g_u,
                                                                     (const float*)g_grad, cot);
    }
    const long long items = (long long)NB + (P + kChunk - 1) / kChunk;
    if (g_coef && p->deterministic && sizeof(TR) == 4) {
        // the fixed-point accumulator of the deterministic spread and its bound word
        if ((rc = p->det.grow(sizeof(long long) * 3 * (size_t)p->N * p->N * p->N + 16))) return rc;
    }
    if (g_coef) {
        StageTimer tm(p, BSPLINE_STAGE_SPREAD);
        rc = adjoint_order<CT, TR>(p, coeffs, w, g, items, g_u, g_grad, g_coef, nullptr, cot);
        if (rc) return rc;
    }
    if (g_x) {
        StageTimer tm(p, BSPLINE_STAGE_GRAD_X);
        rc = adjoint_order<CT, TR>(p, coeffs, w, g, items, g_u, g_grad, nullptr, g_x, cot);
        if (rc) return rc;
    }
    return set_cuda_error(cudaGetLastError());
}

// Brick order of the particles (bspline_sort_order): count, scan, then each
// particle's original index written to its sorted slot.
template <typename TR>
int run_sort_order(bspline_plan_s* p, const double* x, int64_t P, int* perm) {
    const BrickGrid g = brick_grid(p->N, p->dtype, p->order);
    const unsigned NB = g.NB;
    Ws<TR> w;
    const size_t need = carve<TR>(&w, nullptr, NB, P);
    int rc = p->pws.grow(need);
    if (rc) return rc;
    carve<TR>(&w, p->pws.ptr, NB, P);
    cudaStream_t st = p->stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.count, 0, sizeof(unsigned) * (NB + 2), st)) != cudaSuccess) return set_cuda_error(e);
    if ((e = cudaMemsetAsync(p->d_status, 0, sizeof(unsigned long long) * kStatusParticleWords, st)) != cudaSuccess)
        return set_cuda_error(e);
    const double scale = (double)p->N / p->L;
    const int agg = NB < kAggregateBricks;
    bin_kernel<TR, false, float><<<grid_for(P, 256), 256, 0, st>>>(x, P, p->N, scale, p->order, g, w, p->d_status, agg,
                                                                   (float*)nullptr, (float*)nullptr);
    scan_kernel<false><<<1, 1024, 0, st>>>(w.count, w.offset, w.cursor, w.chunk, w.item, NB, 0u);
    scatter_kernel<TR, float, false, true><<<grid_for(P, 256), 256, 0, st>>>(x, P, p->N, scale, p->order, g, w,
                                                                            (float*)nullptr, (float*)nullptr, agg,
                                                                            p->d_status, perm);
    return set_cuda_error(cudaGetLastError());
}

}  // namespace

int launch_sort_order(bspline_plan_s* p, const double* x, int64_t P, int* perm) {
    if (p->dtype == BSPLINE_F64) return run_sort_order<double>(p, x, P, perm);
    return run_sort_order<float>(p, x, P, perm);
}

int launch_adjoint_particles(bspline_plan_s* p, const void* coeffs, const double* x, int64_t P, const void* g_u,
                             const void* g_grad, void* g_coef, double* g_x) {
    switch (p->dtype) {
        case BSPLINE_F64:
            return run_adjoint_particles<double, double>(p, coeffs, x, P, g_u, g_grad, g_coef, g_x);
        case BSPLINE_F32:
            return run_adjoint_particles<float, float>(p, coeffs, x, P, g_u, g_grad, g_coef, g_x);
        case BSPLINE_BF16:
            return run_adjoint_particles<__nv_bfloat16, float>(p, coeffs, x, P, g_u, g_grad, g_coef, g_x);
    }
    return BSPLINE_ERR_INVALID_ARG;
}

int launch_interp_ws(bspline_plan_s* p, void* ws, unsigned long long* status, const void* coeffs, const double* x,
                     int64_t P, void* out_u, void* out_grad, int flags) {
    switch (p->dtype) {
        case BSPLINE_F64:
            return run_interp_ws<double, double, double>(p, ws, status, coeffs, x, P, out_u, out_grad, flags);
        case BSPLINE_F32:
            return run_interp_ws<float, float, float>(p, ws, status, coeffs, x, P, out_u, out_grad, flags);
        case BSPLINE_BF16:
            return run_interp_ws<__nv_bfloat16, float, float>(p, ws, status, coeffs, x, P, out_u, out_grad, flags);
    }
    return BSPLINE_ERR_INVALID_ARG;
}

size_t interp_workspace_bytes(const bspline_plan_s* p, int64_t P) {
    const BrickGrid g = brick_grid(p->N, p->dtype, p->order);
    const unsigned NB = g.NB;
    if (p->dtype == BSPLINE_F64) {
        Ws<double> w;
        return carve<double>(&w, nullptr, NB, P);
    }
    Ws<float> w;
    return carve<float>(&w, nullptr, NB, P);
}

int launch_interp_split(bspline_plan_s* p, const void* coeffs, const double* x, int64_t P, void* out_u,
                        void* out_grad, int flags, cudaStream_t sort_stream, cudaEvent_t sorted) {
    switch (p->dtype) {
        case BSPLINE_F64:
            return run_interp<double, double, double>(p, coeffs, x, P, out_u, out_grad, flags, sort_stream, sorted);
        case BSPLINE_F32:
            return run_interp<float, float, float>(p, coeffs, x, P, out_u, out_grad, flags, sort_stream, sorted);
        case BSPLINE_BF16:
            return run_interp<__nv_bfloat16, float, float>(p, coeffs, x, P, out_u, out_grad, flags, sort_stream,
                                                           sorted);
    }
    return BSPLINE_ERR_INVALID_ARG;
}

int launch_interp(bspline_plan_s* p, const void* coeffs, const double* x, int64_t P, void* out_u, void* out_grad,
                  int flags) {
    return launch_interp_split(p, coeffs, x, P, out_u, out_grad, flags, nullptr, nullptr);
}

}  // namespace bs

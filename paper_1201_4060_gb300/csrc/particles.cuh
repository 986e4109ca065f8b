// Shared definitions of the particle kernels: workspace layout, weights, gather.
// Included by particles.cu (binning, sort, dispatch) and by the gather_*.cu
// translation units that instantiate the gather for each coefficient type and
// order range (split only to compile in parallel).
#pragma once
#include <cuda.h>

#include <cstring>

#include "internal.h"

namespace bs {
namespace gather_impl {

// Tensor map of the coefficient array [3][N][N][N] (FP32, or BF16 with
// elem_bytes = 2) for TMA tile loads: box (z, y, x, component) = (box_z,
// box_y, box_x, 1).  Defined in particles.cu; BSPLINE_OK, or an error if the
// driver's encoder is missing or refuses (the caller then stages with cp.async).
int encode_coef_tmap(CUtensorMap* map, const void* coef, int N, int box_z, int box_y, int box_x, int elem_bytes = 4);

constexpr int kAnchorBits = 10;          // N <= 1024

// One particle's located record: packed first stencil node
// (ax << 20 | ay << 10 | az), the local variable t per axis and the
// particle's original index.  Exactly one 32-byte sector: the placement pass
// writes records to scattered slots, and a record that filled only part of a
// sector would cost a read-modify-write of it in DRAM.
template <typename TR> struct Rec;
template <> struct __align__(32) Rec<float> {
    unsigned cell;
    float t[3];
    unsigned idx;
    unsigned pad[3];    // written as zeros, so that every store covers the whole sector
};
template <> struct __align__(32) Rec<double> {
    unsigned cell;
    unsigned idx;
    double t[3];
};
static_assert(sizeof(Rec<float>) == 32 && sizeof(Rec<double>) == 32, "one sector per record");

// Particles per gather work item: a brick with more particles is split into
// several items, each staging the brick's tile, so no CTA serialises a clump.
constexpr unsigned kChunk = 2048;

template <typename TR> struct Ws {
    unsigned* count;    // [NB + 2]  particles per brick; slot NB = invalid positions; NB + 1 = *unsorted
    unsigned* unsorted; // nonzero if positions passed as sorted were not in brick order (count pass)
    unsigned* offset;   // [NB + 3]  start of each brick's sorted segment; [NB] end of the valid
                        //           particles, [NB + 1] end of all, [NB + 2] start of the sparse range
    unsigned* cursor;   // [NB + 1]  next free sorted slot of each brick (starts at offset)
    unsigned* chunk;    // [NB + 1]  exclusive prefix sum of ceil(count / kChunk): first work item of a brick
    unsigned* item;     // [NB + ceil(P / kChunk)]  brick of each work item (the first chunk[NB] are set)
    long long P;        // particles
    Rec<TR>* s_rec;     // [P]       located records sorted by brick
};

inline size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename TR> size_t carve(Ws<TR>* w, void* base, unsigned NB, int64_t P, unsigned chunk_len = kChunk) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void* ptr = base ? (void*)((char*)base + off) : nullptr;
        off += align_up(bytes);
        return ptr;
    };
    w->P = P;
    w->count = (unsigned*)take(sizeof(unsigned) * (NB + 2));
    w->unsorted = base ? w->count + NB + 1 : nullptr;
    w->offset = (unsigned*)take(sizeof(unsigned) * (NB + 3));
    w->cursor = (unsigned*)take(sizeof(unsigned) * (NB + 1));
    w->chunk = (unsigned*)take(sizeof(unsigned) * (NB + 1));
    w->item = (unsigned*)take(sizeof(unsigned) * (NB + (P + chunk_len - 1) / chunk_len));
    w->s_rec = (Rec<TR>*)take(sizeof(Rec<TR>) * P);
    return off;
}

// Periodic grid index of i >= 0 (a single subtraction in the common case i < 2N).
__device__ __forceinline__ int wrap_index(int i, int N) { return i < N ? i : (i < 2 * N ? i - N : i % N); }

// ------------------------------------------------------------------ locate
// For 0 <= s < 2^52: base = floor(s - n/2) and t = (s - n/2) - base rounded to
// float, computed exactly from the bits of s with integer operations (GB300's
// FP64 pipe is narrow: only s = x N / L stays in FP64).  s = fl + fr 2^-sa
// with integer fl and an sa-bit fraction fr; for odd n the half is folded
// into the fraction.  Returns false outside that range.
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }   // -126 <= k <= 127

__device__ __forceinline__ bool locate_nonneg(double s, int n, long long* base, float* t) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    if (b >> 63) return false;                                 // negative
    const int e = (int)(b >> 52) - 1023;                       // unbiased exponent
    if (e >= 52) return false;                                 // >= 2^52, Inf or NaN
    const unsigned long long m = (b & ((1ULL << 52) - 1)) | (1ULL << 52);
    const long long hfl = n >> 1;                              // floor(n / 2)
    if (e < 0) {                                               // s in [0, 1)
        // below 2^-60 (or subnormal) s is 0 to the FP32 accuracy of the weights
        const float sf = (e < -60) ? 0.f : __ull2float_rn(m) * pow2f(e - 52);
        if (!(n & 1)) {
            *base = -hfl;
            *t = sf;
        } else if (e == -1) {                                  // s in [0.5, 1): s - 1/2 = (m - 2^52) 2^-53
            *base = -hfl;
            *t = __ull2float_rn(m - (1ULL << 52)) * pow2f(-53);
        } else {                                               // s in [0, 0.5)
            *base = -hfl - 1;
            *t = sf + 0.5f;
        }
        return true;
    }
    const int sa = 52 - e;                                     // fraction bits, 1..52
    const long long fl = (long long)(m >> sa);
    const unsigned long long fr = m & ((1ULL << sa) - 1);
    if (!(n & 1)) {
        *base = fl - hfl;
        *t = __ull2float_rn(fr) * pow2f(-sa);
    } else {
        const unsigned long long hb = 1ULL << (sa - 1);        // one half in the fraction's units
        if (fr >= hb) {
            *base = fl - hfl;
            *t = __ull2float_rn(fr - hb) * pow2f(-sa);
        } else {
            *base = fl - hfl - 1;
            *t = __ull2float_rn(fr + hb) * pow2f(-sa);
        }
    }
    return true;
}

// First stencil node modulo N (N a power of two, or 3 times one).
__device__ __forceinline__ unsigned wrap_anchor(long long a, int N) {
    if ((N & (N - 1)) == 0) return (unsigned)(a & (long long)(N - 1));
    long long r = a % N;
    return (unsigned)(r < 0 ? r + N : r);
}

// Locate one particle (Eq. alg-int-6): its brick key and record; the key is NB
// for a non-finite position or one with no fractional bits left.
template <typename TR>
__device__ __forceinline__ unsigned locate_particle(const double* __restrict__ x, long long p, int N, double scale,
                                                    int order, const BrickGrid& g, Rec<TR>* r) {
    const unsigned NB = g.NB;
    unsigned anc[3];
    TR tt[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double s = x[3 * p + a] * scale;
        if constexpr (sizeof(TR) == 4) {
            long long base;
            float tf;
            if (locate_nonneg(s, order, &base, &tf)) {
                tt[a] = tf;
                anc[a] = wrap_anchor(base + 1, N);
                continue;
            }
        }
        const double sh = s - 0.5 * order;
        if (!(fabs(sh) < 4.0e15)) {      // NaN, Inf, or no fractional bits left
            ok = false;
            anc[a] = 0;
            tt[a] = 0;
            continue;
        }
        const double f = floor(sh);
        tt[a] = (TR)(sh - f);
        anc[a] = wrap_anchor((long long)f + 1, N);
    }
    if (!ok) return NB;
    r->cell = (anc[0] << (2 * kAnchorBits)) | (anc[1] << kAnchorBits) | anc[2];
    r->t[0] = tt[0];
    r->t[1] = tt[1];
    r->t[2] = tt[2];
    return ((anc[0] >> g.bshift) * (unsigned)g.nby + anc[1] / (unsigned)g.by) * (unsigned)g.nbz + (anc[2] >> g.bshift);
}

// ------------------------------------------------------------------ weights
// v[m] = M_k(t + m), m = 0..k-1, for the cardinal B-spline of order k.
// Node j (0-based, j = 0 leftmost) of an order-n stencil has weight
// B(t + n/2 - 1 - j) = M_n(t + n - 1 - j) and derivative
// M_{n-1}(t + n - 1 - j) - M_{n-1}(t + n - 2 - j).
template <int n, typename A>
__device__ __forceinline__ void bspline_weights(A t, A (&w)[n], A (&dw)[n]) {
    A v[n];
    v[0] = A(1);
#pragma unroll
    for (int m = 1; m < n; ++m) v[m] = A(0);
#pragma unroll
    for (int k = 2; k <= n - 1; ++k) {
        const A inv = A(1) / A(k - 1);
#pragma unroll
        for (int m = k - 1; m >= 0; --m) {
            const A left = (m > 0) ? v[m - 1] : A(0);
            v[m] = ((t + A(m)) * v[m] + (A(k - m) - t) * left) * inv;
        }
    }
    // v = order n-1 values; one more step for order n, derivative by differencing
    const A inv = A(1) / A(n - 1);
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const int m = n - 1 - j;
        const A vm = (m <= n - 2) ? v[m] : A(0);
        const A vl = (m >= 1) ? v[m - 1] : A(0);
        w[j] = ((t + A(m)) * vm + (A(n - m) - t) * vl) * inv;
        dw[j] = vm - vl;
    }
}

// ------------------------------------------------------------------ gather
// Coefficient tile of one brick: (BX + ORD - 1) x (BY + ORD - 1) x (BZ + ORD - 1)
// nodes per component, [c][x][y][z] with z fastest and z rows of PZ entries
// (FP32/BF16: padded to a multiple of 4 so every row starts 16-byte
// aligned), periodic wrap of the grid indices on staging.  FP32 and BF16
// coefficients are staged as FP32 (BF16 widened on load).
template <typename CT> struct TileT { using T = float; };
template <> struct TileT<double> { using T = double; };

template <typename CT> __device__ __forceinline__ typename TileT<CT>::T widen(CT v) { return v; }
template <> __device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// BYO: brick y extent other than the plan's default (batches tune it; 0 = brick_y).
template <typename CT, int ORD, int BYO = 0> struct Shape {
    static constexpr bool F64 = sizeof(CT) == 8;
    static constexpr int BX = brick_x(F64 ? BSPLINE_F64 : BSPLINE_F32);
    static constexpr int BY = BYO ? BYO : brick_y(F64 ? BSPLINE_F64 : BSPLINE_F32, ORD);
    static constexpr int BZ = BX;
    static constexpr int EX = BX + ORD - 1, EY = BY + ORD - 1, EZ = BZ + ORD - 1;
    static constexpr int PZ = F64 ? EZ : ((EZ + 3) & ~3);
    // strides of y, x and the component; FP32 tiles pad the component to 128 bytes (TMA destinations)
    static constexpr int SY = PZ, SX = EY * PZ, TS = F64 ? EX * SX : ((EX * SX + 31) & ~31);
};

template <int ORD, typename CT, int BYO = 0>
constexpr size_t tile_bytes() {
    return sizeof(typename TileT<CT>::T) * 3 * (size_t)Shape<CT, ORD, BYO>::TS;
}

// Brick index -> first cell of the brick.
template <int BX, int BY, int BZ>
__device__ __forceinline__ void brick_origin(unsigned brick, const BrickGrid& g, int* x0, int* y0, int* z0) {
    const unsigned bz = brick % (unsigned)g.nbz, t = brick / (unsigned)g.nbz;
    *z0 = (int)bz * BZ;
    *y0 = (int)(t % (unsigned)g.nby) * BY;
    *x0 = (int)(t / (unsigned)g.nby) * BX;
}

constexpr int kGatherThreads = 384;

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
// 16 bytes, cached in L2 only (each tile is read once per work item).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- TMA tile loads completing on a shared-memory mbarrier
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");   // visible to the async proxy
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}
// Box at coordinates (z, y, x, c) of `map` into shared memory at dst (128-byte aligned).
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int z, int y, int x, int c,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(z), "r"(y), "r"(x), "r"(c), "r"(smem_u32(bar))
        : "memory");
}
// Bounded wait for phase `parity` of the mbarrier (about a second of polls): false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
    for (long long it = 0; it < (1LL << 22); ++it) {
        if (mbar_test(bar, parity)) return true;
        __nanosleep(64);
    }
    return false;
}

// Copy the brick's tile into shared memory, one z-row per warp step: lane =
// z offset (lanes >= EZ idle).  Rows are walked in (c, ix, iy) order; indices
// wrap periodically.  Same-type coefficients go through cp.async (no register
// round trip); BF16 is widened to FP32 through registers.  The caller
// synchronises the CTA after cp_async_wait_all.
template <int ORD, typename CT, int BYO = 0>
__device__ __forceinline__ void stage_tile(typename TileT<CT>::T* tile, const CT* __restrict__ coef, int N, int x0,
                                           int y0, int z0) {
    using TT = typename TileT<CT>::T;
    using S = Shape<CT, ORD, BYO>;
    static_assert(S::EZ <= 32, "one z-row per warp step");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane >= S::EZ) return;
    const int gz = wrap_index(z0 + lane, N);
    // planes (c, ix): 3 EX of them, each EY rows along y; warps take planes round-robin
    for (int pl = warp; pl < 3 * S::EX; pl += nw) {
        const int c = pl / S::EX, ix = pl - c * S::EX;
        const CT* plane = coef + ((size_t)c * N + wrap_index(x0 + ix, N)) * (size_t)N * N + gz;
        TT* dst = tile + (size_t)c * S::TS + (size_t)ix * S::SX + lane;
        auto copy = [&](int iy, const CT* s) {
            if constexpr (sizeof(CT) == sizeof(TT)) {
                if constexpr (sizeof(CT) == 4) cp_async4(dst + iy * S::SY, s);
                else cp_async8(dst + iy * S::SY, s);
            } else {
                dst[iy * S::SY] = widen<CT>(*s);
            }
        };
        if (N >= S::EY) {
            // rows y0.. up to the end of the period advance by N; the rest wrap to row 0
            const int nrun = min(S::EY, N - y0);
            const CT* s = plane + (size_t)y0 * N;
#pragma unroll 7
            for (int iy = 0; iy < nrun; ++iy, s += N) copy(iy, s);
            s = plane;
            for (int iy = nrun; iy < S::EY; ++iy, s += N) copy(iy, s);
        } else {
            for (int iy = 0; iy < S::EY; ++iy) copy(iy, plane + (size_t)wrap_index(y0 + iy, N) * N);
        }
    }
}

// FP32 tiles with 16-byte copies: a tile row is PZ / 4 chunks of 4
// coefficients, 16-byte aligned in both memories (z0 and N are multiples of
// 4, so a chunk never straddles the periodic wrap).  Within a (c, ix) plane
// the lane -> (row, chunk) assignment and its offsets are the same for every
// plane, so they are computed once.
template <int ORD, int BYO = 0>
__device__ __forceinline__ void stage_tile16(float* tile, const float* __restrict__ coef, int N, int x0, int y0,
                                             int z0) {
    using S = Shape<float, ORD, BYO>;
    constexpr int CH = S::PZ / 4;                     // chunks per row
    constexpr int PER = S::EY * CH;                   // chunks per plane
    constexpr int NI = (PER + 31) / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int goff[NI], soff[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int f = lane + 32 * i;
        const int iy = f / CH, ch = f - iy * CH;
        goff[i] = f < PER ? wrap_index(y0 + iy, N) * N + wrap_index(z0 + 4 * ch, N) : -1;
        soff[i] = iy * S::SY + 4 * ch;
    }
    for (int pl = warp; pl < 3 * S::EX; pl += nw) {
        const int c = pl / S::EX, ix = pl - c * S::EX;
        const float* plane = coef + ((size_t)c * N + wrap_index(x0 + ix, N)) * (size_t)N * N;
        float* dst = tile + (size_t)c * S::TS + (size_t)ix * S::SX;
#pragma unroll
        for (int i = 0; i < NI; ++i)
            if (goff[i] >= 0) cp_async16(dst + soff[i], plane + goff[i]);
    }
}

// BF16 coefficients: 16-byte loads of 8 values (rows start at z0, a multiple
// of 16, and N is a multiple of 8, so a chunk never straddles the wrap),
// widened to FP32 in registers and stored as two 16-byte words.  All of a
// lane's loads of a plane are issued together, and the next plane's before
// this plane's stores (registers stand in for the asynchronous copy).
template <int ORD, int BYO = 0>
__device__ __forceinline__ void stage_tile_bf16(float* tile, const __nv_bfloat16* __restrict__ coef, int N, int x0,
                                                int y0, int z0) {
    using S = Shape<__nv_bfloat16, ORD, BYO>;
    constexpr int CH = (S::PZ + 7) / 8;               // chunks of 8 per row (the last may overhang the pitch)
    constexpr int PER = S::EY * CH;
    constexpr int NI = (PER + 31) / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int goff[NI], soff[NI], nst[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int f = lane + 32 * i;
        const int iy = f / CH, ch = f - iy * CH;
        goff[i] = f < PER ? wrap_index(y0 + iy, N) * N + wrap_index(z0 + 8 * ch, N) : -1;
        soff[i] = iy * S::SY + 8 * ch;
        nst[i] = (S::PZ - 8 * ch) >= 8 ? 2 : 1;       // 16-byte stores that stay inside the row pitch
    }
    // a warp's planes (c, ix) in turn, the next plane's loads in flight while this one is widened and stored
    auto load = [&](int pl, uint4 (&v)[NI]) {
        const int c = pl / S::EX, ix = pl - c * S::EX;
        const __nv_bfloat16* plane = coef + ((size_t)c * N + wrap_index(x0 + ix, N)) * (size_t)N * N;
#pragma unroll
        for (int i = 0; i < NI; ++i)
            if (goff[i] >= 0) v[i] = __ldg(reinterpret_cast<const uint4*>(plane + goff[i]));
    };
    uint4 v[NI], vn[NI];
    if (warp < 3 * S::EX) load(warp, vn);
    for (int pl = warp; pl < 3 * S::EX; pl += nw) {
#pragma unroll
        for (int i = 0; i < NI; ++i) v[i] = vn[i];
        if (pl + nw < 3 * S::EX) load(pl + nw, vn);
        const int c = pl / S::EX, ix = pl - c * S::EX;
        float* dst = tile + (size_t)c * S::TS + (size_t)ix * S::SX;
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            if (goff[i] < 0) continue;
            const unsigned w4[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
            float f[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                f[2 * q] = __uint_as_float(w4[q] << 16);             // bf16 -> fp32: the high half of the word
                f[2 * q + 1] = __uint_as_float(w4[q] & 0xffff0000u);
            }
            *reinterpret_cast<float4*>(dst + soff[i]) = make_float4(f[0], f[1], f[2], f[3]);
            if (nst[i] == 2) *reinterpret_cast<float4*>(dst + soff[i] + 4) = make_float4(f[4], f[5], f[6], f[7]);
        }
    }
}

// BF16 coefficients stay BF16 in shared memory, in two copies of the tile
// ([c][x][y][z], rows of PZ elements, 16-byte aligned): copy A holds element
// z of a row at z, copy B holds element z + 1 at z.  A stencil line of ORD
// values starting at tile z = oz is then ceil(ORD / 2) aligned 32-bit words:
// copy A from word oz / 2 if oz is even, copy B from word (oz - 1) / 2 if it
// is odd.  Each word carries two consecutive values (the lower z in its low
// half), widened to FP32 in registers, so the contraction reads half the
// shared-memory bytes of an FP32 tile with the same FP32 arithmetic.
template <int ORD, int BYO = 0> struct Bf16Pair {
    using S = Shape<__nv_bfloat16, ORD, BYO>;
    static constexpr int EX = S::EX, EY = S::EY, EZ = S::EZ;
    static constexpr int PZ = (EZ + 7) & ~7;            // elements per row: 16-byte rows
    static constexpr int SYW = PZ / 2, SXW = EY * SYW;  // words per row, per x-plane
    static constexpr int TSW = (EX * SXW + 31) & ~31;   // words per component
    static constexpr int COPYW = 3 * TSW;               // words per copy
    static constexpr int NWL = (ORD + 1) / 2;           // words per stencil line
    static constexpr size_t bytes = 2 * sizeof(unsigned) * (size_t)COPYW;
};

// Copy A of a brick: 16-byte cp.async chunks of 8 values (z0 is a multiple of
// 16 and N of 8, so no chunk straddles the periodic wrap); element by element
// below N = 16.  The caller waits for the copies and synchronises.
template <int ORD, int BYO>
__device__ __forceinline__ void stage_bf16_copy_a(unsigned* words, const __nv_bfloat16* __restrict__ coef, int N,
                                                  int x0, int y0, int z0) {
    using T = Bf16Pair<ORD, BYO>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (N >= 16) {
        constexpr int CH = T::PZ / 8;                   // chunks per row
        constexpr int PER = T::EY * CH;                 // chunks per (c, x) plane
        constexpr int NI = (PER + 31) / 32;
        int goff[NI], soff[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int f = lane + 32 * i;
            const int iy = f / CH, ch = f - iy * CH;
            goff[i] = f < PER ? wrap_index(y0 + iy, N) * N + wrap_index(z0 + 8 * ch, N) : -1;
            soff[i] = iy * T::SYW + 4 * ch;
        }
        for (int pl = warp; pl < 3 * T::EX; pl += nw) {
            const int c = pl / T::EX, ix = pl - c * T::EX;
            const __nv_bfloat16* plane = coef + ((size_t)c * N + wrap_index(x0 + ix, N)) * (size_t)N * N;
            unsigned* dst = words + (size_t)c * T::TSW + (size_t)ix * T::SXW;
#pragma unroll
            for (int i = 0; i < NI; ++i)
                if (goff[i] >= 0) cp_async16(dst + soff[i], plane + goff[i]);
        }
    } else {
        __nv_bfloat16* e = reinterpret_cast<__nv_bfloat16*>(words);
        for (int k = threadIdx.x; k < 3 * T::EX * T::EY * T::PZ; k += blockDim.x) {
            const int z = k % T::PZ, r = k / T::PZ, iy = r % T::EY, ix = (r / T::EY) % T::EX, c = r / (T::EY * T::EX);
            e[2 * ((size_t)c * T::TSW + (size_t)ix * T::SXW + (size_t)iy * T::SYW) + z] =
                coef[(((size_t)c * N + wrap_index(x0 + ix, N)) * N + wrap_index(y0 + iy, N)) * N + wrap_index(z0 + z, N)];
        }
    }
}

// Copy B from copy A: word j = (A[2j + 1], A[2j + 2]), four words per
// thread and step (16-byte accesses).  The upper value of a row's last word
// comes from the next row (or is zero at the end of the copy): it is never
// part of a stencil line.  Call after copy A is complete and visible; ends
// with a barrier.
template <int ORD, int BYO>
__device__ __forceinline__ void build_bf16_copy_b(unsigned* words) {
    using T = Bf16Pair<ORD, BYO>;
    static_assert(T::COPYW % 4 == 0, "16-byte steps");
    const uint4* a4 = reinterpret_cast<const uint4*>(words);
    uint4* b4 = reinterpret_cast<uint4*>(words + T::COPYW);
    for (int v = threadIdx.x; v < T::COPYW / 4; v += blockDim.x) {
        const uint4 a = a4[v];
        const unsigned nx = (4 * v + 4 < T::COPYW) ? words[4 * v + 4] : 0u;
        b4[v] = make_uint4(__byte_perm(a.x, a.y, 0x5432), __byte_perm(a.y, a.z, 0x5432), __byte_perm(a.z, a.w, 0x5432),
                           __byte_perm(a.w, nx, 0x5432));
    }
    __syncthreads();
}


__device__ __forceinline__ float bf16_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }

// TMA staging of an FP32 brick away from the periodic seams: thread 0 arms the
// mbarrier and issues one box (PZ, EY, EX, 1) per component; the boxes never
// leave the grid there (z0 <= N - 32 when z0 + EZ <= N), and the padding z
// rows beyond EZ are never read.  Returns whether the brick was staged this
// way (the caller stages the others with cp.async).  use_tma: 0 = never,
// kTmaOn = interior bricks, kTmaArmOnly = arm the barrier for the tile's bytes
// but issue no copy (test hook: the wait then runs out with nothing in flight).
constexpr int kTmaOn = 1, kTmaArmOnly = 2;
template <int ORD, typename CT, int BYO = 0>
__device__ __forceinline__ bool stage_tile_tma(float* tile, const CUtensorMap* map, unsigned long long* bar, int N,
                                               int x0, int y0, int z0, int use_tma) {
    using S = Shape<CT, ORD, BYO>;
    const bool tma = sizeof(CT) == 4 && use_tma && x0 + S::EX <= N && y0 + S::EY <= N && z0 + S::EZ <= N;
    if (tma && threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, 3u * S::PZ * S::EY * S::EX * (unsigned)sizeof(float));
        if (use_tma != kTmaArmOnly) {
#pragma unroll
            for (int c = 0; c < 3; ++c) tma_load_4d(tile + c * S::TS, map, z0, y0, x0, c, bar);
        }
    }
    return tma;
}

// TMA staging of copy A of a BF16 pair tile away from the periodic seams (as
// stage_tile_tma: one box (PZ, EY, EX, 1) per component, into the component's
// 128-byte aligned words); returns whether the brick was staged this way.
template <int ORD, int BYO>
__device__ __forceinline__ bool stage_bf16_tma(unsigned* words, const CUtensorMap* map, unsigned long long* bar,
                                               int N, int x0, int y0, int z0, int use_tma) {
    using T = Bf16Pair<ORD, BYO>;
    const bool tma = use_tma && x0 + T::EX <= N && y0 + T::EY <= N && z0 + T::EZ <= N;
    if (tma && threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, 3u * T::PZ * T::EY * T::EX * 2u);
        if (use_tma != kTmaArmOnly) {
#pragma unroll
            for (int c = 0; c < 3; ++c) tma_load_4d(words + c * T::TSW, map, z0, y0, x0, c, bar);
        }
    }
    return tma;
}

// Every thread waits for the TMA tile (observing the barrier's phase makes the
// bytes visible to it).  A wait that runs out (about a second) sets *flag,
// waits once more for the copies in flight, and returns false for the whole
// CTA, which then abandons its item.  Call after a barrier that follows the
// mbarrier's initialisation.
__device__ __forceinline__ bool tma_tile_wait(unsigned long long* bar, unsigned long long* flag) {
    const bool timed_out = __syncthreads_or(mbar_wait_bounded(bar, 0) ? 0 : 1) != 0;
    if (timed_out) {
        if (threadIdx.x == 0) atomicOr(flag, 1ULL);
        mbar_wait_bounded(bar, 0);
        return false;
    }
    return true;
}

// Outputs of an abandoned work item: NaN for each of its particles, so that a
// time-out never leaves stale values behind (the status word says why).
template <typename TR, typename AT>
__device__ __forceinline__ void fill_nan_item(const Ws<TR>& w, unsigned c0, unsigned n, AT* __restrict__ out_u,
                                              AT* __restrict__ out_grad, int ncomp_u) {
    const AT nan = (AT)NAN;
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
        const size_t idx = w.s_rec[c0 + i].idx;
        if (out_u) {
            for (int k = 0; k < ncomp_u; ++k) out_u[(size_t)ncomp_u * idx + k] = nan;
        }
        if (out_grad) {
#pragma unroll
            for (int k = 0; k < 9; ++k) out_grad[9 * idx + k] = nan;
        }
    }
}

template <int ORD, typename CT, int BYO = 0>
__device__ __forceinline__ void stage_brick(typename TileT<CT>::T* tile, const CT* __restrict__ coef, int N, int x0,
                                            int y0, int z0) {
    if constexpr (sizeof(CT) == 4) {
        if (N >= 16) {
            stage_tile16<ORD, BYO>(tile, coef, N, x0, y0, z0);
            return;
        }
    } else if constexpr (sizeof(CT) == 2) {
        if (N >= 16) {
            stage_tile_bf16<ORD, BYO>(tile, coef, N, x0, y0, z0);
            return;
        }
    }
    stage_tile<ORD, CT, BYO>(tile, coef, N, x0, y0, z0);
}

// u and grad u of one particle from the staged tile (Table 1 contraction,
// z axis first).  base points at the particle's first stencil node.
template <int ORD, typename A, bool GRAD, int SX, int SY, int TS>
__device__ __forceinline__ void eval_particle(const A* __restrict__ base, A tx, A ty, A tz, A dscale,
                                              A* __restrict__ out_u, A* __restrict__ out_grad) {
    A wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
    bspline_weights<ORD, A>(tx, wx, dwx);
    bspline_weights<ORD, A>(ty, wy, dwy);
    bspline_weights<ORD, A>(tz, wz, dwz);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const A* tc = base + c * TS;
        A u = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll
        for (int jx = 0; jx < ORD; ++jx) {
            A y00 = 0, y10 = 0, y01 = 0;
#pragma unroll
            for (int jy = 0; jy < ORD; ++jy) {
                const A* line = tc + jx * SX + jy * SY;
                A z0v = 0, z1v = 0;
#pragma unroll
                for (int jz = 0; jz < ORD; ++jz) {
                    const A a = line[jz];
                    z0v = fma(wz[jz], a, z0v);
                    if (GRAD) z1v = fma(dwz[jz], a, z1v);
                }
                y00 = fma(wy[jy], z0v, y00);
                if (GRAD) {
                    y10 = fma(dwy[jy], z0v, y10);
                    y01 = fma(wy[jy], z1v, y01);
                }
            }
            u = fma(wx[jx], y00, u);
            if (GRAD) {
                gx = fma(dwx[jx], y00, gx);
                gy = fma(wx[jx], y10, gy);
                gz = fma(wx[jx], y01, gz);
            }
        }
        out_u[c] = u;
        if (GRAD) {
            out_grad[3 * c + 0] = gx * dscale;
            out_grad[3 * c + 1] = gy * dscale;
            out_grad[3 * c + 2] = gz * dscale;
        }
    }
}

// Packed two-way FP32 contraction (fma.rn.f32x2) of one component:
// adjacent y-lines jy, jy + 1 are contracted along z together (their loads
// form the pair, the z weight is duplicated), and their y-sums are kept as
// (even, odd) pairs that are added at the end of each x-plane.  Same
// arithmetic per term as eval_particle; the sums are grouped by parity of jy.
// ld(jx, jy, jz) gives the coefficient at stencil node (jx, jy, jz): the
// staged gather reads its shared-memory tile, the direct gather global
// memory, with the same arithmetic in the same order, so the two agree bit
// for bit.
template <int ORD> struct PairWeights {
    static constexpr int NP = ORD / 2;                // pairs of y-lines
    float2 wz2[ORD], dwz2[ORD], wyp[NP > 0 ? NP : 1], dwyp[NP > 0 ? NP : 1];
    __device__ __forceinline__ PairWeights(const float (&wz)[ORD], const float (&dwz)[ORD], const float (&wy)[ORD],
                                           const float (&dwy)[ORD]) {
#pragma unroll
        for (int j = 0; j < ORD; ++j) {
            wz2[j] = make_float2(wz[j], wz[j]);
            dwz2[j] = make_float2(dwz[j], dwz[j]);
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            wyp[p] = make_float2(wy[2 * p], wy[2 * p + 1]);
            dwyp[p] = make_float2(dwy[2 * p], dwy[2 * p + 1]);
        }
    }
};

// One x-row of the contraction: ldr(jy, jz) gives the coefficient at
// (jy, jz) of the row; returns the row's sums s00 = sum_y wy sum_z wz c, s10
// with dwy, s01 with dwz.
template <int ORD, bool GRAD, typename LDR>
__device__ __forceinline__ void row_x2(LDR ldr, const PairWeights<ORD>& pw, const float (&wy)[ORD],
                                       const float (&dwy)[ORD], const float (&wz)[ORD], const float (&dwz)[ORD],
                                       float* s00, float* s10, float* s01) {
    constexpr int NP = ORD / 2;
    float2 y00 = make_float2(0.f, 0.f), y10 = y00, y01 = y00;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float2 z0 = make_float2(0.f, 0.f), z1 = z0;
#pragma unroll
        for (int jz = 0; jz < ORD; ++jz) {
            const float2 a = make_float2(ldr(2 * p, jz), ldr(2 * p + 1, jz));
            z0 = __ffma2_rn(pw.wz2[jz], a, z0);
            if (GRAD) z1 = __ffma2_rn(pw.dwz2[jz], a, z1);
        }
        y00 = __ffma2_rn(pw.wyp[p], z0, y00);
        if (GRAD) {
            y10 = __ffma2_rn(pw.dwyp[p], z0, y10);
            y01 = __ffma2_rn(pw.wyp[p], z1, y01);
        }
    }
    if constexpr (ORD % 2 == 1) {                   // the unpaired last line
        float z0 = 0.f, z1 = 0.f;
#pragma unroll
        for (int jz = 0; jz < ORD; ++jz) {
            const float a = ldr(ORD - 1, jz);
            z0 = fmaf(wz[jz], a, z0);
            if (GRAD) z1 = fmaf(dwz[jz], a, z1);
        }
        y00.x = fmaf(wy[ORD - 1], z0, y00.x);
        if (GRAD) {
            y10.x = fmaf(dwy[ORD - 1], z0, y10.x);
            y01.x = fmaf(wy[ORD - 1], z1, y01.x);
        }
    }
    *s00 = y00.x + y00.y;
    *s10 = y10.x + y10.y;
    *s01 = y01.x + y01.y;
}

// row_x2 on a BF16 pair tile: line jy of the x-row starts at word row0 + jy
// SYW; the same terms in the same order as row_x2 (pairs of y-lines, z
// ascending), each value the exact FP32 value of its BF16 coefficient.
template <int ORD, bool GRAD, int SYW>
__device__ __forceinline__ void row_x2_words(const unsigned* __restrict__ row0, const PairWeights<ORD>& pw,
                                             const float (&wy)[ORD], const float (&dwy)[ORD], const float (&wz)[ORD],
                                             const float (&dwz)[ORD], float* s00, float* s10, float* s01) {
    constexpr int NP = ORD / 2, NWL = (ORD + 1) / 2;
    float2 y00 = make_float2(0.f, 0.f), y10 = y00, y01 = y00;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const unsigned* l0 = row0 + (2 * p) * SYW;
        const unsigned* l1 = l0 + SYW;
        float2 z0 = make_float2(0.f, 0.f), z1 = z0;
#pragma unroll
        for (int k = 0; k < NWL; ++k) {
            const unsigned a = l0[k], b = l1[k];
            const float2 v0 = make_float2(bf16_lo(a), bf16_lo(b));
            z0 = __ffma2_rn(pw.wz2[2 * k], v0, z0);
            if (GRAD) z1 = __ffma2_rn(pw.dwz2[2 * k], v0, z1);
            if (2 * k + 1 < ORD) {
                const float2 v1 = make_float2(bf16_hi(a), bf16_hi(b));
                z0 = __ffma2_rn(pw.wz2[2 * k + 1], v1, z0);
                if (GRAD) z1 = __ffma2_rn(pw.dwz2[2 * k + 1], v1, z1);
            }
        }
        y00 = __ffma2_rn(pw.wyp[p], z0, y00);
        if (GRAD) {
            y10 = __ffma2_rn(pw.dwyp[p], z0, y10);
            y01 = __ffma2_rn(pw.wyp[p], z1, y01);
        }
    }
    if constexpr (ORD % 2 == 1) {                   // the unpaired last line
        const unsigned* l = row0 + (ORD - 1) * SYW;
        float z0 = 0.f, z1 = 0.f;
#pragma unroll
        for (int k = 0; k < NWL; ++k) {
            const unsigned a = l[k];
            z0 = fmaf(wz[2 * k], bf16_lo(a), z0);
            if (GRAD) z1 = fmaf(dwz[2 * k], bf16_lo(a), z1);
            if (2 * k + 1 < ORD) {
                z0 = fmaf(wz[2 * k + 1], bf16_hi(a), z0);
                if (GRAD) z1 = fmaf(dwz[2 * k + 1], bf16_hi(a), z1);
            }
        }
        y00.x = fmaf(wy[ORD - 1], z0, y00.x);
        if (GRAD) {
            y10.x = fmaf(dwy[ORD - 1], z0, y10.x);
            y01.x = fmaf(wy[ORD - 1], z1, y01.x);
        }
    }
    *s00 = y00.x + y00.y;
    *s10 = y10.x + y10.y;
    *s01 = y01.x + y01.y;
}

// Accumulation of one x-row's sums into u and the gradient.
template <bool GRAD>
__device__ __forceinline__ void add_row(float wxj, float dwxj, float s00, float s10, float s01, float* u, float* gx,
                                        float* gy, float* gz) {
    *u = fmaf(wxj, s00, *u);
    if (GRAD) {
        *gx = fmaf(dwxj, s00, *gx);
        *gy = fmaf(wxj, s10, *gy);
        *gz = fmaf(wxj, s01, *gz);
    }
}

template <int ORD, bool GRAD, typename LD>
__device__ __forceinline__ void contract_x2(LD ld, const PairWeights<ORD>& pw, const float (&wx)[ORD],
                                            const float (&dwx)[ORD], const float (&wy)[ORD], const float (&dwy)[ORD],
                                            const float (&wz)[ORD], const float (&dwz)[ORD], float dscale,
                                            float* __restrict__ out_u, float* __restrict__ out_grad) {
    float u = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int jx = 0; jx < ORD; ++jx) {
        float s00, s10, s01;
        row_x2<ORD, GRAD>([&](int jy, int jz) { return ld(jx, jy, jz); }, pw, wy, dwy, wz, dwz, &s00, &s10, &s01);
        add_row<GRAD>(wx[jx], dwx[jx], s00, s10, s01, &u, &gx, &gy, &gz);
    }
    *out_u = u;
    if (GRAD) {
        out_grad[0] = gx * dscale;
        out_grad[1] = gy * dscale;
        out_grad[2] = gz * dscale;
    }
}

// All three components of one particle from the staged tile (weights once).
template <int ORD, bool GRAD, int SX, int SY, int TS>
__device__ __forceinline__ void eval_particle_x2(const float* __restrict__ base, float tx, float ty, float tz,
                                                 float dscale, float* __restrict__ out_u,
                                                 float* __restrict__ out_grad) {
    float wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
    bspline_weights<ORD, float>(tx, wx, dwx);
    bspline_weights<ORD, float>(ty, wy, dwy);
    bspline_weights<ORD, float>(tz, wz, dwz);
    const PairWeights<ORD> pw(wz, dwz, wy, dwy);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float* tc = base + c * TS;
        contract_x2<ORD, GRAD>([&](int jx, int jy, int jz) { return tc[jx * SX + jy * SY + jz]; }, pw, wx, dwx, wy,
                               dwy, wz, dwz, dscale, &out_u[c], &out_grad[3 * c]);
    }
}

// One component of eval_particle_x2; base points at the component's first stencil node.
template <int ORD, bool GRAD, int SX, int SY>
__device__ __forceinline__ void eval_component_x2(const float* __restrict__ base, float tx, float ty, float tz,
                                                  float dscale, float* __restrict__ out_u,
                                                  float* __restrict__ out_grad) {
    float wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
    bspline_weights<ORD, float>(tx, wx, dwx);
    bspline_weights<ORD, float>(ty, wy, dwy);
    bspline_weights<ORD, float>(tz, wz, dwz);
    const PairWeights<ORD> pw(wz, dwz, wy, dwy);
    contract_x2<ORD, GRAD>([&](int jx, int jy, int jz) { return base[jx * SX + jy * SY + jz]; }, pw, wx, dwx, wy,
                           dwy, wz, dwz, dscale, out_u, out_grad);
}

// Components c0..c0+NC-1 of one particle from a BF16 pair tile (weights once);
// base = the particle's first stencil word of component 0 in its copy.
template <int ORD, bool GRAD, typename T, int NC>
__device__ __forceinline__ void eval_bf16(const unsigned* __restrict__ base, int c0, float tx, float ty, float tz,
                                          float dscale, float* __restrict__ out_u, float* __restrict__ out_grad) {
    float wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
    bspline_weights<ORD, float>(tx, wx, dwx);
    bspline_weights<ORD, float>(ty, wy, dwy);
    bspline_weights<ORD, float>(tz, wz, dwz);
    const PairWeights<ORD> pw(wz, dwz, wy, dwy);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const unsigned* cb = base + (c0 + q) * T::TSW;
        float u = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
        for (int jx = 0; jx < ORD; ++jx) {
            float s00, s10, s01;
            row_x2_words<ORD, GRAD, T::SYW>(cb + jx * T::SXW, pw, wy, dwy, wz, dwz, &s00, &s10, &s01);
            add_row<GRAD>(wx[jx], dwx[jx], s00, s10, s01, &u, &gx, &gy, &gz);
        }
        out_u[q] = u;
        if (GRAD) {
            out_grad[3 * q + 0] = gx * dscale;
            out_grad[3 * q + 1] = gy * dscale;
            out_grad[3 * q + 2] = gz * dscale;
        }
    }
}

// FP64: one thread per particle (the FP64 pipe, not shared memory, bounds it).
template <int ORD, typename TR, bool GRAD>
__global__ void __launch_bounds__(128)
gather_f64(const double* __restrict__ coef, int N, BrickGrid bg, Ws<TR> w, double* __restrict__ out_u,
           double* __restrict__ out_grad, double dscale, unsigned long long* __restrict__ status) {
    using S = Shape<double, ORD>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* tile = reinterpret_cast<double*>(smem_raw);
    const unsigned brick = blockIdx.x;
    const unsigned beg = w.offset[brick], end = beg + w.count[brick];
    if (beg == end) return;
    int x0, y0, z0;
    brick_origin<S::BX, S::BY, S::BZ>(brick, bg, &x0, &y0, &z0);
    stage_brick<ORD, double>(tile, coef, N, x0, y0, z0);
    cp_async_wait_all();
    __syncthreads();
    for (unsigned i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const Rec<TR> rc = w.s_rec[i];
        const int ox = (int)(rc.cell >> (2 * kAnchorBits)) - x0;
        const int oy = (int)((rc.cell >> kAnchorBits) & 1023u) - y0;
        const int oz = (int)(rc.cell & 1023u) - z0;
        const unsigned idx = rc.idx;
        if (!BS_CHECK_OK(ox >= 0 && ox < S::BX && oy >= 0 && oy < S::BY && oz >= 0 && oz < S::BZ &&
                             (long long)idx < w.P,
                         status + kStatusBounds))
            continue;
        double u[3], gr[9];
        eval_particle<ORD, double, GRAD, S::SX, S::SY, S::TS>(tile + ox * S::SX + oy * S::SY + oz, (double)rc.t[0],
                                                               (double)rc.t[1], (double)rc.t[2], dscale, u, gr);
#pragma unroll
        for (int c = 0; c < 3; ++c) out_u[3 * (size_t)idx + c] = u[c];
        if (GRAD) {
#pragma unroll
            for (int k = 0; k < 9; ++k) out_grad[9 * (size_t)idx + k] = gr[k];
        }
    }
}

// A particle's outputs go to its original index, scattered: u (12 bytes) and
// grad u (36 bytes) are written with 8-byte stores where they are 8-byte
// aligned and one 4-byte store for the odd word, chosen by the index's
// parity with selects (no divergence): 2 + 5 store instructions instead of
// 3 + 9, since the load/store queue, not the bytes, is what the scattered
// stores occupy.  Needs 8-byte aligned output arrays (the caller checks).
__device__ __forceinline__ void store_u3(float* p, unsigned odd, const float (&u)[3]) {
    // even index: (u0, u1) at p, u2 at p + 2; odd: u0 at p, (u1, u2) at p + 1
    float* s = odd ? p : p + 2;
    float* v = odd ? p + 1 : p;
    *s = odd ? u[0] : u[2];
    *reinterpret_cast<float2*>(v) = odd ? make_float2(u[1], u[2]) : make_float2(u[0], u[1]);
}
__device__ __forceinline__ void store_g9(float* p, unsigned odd, const float (&g)[9]) {
    // even index: four pairs from p, g8 at p + 8; odd: g0 at p, four pairs from p + 1
    float* s = odd ? p : p + 8;
    float* v = odd ? p + 1 : p;
    *s = odd ? g[0] : g[8];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        *reinterpret_cast<float2*>(v + 2 * k) =
            odd ? make_float2(g[2 * k + 1], g[2 * k + 2]) : make_float2(g[2 * k], g[2 * k + 1]);
}

// FP32 accumulation (FP32 or BF16 coefficients).  Each particle reads
// 3 ORD^3 tile values from shared memory, and a warp load costs one cycle per
// distinct address in the busiest of the 32 banks; random stencil origins
// would make most loads 3-4 way conflicted.  Within a chunk, particles are
// therefore bucketed by the bank of their stencil origin (residue mod 32),
// ranked within their bucket, and ordered rank-major, bank-minor: a warp
// that takes 32 consecutive particles of that order sees each bank at most
// once per rank it spans.
// One CTA per work item: item i is chunk i - chunk[b] of the brick b with
// chunk[b] <= i < chunk[b + 1] (at most kChunk particles); the grid is an
// upper bound on the number of items and surplus CTAs return at once.
// Two CTAs per SM (80 registers): orders 7 and 8 would otherwise take 84 and
// 102 registers and run one CTA per SM, 22 % and 16 % slower at 256^3.
// gather_f32_item evaluates work item `item` (at most chunk_len <= kChunk
// particles of one brick); the kernel gather_f32 runs one item per CTA, the
// batch kernel many per CTA (BYO: its brick y extent).  The caller has
// checked item < w.chunk[NB] and keeps every thread of the CTA here.
template <int ORD, typename CT, typename TR, bool GRAD, int BYO = 0>
__device__ __forceinline__ void gather_f32_item(unsigned item, unsigned chunk_len, const CT* __restrict__ coef, int N,
                                                const BrickGrid& bg, const Ws<TR>& w, float* __restrict__ out_u,
                                                float* __restrict__ out_grad, float dscale, const CUtensorMap* tmap,
                                                int use_tma, unsigned long long* __restrict__ status) {
    using S = Shape<CT, ORD, BYO>;
    constexpr int NW = kGatherThreads / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the tile 128-byte aligned (TMA destinations; the launch adds 128 bytes of slack), offset from the
    // shared array itself so that its loads stay shared-memory loads (an address rebuilt from an integer
    // would be a generic one)
    float* tile = reinterpret_cast<float*>(smem_raw + ((0u - smem_u32(smem_raw)) & 127u));
    __shared__ unsigned s_bucket[32];
    __shared__ unsigned short s_order[kChunk];
    __shared__ __align__(8) unsigned long long s_mbar;
    const unsigned brick = w.item[item];
    const unsigned c0 = w.offset[brick] + (item - w.chunk[brick]) * chunk_len;
    const unsigned end = w.offset[brick] + w.count[brick];
    int x0, y0, z0;
    brick_origin<S::BX, S::BY, S::BZ>(brick, bg, &x0, &y0, &z0);
    // BF16: the pair tile (copy A now, asynchronously; copy B after the bucketing)
    constexpr bool kBf16 = sizeof(CT) == 2;
    using T2 = Bf16Pair<ORD, BYO>;
    unsigned* words = reinterpret_cast<unsigned*>(tile);
    // bricks away from the periodic seams by TMA, the others with cp.async
    bool tma;
    if constexpr (kBf16) tma = stage_bf16_tma<ORD, BYO>(words, tmap, &s_mbar, N, x0, y0, z0, use_tma);
    else tma = stage_tile_tma<ORD, CT, BYO>(tile, tmap, &s_mbar, N, x0, y0, z0, use_tma);
    if (tma) {
    } else if constexpr (kBf16) {
        stage_bf16_copy_a<ORD, BYO>(words, reinterpret_cast<const __nv_bfloat16*>(coef), N, x0, y0, z0);
    } else {
        stage_brick<ORD, CT, BYO>(tile, coef, N, x0, y0, z0);
    }
    // shared-memory bank (word index mod 32) of a particle's first stencil value
    auto bank_of = [&](int ox, int oy, int oz) -> unsigned {
        if constexpr (kBf16)
            return (unsigned)(((oz & 1) ? T2::COPYW : 0) + (ox * T2::EY + oy) * T2::SYW + (oz >> 1)) & 31u;
        else
            return (unsigned)(ox * S::SX + oy * S::SY + oz) & 31u;
    };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec_out = ((reinterpret_cast<uintptr_t>(out_u) | (GRAD ? reinterpret_cast<uintptr_t>(out_grad) : 0u)) &
                          7u) == 0u;
    // checks build: the stencil inside the staged tile, the output index inside the arrays
    auto origin_ok = [&](int ox, int oy, int oz, unsigned idx) {
        return BS_CHECK_OK(ox >= 0 && ox < S::BX && oy >= 0 && oy < S::BY && oz >= 0 && oz < S::BZ &&
                               (long long)idx < w.P,
                           status + kStatusBounds);
    };
    {
        const int n = (int)min(chunk_len, end - c0);
        if (threadIdx.x < 32) s_bucket[threadIdx.x] = 0;
        __syncthreads();                                  // the tile copies stay in flight while bucketing
        // bucket (bank residue of the stencil origin) and rank within it, kept in registers
        constexpr int KT = (kChunk + kGatherThreads - 1) / kGatherThreads;
        unsigned packed[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int i = threadIdx.x + k * kGatherThreads;
            if (i < n) {
                const unsigned cp = w.s_rec[c0 + i].cell;
                const int ox = (int)(cp >> (2 * kAnchorBits)) - x0;
                const int oy = (int)((cp >> kAnchorBits) & 1023u) - y0;
                const int oz = (int)(cp & 1023u) - z0;
                const unsigned r = bank_of(ox, oy, oz);
                packed[k] = (atomicAdd(&s_bucket[r], 1u) << 5) | r;
            }
        }
        __syncthreads();
        // job-sorted position: all particles of smaller rank, then the same rank in smaller buckets
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const int i = threadIdx.x + k * kGatherThreads;
            if (i < n) {
                const unsigned r = packed[k] & 31u, rk = packed[k] >> 5;
                unsigned pos = 0;
#pragma unroll 8
                for (unsigned q = 0; q < 32; ++q) {
                    const unsigned bq = s_bucket[q];
                    pos += min(bq, rk) + ((q < r && bq > rk) ? 1u : 0u);
                }
                if (BS_CHECK_OK(pos < (unsigned)n, status + kStatusBounds)) s_order[pos] = (unsigned short)i;
            }
        }
        cp_async_wait_all();
        if (tma && !tma_tile_wait(&s_mbar, status + kStatusParticleTimeout)) {
            fill_nan_item<TR, float>(w, c0, (unsigned)n, out_u, GRAD ? out_grad : nullptr, 3);
            return;
        }
        __syncthreads();                                  // tile and order ready
        if constexpr (kBf16) build_bf16_copy_b<ORD, BYO>(words);
        // Warp jobs over that order.  Rank j holds #{banks with more than j
        // particles} particles, non-increasing in j.  While a rank holds at
        // least 16 particles it is one job (every load conflict-free); the
        // sparse tail ranks are packed 32 to a job: a job spanning k ranks
        // costs k-way conflicts, as k separate jobs would, in one instruction
        // stream instead of k.
        const unsigned my_bucket = s_bucket[lane];
        unsigned above = 0;                               // buckets ordered before this lane's
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const unsigned bq = __shfl_sync(0xffffffffu, my_bucket, q);
            above += (bq > my_bucket || (bq == my_bucket && q < lane)) ? 1u : 0u;
        }
        const unsigned src16 = __ffs(__ballot_sync(0xffffffffu, above == 15u)) - 1;
        const unsigned j16 = __shfl_sync(0xffffffffu, my_bucket, src16);   // ranks j < j16 hold >= 16
        const unsigned pos16 = __reduce_add_sync(0xffffffffu, min(my_bucket, j16));
        const unsigned njobs = j16 + ((unsigned)n - pos16 + 31u) / 32u;
        auto job_range = [&](unsigned j, unsigned* lo, unsigned* hi) {
            if (j < j16) {
                *lo = __reduce_add_sync(0xffffffffu, min(my_bucket, j));
                *hi = __reduce_add_sync(0xffffffffu, min(my_bucket, j + 1));
            } else {
                *lo = pos16 + 32u * (j - j16);
                *hi = min((unsigned)n, *lo + 32u);
            }
        };
        // the next job's record is loaded while the current one is evaluated
        Rec<TR> rc_n;
        bool v_n = false;
        auto fetch = [&](unsigned j) {
            unsigned lo, hi;
            job_range(j, &lo, &hi);
            const unsigned pos = lo + (unsigned)lane;
            v_n = pos < hi;
            if (v_n) {
                const unsigned i = c0 + s_order[pos];
                rc_n = w.s_rec[i];
            }
        };
        // Jobs are dealt to the NW warps in rounds.  A last, partly filled round
        // of m <= 2 NW / 3 jobs is run per component instead: 3 m shorter warp
        // tasks (one component of the job's 32 particles each), so the item
        // does not wait a whole job time on a few warps.
        const unsigned m_tail = njobs % NW;
        const unsigned jfull = (m_tail != 0 && 3 * m_tail <= 2 * NW) ? njobs - m_tail : njobs;
        if ((unsigned)warp < jfull) fetch(warp);
        for (unsigned j = warp; j < jfull; j += NW) {
            const Rec<TR> rc = rc_n;
            const unsigned idx = rc.idx;
            const bool v = v_n;
            v_n = false;
            if (j + NW < jfull) fetch(j + NW);
            if (v) {
                const int ox = (int)(rc.cell >> (2 * kAnchorBits)) - x0;
                const int oy = (int)((rc.cell >> kAnchorBits) & 1023u) - y0;
                const int oz = (int)(rc.cell & 1023u) - z0;
                if (!origin_ok(ox, oy, oz, idx)) continue;
                float u[3], g[9];
                if constexpr (kBf16)
                    eval_bf16<ORD, GRAD, T2, 3>(words + ((oz & 1) ? T2::COPYW : 0) + (ox * T2::EY + oy) * T2::SYW +
                                                    (oz >> 1),
                                                0, (float)rc.t[0], (float)rc.t[1], (float)rc.t[2], dscale, u, g);
                else
                    eval_particle_x2<ORD, GRAD, S::SX, S::SY, S::TS>(tile + ox * S::SX + oy * S::SY + oz,
                                                                      (float)rc.t[0], (float)rc.t[1], (float)rc.t[2],
                                                                      dscale, u, g);
                if (vec_out) {
                    store_u3(out_u + 3 * (size_t)idx, idx & 1u, u);
                    if (GRAD) store_g9(out_grad + 9 * (size_t)idx, idx & 1u, g);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) out_u[3 * (size_t)idx + c] = u[c];
                    if (GRAD) {
#pragma unroll
                        for (int k = 0; k < 9; ++k) out_grad[9 * (size_t)idx + k] = g[k];
                    }
                }
            }
        }
        for (unsigned q = warp; q < 3 * (njobs - jfull); q += NW) {
            const unsigned c = q % 3;
            unsigned lo, hi;
            job_range(jfull + q / 3, &lo, &hi);
            const unsigned pos = lo + (unsigned)lane;
            if (pos < hi) {
                const unsigned i = c0 + s_order[pos];
                const Rec<TR> rc = w.s_rec[i];
                const unsigned idx = rc.idx;
                const int ox = (int)(rc.cell >> (2 * kAnchorBits)) - x0;
                const int oy = (int)((rc.cell >> kAnchorBits) & 1023u) - y0;
                const int oz = (int)(rc.cell & 1023u) - z0;
                if (!origin_ok(ox, oy, oz, idx)) continue;
                float u, g[3];
                if constexpr (kBf16)
                    eval_bf16<ORD, GRAD, T2, 1>(words + ((oz & 1) ? T2::COPYW : 0) + (ox * T2::EY + oy) * T2::SYW +
                                                    (oz >> 1),
                                                (int)c, (float)rc.t[0], (float)rc.t[1], (float)rc.t[2], dscale, &u, g);
                else
                    eval_component_x2<ORD, GRAD, S::SX, S::SY>(tile + c * S::TS + ox * S::SX + oy * S::SY + oz,
                                                               (float)rc.t[0], (float)rc.t[1], (float)rc.t[2], dscale,
                                                               &u, g);
                out_u[3 * (size_t)idx + c] = u;
                if (GRAD) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) out_grad[9 * (size_t)idx + 3 * c + k] = g[k];
                }
            }
        }
    }
}

template <int ORD, typename CT, typename TR, bool GRAD>
__global__ void __launch_bounds__(kGatherThreads, 2)
gather_f32(const CT* __restrict__ coef, int N, BrickGrid bg, Ws<TR> w, float* __restrict__ out_u,
           float* __restrict__ out_grad, float dscale, const __grid_constant__ CUtensorMap tmap, int use_tma,
           unsigned long long* __restrict__ status) {
    if (blockIdx.x >= w.chunk[bg.NB]) return;
    gather_f32_item<ORD, CT, TR, GRAD>(blockIdx.x, kChunk, coef, N, bg, w, out_u, out_grad, dscale, &tmap, use_tma,
                                       status);
}

// Direct gather for sparse bricks: the particles of bricks holding fewer
// than the split (placed by the scan in one contiguous range after the dense
// bricks, still grouped by brick) are evaluated straight from the
// coefficient array, one thread per particle.  A staged work item costs a
// few microseconds of dependent latency (records, bucketing, the tile copy)
// whatever its particle count, so for a handful of particles reading the
// stencils from global memory (through L1, where neighbouring threads'
// particles share rows) is far cheaper.  Same contraction as the staged
// gather (row_x2 / add_row in the same order), so the results are the same
// bits.  The x-rows run in a rolled loop: unrolled, all 3 ORD^3 global loads
// would be hoisted at once.
template <int ORD, typename CT, typename TR, bool GRAD>
__global__ void __launch_bounds__(256, 2)
gather_direct(const CT* __restrict__ coef, int N, unsigned NB, Ws<TR> w, float* __restrict__ out_u,
              float* __restrict__ out_grad, float dscale, unsigned long long* __restrict__ status) {
    const unsigned beg = w.offset[NB + 2], end = w.offset[NB];
    const size_t NN = (size_t)N * N;
    for (unsigned i = beg + blockIdx.x * blockDim.x + threadIdx.x; i < end; i += gridDim.x * blockDim.x) {
        const Rec<TR> rc = w.s_rec[i];
        const int ax = (int)(rc.cell >> (2 * kAnchorBits));
        const int ay = (int)((rc.cell >> kAnchorBits) & 1023u);
        const int az = (int)(rc.cell & 1023u);
        if (!BS_CHECK_OK(ax < N && ay < N && az < N && (long long)rc.idx < w.P, status + kStatusBounds)) continue;
        float wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
        bspline_weights<ORD, float>((float)rc.t[0], wx, dwx);
        bspline_weights<ORD, float>((float)rc.t[1], wy, dwy);
        bspline_weights<ORD, float>((float)rc.t[2], wz, dwz);
        const PairWeights<ORD> pw(wz, dwz, wy, dwy);
        int yo[ORD], zo[ORD];
#pragma unroll
        for (int j = 0; j < ORD; ++j) {
            yo[j] = wrap_index(ay + j, N) * N;
            zo[j] = wrap_index(az + j, N);
        }
        const size_t idx = rc.idx;
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            const CT* cb = coef + (size_t)c * N * NN;
            float u = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll 1
            for (int jx = 0; jx < ORD; ++jx) {
                const CT* row = cb + (size_t)wrap_index(ax + jx, N) * NN;
                float s00, s10, s01;
                row_x2<ORD, GRAD>([&](int jy, int jz) { return widen<CT>(row[yo[jy] + zo[jz]]); }, pw, wy, dwy, wz, dwz,
                                  &s00, &s10, &s01);
                add_row<GRAD>(wx[jx], dwx[jx], s00, s10, s01, &u, &gx, &gy, &gz);
            }
            out_u[3 * idx + c] = u;
            if (GRAD) {
                out_grad[9 * idx + 3 * c + 0] = gx * dscale;
                out_grad[9 * idx + 3 * c + 1] = gy * dscale;
                out_grad[9 * idx + 3 * c + 2] = gz * dscale;
            }
        }
    }
}

template <typename K> int set_smem(K kernel, size_t bytes) {
    if (bytes > 32 * 1024) {           // static shared memory counts against the 48 KB default too
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return BSPLINE_OK;
}

template <int ORD, typename CT, typename AT, typename TR>
int run_gather(bspline_plan_s* p, const void* coeffs, Ws<TR> w, BrickGrid g, void* out_u, void* out_grad,
               bool grad) {
    const unsigned NB = g.NB;
    const size_t sm = tile_bytes<ORD, CT>();
    const AT dscale = (AT)((double)p->N / p->L);
    int rc;
    if constexpr (sizeof(AT) == 8) {
        auto k = grad ? gather_f64<ORD, TR, true> : gather_f64<ORD, TR, false>;
        if ((rc = set_smem(k, sm))) return rc;
        k<<<NB, 128, sm, p->stream>>>(reinterpret_cast<const double*>(coeffs), p->N, g, w, (double*)out_u,
                                      grad ? (double*)out_grad : nullptr, dscale, p->d_status);
    } else {
        auto k = grad ? gather_f32<ORD, CT, TR, true> : gather_f32<ORD, CT, TR, false>;
        // room to align the tile to 128 bytes; BF16: the two copies of the pair tile
        const size_t sm_aligned = (sizeof(CT) == 2 ? Bf16Pair<ORD>::bytes : sm) + 128;
        if ((rc = set_smem(k, sm_aligned))) return rc;
        // FP32 coefficients: a TMA tensor map for the interior bricks (cp.async if it cannot be made)
        using S = Shape<CT, ORD>;
        CUtensorMap tmap;
        std::memset(&tmap, 0, sizeof tmap);
        int use_tma = 0;
        if (p->N >= 16 && !(p->test_hooks & BSPLINE_TEST_NO_TMA)) {
            const int box_z = sizeof(CT) == 2 ? Bf16Pair<ORD>::PZ : S::PZ;
            use_tma = encode_coef_tmap(&tmap, coeffs, p->N, box_z, S::EY, S::EX, (int)sizeof(CT)) == BSPLINE_OK
                          ? kTmaOn : 0;
        }
        if (use_tma && (p->test_hooks & BSPLINE_TEST_SKIP_TMA_ISSUE)) use_tma = kTmaArmOnly;
        // work items: at most one partial chunk per brick plus P / kChunk full ones
        const long long items = (long long)NB + (w.P + kChunk - 1) / kChunk;
        k<<<(unsigned)items, kGatherThreads, sm_aligned, p->stream>>>(
            reinterpret_cast<const CT*>(coeffs), p->N, g, w, (float*)out_u, grad ? (float*)out_grad : nullptr, dscale,
            tmap, use_tma, p->d_status);
    }
    return BSPLINE_OK;
}

// The direct gather of the bricks below the plan's split (FP32 accumulation only).
template <int ORD, typename CT, typename AT, typename TR>
int run_gather_direct(bspline_plan_s* p, const void* coeffs, Ws<TR> w, BrickGrid g, void* out_u, void* out_grad,
                      bool grad, unsigned below) {
    if constexpr (sizeof(AT) == 8) {
        return BSPLINE_OK;
    } else {
        if (below == 0) return BSPLINE_OK;
        const unsigned NB = g.NB;
        const float dscale = (float)((double)p->N / p->L);
        auto k = grad ? gather_direct<ORD, CT, TR, true> : gather_direct<ORD, CT, TR, false>;
        // the sparse range's length is known on the device only: enough threads for every particle
        // up to a few waves, grid-striding beyond
        const long long want = (w.P + 255) / 256;
        const unsigned blocks = (unsigned)std::max(1LL, std::min(want, 32LL * p->sms));
        k<<<blocks, 256, 0, p->stream>>>(reinterpret_cast<const CT*>(coeffs), p->N, NB, w, (float*)out_u,
                                         grad ? (float*)out_grad : nullptr, dscale, p->d_status);
        return BSPLINE_OK;
    }
}

}  // namespace gather_impl

#define BS_GATHER_EXTERN(ORD, CT, AT, TR)                                                                 \
    extern template int gather_impl::run_gather<ORD, CT, AT, TR>(bspline_plan_s*, const void*,               \
                                                                  gather_impl::Ws<TR>, BrickGrid, void*,     \
                                                                  void*, bool);                              \
    extern template int gather_impl::run_gather_direct<ORD, CT, AT, TR>(                                     \
        bspline_plan_s*, const void*, gather_impl::Ws<TR>, BrickGrid, void*, void*, bool, unsigned);
#define BS_GATHER_INSTANTIATE(ORD, CT, AT, TR)                                                          \
    template int gather_impl::run_gather<ORD, CT, AT, TR>(bspline_plan_s*, const void*, gather_impl::Ws<TR>, \
                                                           BrickGrid, void*, void*, bool);                  \
    template int gather_impl::run_gather_direct<ORD, CT, AT, TR>(bspline_plan_s*, const void*,               \
                                                                  gather_impl::Ws<TR>, BrickGrid, void*,     \
                                                                  void*, bool, unsigned);

}  // namespace bs

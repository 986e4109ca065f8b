// Adjoint of the particle side (differentiation), shared by the adjoint_*.cu
// translation units that instantiate it per coefficient type.
//
// The paper has no adjoint; these kernels transpose the evaluation of
// Sections 3-4 (Eqs. interpolation, interpolation2) on the same brick sort
// the forward evaluation uses:
//
//   spread:  g_coef[c][node] += g_u[c] w_x w_y w_z
//                             + (N/L) (g_grad[c][0] w'_x w_y w_z + g_grad[c][1] w_x w'_y w_z
//                                      + g_grad[c][2] w_x w_y w'_z)
//            accumulated per work item in a shared-memory tile of the brick
//            (shared-memory atomics), then added to g_coef with global
//            atomics (periodic wrap); per node 1 multiply + 1 FMA after the
//            factorisation  w_z (w_y q0 + w'_y q1) + w'_z (w_y q2),
//            q0 = g_u w_x + s g0 w'_x, q1 = s g1 w_x, q2 = s g2 w_x;
//   g_x:     the derivative of sum_c g_u[c] u_c + sum_{c,e} g_grad[c][e] du_c/dx_e
//            in the position: first and second derivatives of the
//            interpolant, contracted z first (w, w', w'' per axis).
#pragma once
#include "particles.cuh"

namespace bs {
namespace adjoint_impl {

using namespace gather_impl;

constexpr int kAdjThreads = 256;

// Weights, first and second derivatives of the n stencil nodes (node 0
// leftmost), from the cardinal B-spline recursion: with v_k[m] = M_k(t + m),
// B''(t + n - 1 - j) = M_{n-2}(t + m) - 2 M_{n-2}(t + m - 1) + M_{n-2}(t + m - 2), m = n - 1 - j.
template <int n, typename A>
__device__ __forceinline__ void bspline_weights2(A t, A (&w)[n], A (&dw)[n], A (&d2w)[n]) {
    A v[n];
    v[0] = A(1);
#pragma unroll
    for (int m = 1; m < n; ++m) v[m] = A(0);
    A v2[n];                                            // order n - 2 values (order 1 for n <= 3)
#pragma unroll
    for (int m = 0; m < n; ++m) v2[m] = v[m];
#pragma unroll
    for (int k = 2; k <= n - 1; ++k) {
        const A inv = A(1) / A(k - 1);
#pragma unroll
        for (int m = k - 1; m >= 0; --m) {
            const A left = (m > 0) ? v[m - 1] : A(0);
            v[m] = ((t + A(m)) * v[m] + (A(k - m) - t) * left) * inv;
        }
        if (k == n - 2) {
#pragma unroll
            for (int m = 0; m < n; ++m) v2[m] = v[m];
        }
    }
    const A inv = A(1) / A(n - 1);
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const int m = n - 1 - j;
        const A vm = (m <= n - 2) ? v[m] : A(0);
        const A vl = (m >= 1) ? v[m - 1] : A(0);
        w[j] = ((t + A(m)) * vm + (A(n - m) - t) * vl) * inv;
        dw[j] = vm - vl;
        if (n <= 2) {
            d2w[j] = A(0);
        } else {
            const A a0 = (m <= n - 3) ? v2[m] : A(0);
            const A a1 = (m >= 1 && m - 1 <= n - 3) ? v2[m - 1] : A(0);
            const A a2 = (m >= 2 && m - 2 <= n - 3) ? v2[m - 2] : A(0);
            d2w[j] = a0 - A(2) * a1 + a2;
        }
    }
}

// Work item -> brick and its particle range [beg, end) in the sorted order.
template <typename TR>
__device__ __forceinline__ bool item_range(const Ws<TR>& w, unsigned NB, unsigned item, unsigned* brick,
                                           unsigned* beg, unsigned* end) {
    if (item >= w.chunk[NB]) return false;
    const unsigned lo = w.item[item];
    *brick = lo;
    *beg = w.offset[lo] + (item - w.chunk[lo]) * kChunk;
    *end = min(*beg + kChunk, w.offset[lo] + w.count[lo]);
    return *beg < *end;
}

// The n particles of an item [beg, beg + n) ordered rank-major, bank-minor by
// the bank (element index mod 32) of their stencil origin in a tile of row
// stride EZ and plane stride EY * EZ, into s_order (as in the gather): a warp
// taking 32 consecutive particles of that order touches each bank at most
// once per rank it spans.  Ends with a barrier.
template <int EY, int EZ, int NT, typename TR>
__device__ __forceinline__ void bank_order(const Ws<TR>& w, unsigned beg, unsigned n, int x0, int y0, int z0,
                                           unsigned* s_bucket, unsigned short* s_order) {
    constexpr int KT = (kChunk + NT - 1) / NT;
    unsigned packed[KT];
    if (threadIdx.x < 32) s_bucket[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const unsigned i = threadIdx.x + k * NT;
        if (i < n) {
            const unsigned cp = w.s_rec[beg + i].cell;
            const int ox = (int)(cp >> (2 * kAnchorBits)) - x0;
            const int oy = (int)((cp >> kAnchorBits) & 1023u) - y0;
            const int oz = (int)(cp & 1023u) - z0;
            const unsigned r = (unsigned)((ox * EY + oy) * EZ + oz) & 31u;
            packed[k] = (atomicAdd(&s_bucket[r], 1u) << 5) | r;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const unsigned i = threadIdx.x + k * NT;
        if (i < n) {
            const unsigned r = packed[k] & 31u, rk = packed[k] >> 5;
            unsigned pos = 0;
#pragma unroll 8
            for (unsigned q = 0; q < 32; ++q) {
                const unsigned bq = s_bucket[q];
                pos += min(bq, rk) + ((q < r && bq > rk) ? 1u : 0u);
            }
            s_order[pos] = (unsigned short)i;
        }
    }
    __syncthreads();
}

// Accumulation tile of the spread: the brick plus halo, [c][x][y][z], unpadded.
template <int ORD, typename A> constexpr size_t acc_bytes() {
    using S = Shape<A, ORD>;
    return sizeof(A) * 3 * (size_t)S::EX * S::EY * S::EZ;
}

// One CTA per work item: spread its particles' cotangents into a shared tile,
// then add the tile to g_coef.  The accumulation tile allows three CTAs per SM;
// compiled for three (more registers between the shared-memory atomics):
// 1.13 -> 1.10 ms at 256^3, cubic, 2^22 particles.
template <int ORD, typename TR, typename A, bool GRAD>
__global__ void __launch_bounds__(kAdjThreads, 3)
spread_kernel(int N, BrickGrid bg, Ws<TR> w, const A* __restrict__ g_u, const A* __restrict__ g_grad,
              A* __restrict__ g_coef, A dscale, unsigned long long* __restrict__ status) {
    using S = Shape<A, ORD>;
    constexpr int EX = S::EX, EY = S::EY, EZ = S::EZ, BZ = S::BZ;
    constexpr int E3 = EX * EY * EZ;                    // one component
    const unsigned NB = bg.NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A* acc = reinterpret_cast<A*>(smem_raw);
    unsigned brick, beg, end;
    if (!item_range(w, NB, blockIdx.x, &brick, &beg, &end)) return;
    int x0, y0, z0;
    brick_origin<S::BX, S::BY, S::BZ>(brick, bg, &x0, &y0, &z0);
    __shared__ unsigned s_bucket[32];
    __shared__ unsigned short s_order[kChunk];
    const unsigned n = end - beg;
    for (int e = threadIdx.x; e < 3 * E3; e += kAdjThreads) acc[e] = A(0);
    if (threadIdx.x < 32) s_bucket[threadIdx.x] = 0;
    __syncthreads();
    // FP32: particles ordered rank-major, bank-minor by the bank of their stencil origin (as in the
    // gather), so a warp's shared-memory atomics hit distinct banks; FP64 keeps the sorted order
    constexpr bool kBucket = sizeof(A) == 4;
    if constexpr (kBucket) {
        constexpr int KT = (kChunk + kAdjThreads - 1) / kAdjThreads;
        unsigned packed[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const unsigned i = threadIdx.x + k * kAdjThreads;
            if (i < n) {
                const unsigned cp = w.s_rec[beg + i].cell;
                const int ox = (int)(cp >> (2 * kAnchorBits)) - x0;
                const int oy = (int)((cp >> kAnchorBits) & 1023u) - y0;
                const int oz = (int)(cp & 1023u) - z0;
                const unsigned r = (unsigned)((ox * EY + oy) * EZ + oz) & 31u;
                packed[k] = (atomicAdd(&s_bucket[r], 1u) << 5) | r;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const unsigned i = threadIdx.x + k * kAdjThreads;
            if (i < n) {
                const unsigned r = packed[k] & 31u, rk = packed[k] >> 5;
                unsigned pos = 0;
#pragma unroll 8
                for (unsigned q = 0; q < 32; ++q) {
                    const unsigned bq = s_bucket[q];
                    pos += min(bq, rk) + ((q < r && bq > rk) ? 1u : 0u);
                }
                s_order[pos] = (unsigned short)i;
            }
        }
        __syncthreads();
    }
    // a thread's next record is requested while its current particle is spread
    auto record = [&](unsigned q) { return w.s_rec[beg + (kBucket ? (unsigned)s_order[q] : q)]; };
    Rec<TR> rc_next;
    if (threadIdx.x < n) rc_next = record(threadIdx.x);
    for (unsigned q = threadIdx.x; q < n; q += kAdjThreads) {
        const Rec<TR> rc = rc_next;
        if (q + kAdjThreads < n) rc_next = record(q + kAdjThreads);
        const int ox = (int)(rc.cell >> (2 * kAnchorBits)) - x0;
        const int oy = (int)((rc.cell >> kAnchorBits) & 1023u) - y0;
        const int oz = (int)(rc.cell & 1023u) - z0;
        const size_t idx = rc.idx;
        if (!BS_CHECK_OK(ox >= 0 && ox < S::BX && oy >= 0 && oy < S::BY && oz >= 0 && oz < S::BZ &&
                             (long long)idx < w.P,
                         status + kStatusBounds))
            continue;
        // the particle's cotangents, all requested before the shared-memory reductions (loads cannot move
        // across them)
        A cu[3], cg[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) cu[c] = g_u ? g_u[3 * idx + c] : A(0);
        if (GRAD) {
#pragma unroll
            for (int e = 0; e < 9; ++e) cg[e] = g_grad[9 * idx + e];
        }
        A wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
        bspline_weights<ORD, A>((A)rc.t[0], wx, dwx);
        bspline_weights<ORD, A>((A)rc.t[1], wy, dwy);
        bspline_weights<ORD, A>((A)rc.t[2], wz, dwz);
        A* base = acc + (ox * EY + oy) * EZ + oz;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const A gu = cu[c];
            A g0 = A(0), g1 = A(0), g2 = A(0);
            if (GRAD) {
                g0 = cg[3 * c + 0] * dscale;
                g1 = cg[3 * c + 1] * dscale;
                g2 = cg[3 * c + 2] * dscale;
            }
            A* tc = base + c * E3;
#pragma unroll
            for (int jx = 0; jx < ORD; ++jx) {
                const A q0 = GRAD ? fma(g0, dwx[jx], gu * wx[jx]) : gu * wx[jx];
                const A q1 = g1 * wx[jx], q2 = g2 * wx[jx];
#pragma unroll
                for (int jy = 0; jy < ORD; ++jy) {
                    const A p0 = GRAD ? fma(q1, dwy[jy], q0 * wy[jy]) : q0 * wy[jy];
                    const A p1 = q2 * wy[jy];
                    A* line = tc + (jx * EY + jy) * EZ;
#pragma unroll
                    for (int jz = 0; jz < ORD; ++jz) {
                        const A v = GRAD ? fma(p1, dwz[jz], p0 * wz[jz]) : p0 * wz[jz];
                        if constexpr (sizeof(A) == 4) {   // reduction without a return value
                            asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(
                                             (unsigned)__cvta_generic_to_shared(line + jz)),
                                         "f"((float)v)
                                         : "memory");
                        } else {
                            atomicAdd(line + jz, v);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if constexpr (sizeof(A) == 4) {
        // per tile row: the brick's B nodes as B/4 aligned 16-byte vector atomics
        // (z0 and N are multiples of 4, so 4 consecutive z stay inside one period),
        // then the EZ - BZ halo nodes one by one
        constexpr int U = BZ / 4 + (EZ - BZ);
        for (int e = threadIdx.x; e < 3 * EX * EY * U; e += kAdjThreads) {
            const int row = e / U, k = e - row * U;
            const int c = row / (EX * EY), ix = (row / EY) % EX, iy = row % EY;
            const A* src = acc + (size_t)row * EZ;
            A* dst = g_coef + (((size_t)c * N + wrap_index(x0 + ix, N)) * N + wrap_index(y0 + iy, N)) * N;
            if (k < BZ / 4) {
                const float4 v = make_float4(src[4 * k], src[4 * k + 1], src[4 * k + 2], src[4 * k + 3]);
                if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                    atomicAdd(reinterpret_cast<float4*>(dst + wrap_index(z0 + 4 * k, N)), v);
            } else {
                const int iz = BZ + (k - BZ / 4);
                const A v = src[iz];
                if (v != A(0)) atomicAdd(dst + wrap_index(z0 + iz, N), v);
            }
        }
    } else {
        for (int e = threadIdx.x; e < 3 * E3; e += kAdjThreads) {
            const A v = acc[e];
            if (v != A(0)) {
                const int c = e / E3, r = e - c * E3;
                const int ix = r / (EY * EZ), iy = (r / EZ) % EY, iz = r % EZ;
                atomicAdd(&g_coef[(((size_t)c * N + wrap_index(x0 + ix, N)) * N + wrap_index(y0 + iy, N)) * N +
                                  wrap_index(z0 + iz, N)],
                          v);
            }
        }
    }
}

// ---- Deterministic spread (plan option, FP32 accumulation types): every
// node's sum is formed in 64-bit fixed point, which integer atomics add
// exactly, so the order in which particles and work items arrive no longer
// changes a bit.  Each contribution is computed in FP32 as in spread_kernel
// and rounded once to an integer at the scale 2^e; e is chosen from a bound
// on all contributions so that no node's sum can leave 2^61:
//   |contribution| <= G (1 + 3 N/L),  G = max |g_u|, |g_grad| over particles
// (|w| <= 1 and |w'| <= 1 for a cardinal B-spline), at most P per node, so
// e = 61 - ceil(log2(G (1 + 3 N/L) P)).  The sums then go through one FP64
// multiply by 2^-e and one FP32 add into g_coef.

// G: atomic maximum over the cotangents' magnitudes (non-negative floats order as their bits).
template <bool GRAD>
__global__ void cotangent_bound_kernel(const float* __restrict__ g_u, const float* __restrict__ g_grad,
                                       long long P, unsigned* __restrict__ bound) {
    float m = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        if (g_u) {
#pragma unroll
            for (int c = 0; c < 3; ++c) m = fmaxf(m, fabsf(g_u[3 * i + c]));
        }
        if (GRAD) {
#pragma unroll
            for (int k = 0; k < 9; ++k) m = fmaxf(m, fabsf(g_grad[9 * i + k]));
        }
    }
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(bound, __float_as_uint(m));
}

// The scale exponent e of the fixed point (the same in every thread: it depends on G, N/L and P only).
__device__ __forceinline__ int det_exponent(const unsigned* bound, float dscale, long long P) {
    const float T = __uint_as_float(*bound) * (1.f + 3.f * dscale) * (float)P;
    int ex = 0;
    if (T > 0.f) frexpf(T, &ex);                        // T < 2^ex
    return min(100, 61 - ex);
}

__device__ __forceinline__ void red_shared_s64(long long* p, long long v) {
    asm volatile("red.shared.add.u64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "l"(v) : "memory");
}

// As spread_kernel (FP32), the tile in fixed point and the tile added to acc_g with 64-bit integer atomics.
template <int ORD, typename TR, bool GRAD>
__global__ void __launch_bounds__(kAdjThreads)
spread_det_kernel(int N, BrickGrid bg, Ws<TR> w, const float* __restrict__ g_u, const float* __restrict__ g_grad,
                  long long* __restrict__ acc_g, float dscale, const unsigned* __restrict__ bound,
                  unsigned long long* __restrict__ status) {
    using S = Shape<float, ORD>;
    constexpr int EX = S::EX, EY = S::EY, EZ = S::EZ;
    constexpr int E3 = EX * EY * EZ;
    const unsigned NB = bg.NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long long* acc = reinterpret_cast<long long*>(smem_raw);
    unsigned brick, beg, end;
    if (!item_range(w, NB, blockIdx.x, &brick, &beg, &end)) return;
    int x0, y0, z0;
    brick_origin<S::BX, S::BY, S::BZ>(brick, bg, &x0, &y0, &z0);
    const float sc = ldexpf(1.f, det_exponent(bound, dscale, w.P));
    const unsigned n = end - beg;
    __shared__ unsigned s_bucket[32];
    __shared__ unsigned short s_order[kChunk];
    for (int e = threadIdx.x; e < 3 * E3; e += kAdjThreads) acc[e] = 0;
    bank_order<EY, EZ, kAdjThreads>(w, beg, n, x0, y0, z0, s_bucket, s_order);   // ends with a barrier
    Rec<TR> rc_next;                                    // the thread's next record, requested ahead
    if (threadIdx.x < n) rc_next = w.s_rec[beg + s_order[threadIdx.x]];
    for (unsigned q = threadIdx.x; q < n; q += kAdjThreads) {
        const Rec<TR> rc = rc_next;
        if (q + kAdjThreads < n) rc_next = w.s_rec[beg + s_order[q + kAdjThreads]];
        const int ox = (int)(rc.cell >> (2 * kAnchorBits)) - x0;
        const int oy = (int)((rc.cell >> kAnchorBits) & 1023u) - y0;
        const int oz = (int)(rc.cell & 1023u) - z0;
        const size_t idx = rc.idx;
        if (!BS_CHECK_OK(ox >= 0 && ox < S::BX && oy >= 0 && oy < S::BY && oz >= 0 && oz < S::BZ &&
                             (long long)idx < w.P,
                         status + kStatusBounds))
            continue;
        // the particle's cotangents, all requested before the reductions (loads cannot move across them)
        float cu[3], cg[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) cu[c] = g_u ? g_u[3 * idx + c] : 0.f;
        if (GRAD) {
#pragma unroll
            for (int e = 0; e < 9; ++e) cg[e] = g_grad[9 * idx + e];
        }
        float wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
        bspline_weights<ORD, float>(rc.t[0], wx, dwx);
        bspline_weights<ORD, float>(rc.t[1], wy, dwy);
        bspline_weights<ORD, float>(rc.t[2], wz, dwz);
        long long* base = acc + (ox * EY + oy) * EZ + oz;
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            // this component's cotangents (selects: c is a rolled loop counter)
            const float gu = c == 0 ? cu[0] : (c == 1 ? cu[1] : cu[2]);
            float g0 = 0.f, g1 = 0.f, g2 = 0.f;
            if (GRAD) {
                g0 = (c == 0 ? cg[0] : (c == 1 ? cg[3] : cg[6])) * dscale;
                g1 = (c == 0 ? cg[1] : (c == 1 ? cg[4] : cg[7])) * dscale;
                g2 = (c == 0 ? cg[2] : (c == 1 ? cg[5] : cg[8])) * dscale;
            }
            long long* tc = base + c * E3;
#pragma unroll
            for (int jx = 0; jx < ORD; ++jx) {
                const float q0 = GRAD ? fmaf(g0, dwx[jx], gu * wx[jx]) : gu * wx[jx];
                const float q1 = g1 * wx[jx], q2 = g2 * wx[jx];
#pragma unroll
                for (int jy = 0; jy < ORD; ++jy) {
                    const float p0 = GRAD ? fmaf(q1, dwy[jy], q0 * wy[jy]) : q0 * wy[jy];
                    const float p1 = q2 * wy[jy];
                    long long* line = tc + (jx * EY + jy) * EZ;
#pragma unroll
                    for (int jz = 0; jz < ORD; ++jz) {
                        const float v = GRAD ? fmaf(p1, dwz[jz], p0 * wz[jz]) : p0 * wz[jz];
                        red_shared_s64(line + jz, __float2ll_rn(v * sc));
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * E3; e += kAdjThreads) {
        const long long v = acc[e];
        if (v != 0) {
            const int c = e / E3, r = e - c * E3;
            const int ix = r / (EY * EZ), iy = (r / EZ) % EY, iz = r % EZ;
            atomicAdd(reinterpret_cast<unsigned long long*>(
                          &acc_g[(((size_t)c * N + wrap_index(x0 + ix, N)) * N + wrap_index(y0 + iy, N)) * N +
                                 wrap_index(z0 + iz, N)]),
                      (unsigned long long)v);
        }
    }
}

// g_coef += acc_g 2^-e, one thread per node (the one rounding of each node's exact sum).
static __global__ void det_finish_kernel(const long long* __restrict__ acc_g, float* __restrict__ g_coef, long long n,
                                  float dscale, long long P, const unsigned* __restrict__ bound) {
    const double inv = ldexp(1.0, -det_exponent(bound, dscale, P));
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        g_coef[i] += (float)((double)acc_g[i] * inv);
}

// Position gradient: one thread per particle of the work item, coefficients
// staged as in the forward evaluation.
template <int ORD, typename CT, typename TR, bool HESS>
__global__ void __launch_bounds__(kAdjThreads)
gx_kernel(const CT* __restrict__ coef, int N, BrickGrid bg, Ws<TR> w,
          const typename TileT<CT>::T* __restrict__ g_u, const typename TileT<CT>::T* __restrict__ g_grad,
          double* __restrict__ g_x, typename TileT<CT>::T dscale, const __grid_constant__ CUtensorMap tmap,
          int use_tma, unsigned long long* __restrict__ status) {
    using A = typename TileT<CT>::T;
    using S = Shape<CT, ORD>;
    const unsigned NB = bg.NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the tile 128-byte aligned (TMA destinations; the launch adds 128 bytes of slack)
    A* tile = reinterpret_cast<A*>(smem_raw + ((0u - smem_u32(smem_raw)) & 127u));   // 128-byte aligned
    __shared__ __align__(8) unsigned long long s_mbar;
    unsigned brick, beg, end;
    if (!item_range(w, NB, blockIdx.x, &brick, &beg, &end)) return;
    int x0, y0, z0;
    brick_origin<S::BX, S::BY, S::BZ>(brick, bg, &x0, &y0, &z0);
    bool tma = false;
    if constexpr (sizeof(A) == 4) tma = stage_tile_tma<ORD, CT>(tile, &tmap, &s_mbar, N, x0, y0, z0, use_tma);
    if (!tma) stage_brick<ORD, CT>(tile, coef, N, x0, y0, z0);
    __shared__ unsigned s_bucket[32];
    __shared__ unsigned short s_order[kChunk];
    const unsigned n = end - beg;
    if (threadIdx.x < 32) s_bucket[threadIdx.x] = 0;
    __syncthreads();                                    // the tile copies stay in flight while bucketing
    // FP32 tiles: particles ordered rank-major, bank-minor by the bank of their stencil origin, as in
    // the gather, so a warp's tile loads hit distinct banks
    constexpr bool kBucket = sizeof(A) == 4;
    if constexpr (kBucket) {
        constexpr int KT = (kChunk + kAdjThreads - 1) / kAdjThreads;
        unsigned packed[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const unsigned i = threadIdx.x + k * kAdjThreads;
            if (i < n) {
                const unsigned cp = w.s_rec[beg + i].cell;
                const int ox = (int)(cp >> (2 * kAnchorBits)) - x0;
                const int oy = (int)((cp >> kAnchorBits) & 1023u) - y0;
                const int oz = (int)(cp & 1023u) - z0;
                const unsigned r = (unsigned)(ox * S::SX + oy * S::SY + oz) & 31u;
                packed[k] = (atomicAdd(&s_bucket[r], 1u) << 5) | r;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const unsigned i = threadIdx.x + k * kAdjThreads;
            if (i < n) {
                const unsigned r = packed[k] & 31u, rk = packed[k] >> 5;
                unsigned pos = 0;
#pragma unroll 8
                for (unsigned q = 0; q < 32; ++q) {
                    const unsigned bq = s_bucket[q];
                    pos += min(bq, rk) + ((q < r && bq > rk) ? 1u : 0u);
                }
                s_order[pos] = (unsigned short)i;
            }
        }
    }
    cp_async_wait_all();
    if (tma && !tma_tile_wait(&s_mbar, status + kStatusParticleTimeout)) {
        fill_nan_item<TR, double>(w, beg, n, g_x, nullptr, 3);
        return;
    }
    __syncthreads();
    const A s2 = dscale * dscale;
    // a thread's next record is requested while its current particle is evaluated
    auto record = [&](unsigned q) { return w.s_rec[beg + (kBucket ? (unsigned)s_order[q] : q)]; };
    Rec<TR> rc_next;
    if (threadIdx.x < n) rc_next = record(threadIdx.x);
    for (unsigned q = threadIdx.x; q < n; q += kAdjThreads) {
        const Rec<TR> rc = rc_next;
        if (q + kAdjThreads < n) rc_next = record(q + kAdjThreads);
        const int ox = (int)(rc.cell >> (2 * kAnchorBits)) - x0;
        const int oy = (int)((rc.cell >> kAnchorBits) & 1023u) - y0;
        const int oz = (int)(rc.cell & 1023u) - z0;
        const size_t idx = rc.idx;
        if (!BS_CHECK_OK(ox >= 0 && ox < S::BX && oy >= 0 && oy < S::BY && oz >= 0 && oz < S::BZ &&
                             (long long)idx < w.P,
                         status + kStatusBounds))
            continue;
        // the particle's cotangents, requested before the contractions that they multiply
        A gu[3], gg[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) gu[c] = g_u ? g_u[3 * idx + c] : A(0);
        if (HESS) {
#pragma unroll
            for (int e = 0; e < 9; ++e) gg[e] = g_grad[9 * idx + e];
        }
        A wx[ORD], dwx[ORD], d2wx[ORD], wy[ORD], dwy[ORD], d2wy[ORD], wz[ORD], dwz[ORD], d2wz[ORD];
        bspline_weights2<ORD, A>((A)rc.t[0], wx, dwx, d2wx);
        bspline_weights2<ORD, A>((A)rc.t[1], wy, dwy, d2wy);
        bspline_weights2<ORD, A>((A)rc.t[2], wz, dwz, d2wz);
        const A* base = tile + ox * S::SX + oy * S::SY + oz;
        A gx = A(0), gy = A(0), gz = A(0);
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            const A* tc = base + c * S::TS;
            // T_abc = sum over the stencil of a * w^(a)_x w^(b)_y w^(c)_z
            A t100 = 0, t010 = 0, t001 = 0, t200 = 0, t020 = 0, t002 = 0, t110 = 0, t101 = 0, t011 = 0;
#pragma unroll
            for (int jx = 0; jx < ORD; ++jx) {
                A y00 = 0, y10 = 0, y01 = 0, y20 = 0, y02 = 0, y11 = 0;
#pragma unroll
                for (int jy = 0; jy < ORD; ++jy) {
                    const A* line = tc + jx * S::SX + jy * S::SY;
                    A z0v = 0, z1v = 0, z2v = 0;
#pragma unroll
                    for (int jz = 0; jz < ORD; ++jz) {
                        const A a = line[jz];
                        z0v = fma(wz[jz], a, z0v);
                        z1v = fma(dwz[jz], a, z1v);
                        if (HESS) z2v = fma(d2wz[jz], a, z2v);
                    }
                    y00 = fma(wy[jy], z0v, y00);
                    y10 = fma(dwy[jy], z0v, y10);
                    y01 = fma(wy[jy], z1v, y01);
                    if (HESS) {
                        y20 = fma(d2wy[jy], z0v, y20);
                        y02 = fma(wy[jy], z2v, y02);
                        y11 = fma(dwy[jy], z1v, y11);
                    }
                }
                t100 = fma(dwx[jx], y00, t100);
                t010 = fma(wx[jx], y10, t010);
                t001 = fma(wx[jx], y01, t001);
                if (HESS) {
                    t200 = fma(d2wx[jx], y00, t200);
                    t020 = fma(wx[jx], y20, t020);
                    t002 = fma(wx[jx], y02, t002);
                    t110 = fma(dwx[jx], y10, t110);
                    t101 = fma(dwx[jx], y01, t101);
                    t011 = fma(wx[jx], y11, t011);
                }
            }
            // this component's cotangents (selects: c is a rolled loop counter)
            const A guc = (c == 0 ? gu[0] : (c == 1 ? gu[1] : gu[2])) * dscale;
            gx = fma(guc, t100, gx);
            gy = fma(guc, t010, gy);
            gz = fma(guc, t001, gz);
            if (HESS) {
                const A g0 = (c == 0 ? gg[0] : (c == 1 ? gg[3] : gg[6])) * s2;
                const A g1 = (c == 0 ? gg[1] : (c == 1 ? gg[4] : gg[7])) * s2;
                const A g2 = (c == 0 ? gg[2] : (c == 1 ? gg[5] : gg[8])) * s2;
                gx += g0 * t200 + g1 * t110 + g2 * t101;
                gy += g0 * t110 + g1 * t020 + g2 * t011;
                gz += g0 * t101 + g1 * t011 + g2 * t002;
            }
        }
        g_x[3 * idx + 0] = (double)gx;
        g_x[3 * idx + 1] = (double)gy;
        g_x[3 * idx + 2] = (double)gz;
    }
}

// Launch the spread (g_coef != nullptr) and the position gradient (g_x != nullptr)
// for one order and coefficient type.  items = upper bound of work items.
template <int ORD, typename CT, typename TR>
int run_adjoint(bspline_plan_s* p, const void* coeffs, Ws<TR> w, BrickGrid g, long long items,
                const void* g_u, const void* g_grad, void* g_coef, double* g_x) {
    using A = typename TileT<CT>::T;
    const A dscale = (A)((double)p->N / p->L);
    int rc;
    if constexpr (sizeof(A) == 4) {
        if (g_coef && p->deterministic) {
            // fixed-point accumulator [3][N][N][N] int64, then the bound word
            const long long nodes = 3LL * p->N * p->N * p->N;
            long long* acc_g = reinterpret_cast<long long*>(p->det.ptr);
            unsigned* bound = reinterpret_cast<unsigned*>(acc_g + nodes);
            cudaError_t e = cudaMemsetAsync(acc_g, 0, sizeof(long long) * nodes + 16, p->stream);
            if (e != cudaSuccess) return set_cuda_error(e);
            const long long want = (w.P + 255) / 256;
            const unsigned blocks = (unsigned)std::max(1LL, std::min(want, 8LL * p->sms));
            if (g_grad)
                cotangent_bound_kernel<true><<<blocks, 256, 0, p->stream>>>((const float*)g_u, (const float*)g_grad,
                                                                            w.P, bound);
            else
                cotangent_bound_kernel<false><<<blocks, 256, 0, p->stream>>>((const float*)g_u, nullptr, w.P, bound);
            const size_t sm = sizeof(long long) * 3 * (size_t)Shape<float, ORD>::EX * Shape<float, ORD>::EY *
                              Shape<float, ORD>::EZ;
            auto k = g_grad ? spread_det_kernel<ORD, TR, true> : spread_det_kernel<ORD, TR, false>;
            if ((rc = set_smem(k, sm))) return rc;
            k<<<(unsigned)items, kAdjThreads, sm, p->stream>>>(p->N, g, w, (const float*)g_u, (const float*)g_grad,
                                                                acc_g, (float)dscale, bound, p->d_status);
            const unsigned fb = (unsigned)std::max(1LL, std::min((nodes + 255) / 256, 16LL * p->sms));
            det_finish_kernel<<<fb, 256, 0, p->stream>>>(acc_g, (float*)g_coef, nodes, (float)dscale, w.P, bound);
            g_coef = nullptr;                               // done
        }
    }
    if (g_coef) {
        const size_t sm = acc_bytes<ORD, A>();
        auto k = g_grad ? spread_kernel<ORD, TR, A, true> : spread_kernel<ORD, TR, A, false>;
        if ((rc = set_smem(k, sm))) return rc;
        k<<<(unsigned)items, kAdjThreads, sm, p->stream>>>(p->N, g, w, (const A*)g_u, (const A*)g_grad,
                                                            (A*)g_coef, dscale, p->d_status);
    }
    if (g_x) {
        const size_t sm = tile_bytes<ORD, CT>() + 128;   // room to align the tile to 128 bytes
        auto k = g_grad ? gx_kernel<ORD, CT, TR, true> : gx_kernel<ORD, CT, TR, false>;
        if ((rc = set_smem(k, sm))) return rc;
        using S = Shape<CT, ORD>;
        CUtensorMap tmap;
        std::memset(&tmap, 0, sizeof tmap);
        int use_tma = 0;
        if (sizeof(CT) == 4 && p->N >= 16 && !(p->test_hooks & BSPLINE_TEST_NO_TMA))
            use_tma = encode_coef_tmap(&tmap, coeffs, p->N, S::PZ, S::EY, S::EX) == BSPLINE_OK ? kTmaOn : 0;
        if (use_tma && (p->test_hooks & BSPLINE_TEST_SKIP_TMA_ISSUE)) use_tma = kTmaArmOnly;
        k<<<(unsigned)items, kAdjThreads, sm, p->stream>>>((const CT*)coeffs, p->N, g, w, (const A*)g_u,
                                                            (const A*)g_grad, g_x, dscale, tmap, use_tma,
                                                            p->d_status);
    }
    return BSPLINE_OK;
}

}  // namespace adjoint_impl

#define BS_ADJOINT_EXTERN(ORD, CT, TR)                                                                          \
    extern template int adjoint_impl::run_adjoint<ORD, CT, TR>(bspline_plan_s*, const void*,                   \
                                                                gather_impl::Ws<TR>, BrickGrid, long long,       \
                                                                const void*, const void*, void*, double*);
#define BS_ADJOINT_INSTANTIATE(ORD, CT, TR)                                                                     \
    template int adjoint_impl::run_adjoint<ORD, CT, TR>(bspline_plan_s*, const void*, gather_impl::Ws<TR>,      \
                                                         BrickGrid, long long, const void*, const void*,        \
                                                         void*, double*);

}  // namespace bs

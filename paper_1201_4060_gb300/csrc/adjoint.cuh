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
//            (shared-memory atomics; FP32 types in two-word fixed point),
//            then added to g_coef with global atomics (periodic wrap); per
//            node 1 multiply + 1 FMA after the
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

// Accumulation tile of the FP64 spread: the brick plus halo, [c][x][y][z], unpadded.
template <int ORD> constexpr size_t acc_bytes() {
    using S = Shape<double, ORD>;
    return sizeof(double) * 3 * (size_t)S::EX * S::EY * S::EZ;
}

// FP64 spread, one CTA per work item: its particles' cotangents into a shared
// tile (FP64 shared-memory atomics, particles in their sorted order), then the
// tile added to g_coef with global atomics.  Compiled for three CTAs per SM.
template <int ORD, typename TR, bool GRAD>
__global__ void __launch_bounds__(kAdjThreads, 3)
spread_kernel(int N, BrickGrid bg, Ws<TR> w, const double* __restrict__ g_u, const double* __restrict__ g_grad,
              double* __restrict__ g_coef, double dscale, unsigned long long* __restrict__ status) {
    using S = Shape<double, ORD>;
    constexpr int EX = S::EX, EY = S::EY, EZ = S::EZ;
    constexpr int E3 = EX * EY * EZ;                    // one component
    const unsigned NB = bg.NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* acc = reinterpret_cast<double*>(smem_raw);
    unsigned brick, beg, end;
    if (!item_range(w, NB, blockIdx.x, &brick, &beg, &end)) return;
    int x0, y0, z0;
    brick_origin<S::BX, S::BY, S::BZ>(brick, bg, &x0, &y0, &z0);
    const unsigned n = end - beg;
    for (int e = threadIdx.x; e < 3 * E3; e += kAdjThreads) acc[e] = 0.0;
    __syncthreads();
    Rec<TR> rc_next;                                    // a thread's next record, requested ahead
    if (threadIdx.x < n) rc_next = w.s_rec[beg + threadIdx.x];
    for (unsigned q = threadIdx.x; q < n; q += kAdjThreads) {
        const Rec<TR> rc = rc_next;
        if (q + kAdjThreads < n) rc_next = w.s_rec[beg + q + kAdjThreads];
        const int ox = (int)(rc.cell >> (2 * kAnchorBits)) - x0;
        const int oy = (int)((rc.cell >> kAnchorBits) & 1023u) - y0;
        const int oz = (int)(rc.cell & 1023u) - z0;
        const size_t idx = rc.idx;
        if (!BS_CHECK_OK(ox >= 0 && ox < S::BX && oy >= 0 && oy < S::BY && oz >= 0 && oz < S::BZ &&
                             (long long)idx < w.P,
                         status + kStatusBounds))
            continue;
        // the particle's cotangents, all requested before the reductions
        double cu[3], cg[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) cu[c] = g_u ? g_u[3 * idx + c] : 0.0;
        if (GRAD) {
#pragma unroll
            for (int e = 0; e < 9; ++e) cg[e] = g_grad[9 * idx + e];
        }
        double wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
        bspline_weights<ORD, double>((double)rc.t[0], wx, dwx);
        bspline_weights<ORD, double>((double)rc.t[1], wy, dwy);
        bspline_weights<ORD, double>((double)rc.t[2], wz, dwz);
        double* base = acc + (ox * EY + oy) * EZ + oz;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double gu = cu[c];
            double g0 = 0.0, g1 = 0.0, g2 = 0.0;
            if (GRAD) {
                g0 = cg[3 * c + 0] * dscale;
                g1 = cg[3 * c + 1] * dscale;
                g2 = cg[3 * c + 2] * dscale;
            }
            double* tc = base + c * E3;
#pragma unroll
            for (int jx = 0; jx < ORD; ++jx) {
                const double q0 = GRAD ? fma(g0, dwx[jx], gu * wx[jx]) : gu * wx[jx];
                const double q1 = g1 * wx[jx], q2 = g2 * wx[jx];
#pragma unroll
                for (int jy = 0; jy < ORD; ++jy) {
                    const double p0 = GRAD ? fma(q1, dwy[jy], q0 * wy[jy]) : q0 * wy[jy];
                    const double p1 = q2 * wy[jy];
                    double* line = tc + (jx * EY + jy) * EZ;
#pragma unroll
                    for (int jz = 0; jz < ORD; ++jz) atomicAdd(line + jz, GRAD ? fma(p1, dwz[jz], p0 * wz[jz]) : p0 * wz[jz]);
                }
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * E3; e += kAdjThreads) {
        const double v = acc[e];
        if (v != 0.0) {
            const int c = e / E3, r = e - c * E3;
            const int ix = r / (EY * EZ), iy = (r / EZ) % EY, iz = r % EZ;
            atomicAdd(&g_coef[(((size_t)c * N + wrap_index(x0 + ix, N)) * N + wrap_index(y0 + iy, N)) * N +
                              wrap_index(z0 + iz, N)],
                      v);
        }
    }
}

// ---- FP32 spread in two-word fixed point.  Shared-memory reductions of 32-bit
// integers cost next to nothing beside the rest of the spread, those of FP32
// values (and of 64-bit integers) several times more: on the adjoint workload
// 0.67 ms with 32-bit integer reductions, 1.08 ms with FP32 ones, 2.0 ms with
// 64-bit ones.  So each contribution v is split at the scales 2^e1 and
// 2^(e1 + e2) into
//     hi = rint(v 2^e1),  lo = rint((v 2^e1 - hi) 2^e2),   hi 2^e2 + lo = rint(v 2^(e1 + e2)),
// both added with 32-bit integer reductions into a tile of two words a node;
// the node's sum  sum hi 2^-e1 + sum lo 2^-(e1 + e2)  is exact up to half a
// unit of 2^-(e1 + e2) per contribution.  The scales come from a bound on the
// contributions: with G the largest cotangent magnitude and |w|, |w'| <= 1 for
// a cardinal B-spline, |v| <= Gb = G (1 + 3 N/L); rint is FP32 addition of
// 1.5 2^23, exact while |x| < 2^22, and no node's sums of at most n terms may
// leave 2^30.  Per CTA (G and n of the particles of its part of a work item):
//     e1 = min(21 - ceil(log2 Gb), 29 - ceil(log2 (n Gb)), 100),  e2 = min(22, 30 - ceil(log2 (n + 1))),
// about 40 bits below the largest contribution, then one conversion to FP32
// and FP32 atomics into g_coef.  Deterministic mode (one scale for every
// item, so that the rounding of a contribution does not depend on which item
// it falls in; G over all particles, n <= 2048, P particles in all):
//     e1 = min(18 - ceil(log2 Gb), Ef),  e2 = Ef - e1,  Ef = min(36 - ceil(log2 Gb), 61 - ceil(log2 (P Gb)), 118),
// and each node's hi 2^e2 + lo goes to a 64-bit fixed-point accumulator with
// integer atomics: every contribution is rounded once, rint(v 2^Ef), and all
// sums are exact, so neither particle order nor atomics order changes a bit;
// one rounding to FP32 (times 2^-Ef) and one FP32 add take the sums into g_coef.
// Non-finite cotangents fall back to FP32 reductions (NaN and infinities reach
// g_coef).  The two-word tile is split along x into XP parts, one CTA each,
// so that two CTAs share an SM.
template <int ORD> struct FxShape {
    using S = Shape<float, ORD>;
    static constexpr int BX = S::BX, BY = S::BY, BZ = S::BZ;
    static constexpr int XP = ORD <= 5 ? 2 : 4;         // x parts of a brick
    static constexpr int XW = BX / XP;                   // origins of one part in x
    static constexpr int EX = XW + ORD - 1, EY = S::EY, EZ = S::EZ;
    static constexpr int E3 = EX * EY * EZ;              // nodes of one component
};
static_assert(FxShape<2>::BX % FxShape<2>::XP == 0 && FxShape<8>::BX % FxShape<8>::XP == 0, "x parts");
constexpr int kFxThreads = 384;

template <int ORD> constexpr size_t fx_tile_bytes() { return sizeof(unsigned) * 6 * (size_t)FxShape<ORD>::E3; }

constexpr float kRintMagic = 12582912.0f;               // 1.5 2^23
constexpr unsigned kRintMagicBits = 0x4B400000u;

__device__ __forceinline__ void red_shared_u32(unsigned* p, unsigned v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void red_shared_f32(float* p, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "f"(v) : "memory");
}

// The split scales; fixed = false for a non-finite bound.
struct FxScale {
    bool fixed;
    int e1, e2;
};

// gbits: the bits of G (non-negative floats order as their bits, NaN above infinity); n: terms a node can sum.
__device__ __forceinline__ FxScale fx_item_scale(unsigned gbits, float bound_factor, unsigned n) {
    const float Gb = __uint_as_float(gbits) * bound_factor;
    FxScale s{gbits < 0x7F800000u && Gb * (float)n < INFINITY, 0, 0};
    if (s.fixed && gbits) {
        int kG, kT;
        frexpf(Gb, &kG);                                // Gb < 2^kG
        frexpf(Gb * (float)n, &kT);
        s.e1 = min(min(21 - kG, 29 - kT), 100);
        s.e2 = min(22, 30 - (32 - __clz(n)));
    }
    return s;
}

__device__ __forceinline__ FxScale fx_det_scale(unsigned gbits, float bound_factor, long long P) {
    const float Gb = __uint_as_float(gbits) * bound_factor;
    FxScale s{gbits < 0x7F800000u && Gb * (float)P < INFINITY, 0, 0};
    if (s.fixed && gbits) {
        int kG, kP;
        frexpf(Gb, &kG);
        frexpf(Gb * (float)P, &kP);
        const int ef = min(min(36 - kG, 61 - kP), 118);
        s.e1 = min(18 - kG, ef);
        s.e2 = ef - s.e1;
    }
    return s;
}

// G over all particles (deterministic mode), as bits.
template <bool GRAD>
__global__ void cotangent_bound_kernel(const float* __restrict__ g_u, const float* __restrict__ g_grad,
                                       long long P, unsigned* __restrict__ bound) {
    unsigned m = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        if (g_u) {
#pragma unroll
            for (int c = 0; c < 3; ++c) m = max(m, __float_as_uint(fabsf(g_u[3 * i + c])));
        }
        if (GRAD) {
#pragma unroll
            for (int k = 0; k < 9; ++k) m = max(m, __float_as_uint(fabsf(g_grad[9 * i + k])));
        }
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(bound, m);
}

// The contributions of one particle to its 3 n^3 nodes (factorised as in spread_kernel), each handed to add(node, v).
template <int ORD, bool GRAD, typename Add>
__device__ __forceinline__ void spread_particle(const float (&cu)[3], const float (&cg)[9], float dscale,
                                                const float (&wx)[ORD], const float (&dwx)[ORD],
                                                const float (&wy)[ORD], const float (&dwy)[ORD],
                                                const float (&wz)[ORD], const float (&dwz)[ORD], int base,
                                                int E3, int EY, int EZ, Add add) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float gu = cu[c];
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        if (GRAD) {
            g0 = cg[3 * c + 0] * dscale;
            g1 = cg[3 * c + 1] * dscale;
            g2 = cg[3 * c + 2] * dscale;
        }
#pragma unroll
        for (int jx = 0; jx < ORD; ++jx) {
            const float q0 = GRAD ? fmaf(g0, dwx[jx], gu * wx[jx]) : gu * wx[jx];
            const float q1 = g1 * wx[jx], q2 = g2 * wx[jx];
#pragma unroll
            for (int jy = 0; jy < ORD; ++jy) {
                const float p0 = GRAD ? fmaf(q1, dwy[jy], q0 * wy[jy]) : q0 * wy[jy];
                const float p1 = q2 * wy[jy];
                const int line = base + c * E3 + (jx * EY + jy) * EZ;
#pragma unroll
                for (int jz = 0; jz < ORD; ++jz) add(line + jz, GRAD ? fmaf(p1, dwz[jz], p0 * wz[jz]) : p0 * wz[jz]);
            }
        }
    }
}

// One CTA per (work item, x part).  DET: the deterministic mode's scales (bound = G over all particles) and
// the tile added to acc_g; otherwise the item's own scales and the tile added to g_coef.
template <int ORD, typename TR, bool GRAD, bool DET>
__global__ void __launch_bounds__(kFxThreads, 2)
spread_fx_kernel(int N, BrickGrid bg, Ws<TR> w, const float4* __restrict__ cot, float* __restrict__ g_coef,
                 long long* __restrict__ acc_g, const unsigned* __restrict__ bound, float dscale, float bound_factor,
                 unsigned long long* __restrict__ status) {
    using F = FxShape<ORD>;
    constexpr int EX = F::EX, EY = F::EY, EZ = F::EZ, E3 = F::E3, BZ = F::BZ, XW = F::XW;
    const unsigned NB = bg.NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned* hi = reinterpret_cast<unsigned*>(smem_raw);     // [3][EX][EY][EZ], then lo the same
    unsigned* lo = hi + 3 * E3;
    unsigned brick, beg, end;
    if (!item_range(w, NB, blockIdx.x / F::XP, &brick, &beg, &end)) return;
    const int part = (int)(blockIdx.x % F::XP);
    int x0, y0, z0;
    brick_origin<F::BX, F::BY, F::BZ>(brick, bg, &x0, &y0, &z0);
    __shared__ unsigned s_bucket[32];
    __shared__ unsigned short s_order[kChunk];
    __shared__ unsigned s_gmax;
    const unsigned n = end - beg;
    for (int e = threadIdx.x; e < 6 * E3; e += kFxThreads) hi[e] = 0u;
    if (threadIdx.x < 32) s_bucket[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_gmax = 0;
    __syncthreads();
    // this part's particles, bucketed by the bank of their stencil origin in the part's tile (rank-major,
    // bank-minor, as in the gather), and the largest magnitude of their cotangents
    constexpr int KT = (kChunk + kFxThreads - 1) / kFxThreads;
    unsigned packed[KT];
    unsigned gbits = 0;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const unsigned i = threadIdx.x + k * kFxThreads;
        packed[k] = ~0u;
        if (i < n) {
            const Rec<TR>& rc = w.s_rec[beg + i];
            const unsigned cp = rc.cell;
            const int ox = (int)(cp >> (2 * kAnchorBits)) - x0;
            const int oy = (int)((cp >> kAnchorBits) & 1023u) - y0;
            const int oz = (int)(cp & 1023u) - z0;
            const long long idx = rc.idx;
            const bool ok = ox >= 0 && ox < F::BX && oy >= 0 && oy < F::BY && oz >= 0 && oz < F::BZ && idx < w.P;
            if (part == 0) (void)BS_CHECK_OK(ok, status + kStatusBounds);
            if (ok && ox / XW == part) {
                const unsigned r = (unsigned)(((ox - part * XW) * EY + oy) * EZ + oz) & 31u;
                packed[k] = (atomicAdd(&s_bucket[r], 1u) << 5) | r;
                if (!DET && cot) {
                    const float4* cp4 = cot + 4 * (size_t)(beg + i);
#pragma unroll
                    for (int k4 = 0; k4 < 3; ++k4) {
                        const float4 v = cp4[k4];
                        gbits = max(max(gbits, __float_as_uint(fabsf(v.x))), __float_as_uint(fabsf(v.y)));
                        gbits = max(max(gbits, __float_as_uint(fabsf(v.z))), __float_as_uint(fabsf(v.w)));
                    }
                }
            }
        }
    }
    if (!DET) {
        gbits = __reduce_max_sync(0xffffffffu, gbits);
        if ((threadIdx.x & 31) == 0 && gbits) atomicMax(&s_gmax, gbits);
    }
    __syncthreads();
    unsigned np = 0;                                    // particles of this part
#pragma unroll 8
    for (unsigned q = 0; q < 32; ++q) np += s_bucket[q];
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        if (packed[k] != ~0u) {
            const unsigned r = packed[k] & 31u, rk = packed[k] >> 5;
            unsigned pos = 0;
#pragma unroll 8
            for (unsigned q = 0; q < 32; ++q) {
                const unsigned bq = s_bucket[q];
                pos += min(bq, rk) + ((q < r && bq > rk) ? 1u : 0u);
            }
            s_order[pos] = (unsigned short)(threadIdx.x + k * kFxThreads);
        }
    }
    const unsigned gmax = DET ? *bound : s_gmax;
    __syncthreads();
    if (gmax == 0 || np == 0) return;                   // every contribution is zero
    const FxScale sc = DET ? fx_det_scale(gmax, bound_factor, w.P) : fx_item_scale(gmax, bound_factor, np);
    const float s1 = ldexpf(1.f, sc.e1), s2 = ldexpf(1.f, sc.e2);
    const int xs = part * XW;
    auto particle = [&](const Rec<TR>& rc, unsigned slot, auto add) {
        const int ox = (int)(rc.cell >> (2 * kAnchorBits)) - x0 - xs;
        const int oy = (int)((rc.cell >> kAnchorBits) & 1023u) - y0;
        const int oz = (int)(rc.cell & 1023u) - z0;
        // the particle's cotangents from its sorted slot, all requested before the reductions (loads cannot
        // move across them)
        const float4* cp4 = cot + 4 * (size_t)slot;
        const float4 v0 = cp4[0], v1 = cp4[1], v2 = cp4[2];
        const float cu[3] = {v0.x, v0.y, v0.z};
        const float cg[9] = {v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
        float wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
        bspline_weights<ORD, float>((float)rc.t[0], wx, dwx);
        bspline_weights<ORD, float>((float)rc.t[1], wy, dwy);
        bspline_weights<ORD, float>((float)rc.t[2], wz, dwz);
        spread_particle<ORD, GRAD>(cu, cg, dscale, wx, dwx, wy, dwy, wz, dwz, (ox * EY + oy) * EZ + oz, E3, EY, EZ,
                                   add);
    };
    // a thread's next record is requested while its current particle is spread
    auto loop = [&](auto add) {
        Rec<TR> rc_next;
        if (threadIdx.x < np) rc_next = w.s_rec[beg + s_order[threadIdx.x]];
        for (unsigned q = threadIdx.x; q < np; q += kFxThreads) {
            const Rec<TR> rc = rc_next;
            const unsigned slot = beg + s_order[q];
            if (q + kFxThreads < np) rc_next = w.s_rec[beg + s_order[q + kFxThreads]];
            particle(rc, slot, add);
        }
    };
    if (sc.fixed) {
        loop([&](int node, float v) {
            const float h = fmaf(v, s1, kRintMagic);
            const float r = fmaf(v, s1, -(h - kRintMagic));  // exact: v 2^e1 - hi
            const float l = fmaf(r, s2, kRintMagic);
            red_shared_u32(hi + node, __float_as_uint(h) - kRintMagicBits);
            red_shared_u32(lo + node, __float_as_uint(l) - kRintMagicBits);
        });
    } else {
        float* acc = reinterpret_cast<float*>(hi);
        loop([&](int node, float v) { red_shared_f32(acc + node, v); });
    }
    __syncthreads();
    auto dst_row = [&](int row, auto* base) {
        const int c = row / (EX * EY), ix = (row / EY) % EX, iy = row % EY;
        return base + (((size_t)c * N + wrap_index(x0 + xs + ix, N)) * N + wrap_index(y0 + iy, N)) * N;
    };
    if (DET && sc.fixed) {
        // the exact sums, rint(v 2^Ef) each, into the 64-bit accumulator
        for (int e = threadIdx.x; e < 3 * E3; e += kFxThreads) {
            const long long f = ((long long)(int)hi[e] << sc.e2) + (int)lo[e];
            if (f != 0) {
                const int row = e / EZ, iz = e - row * EZ;
                atomicAdd(reinterpret_cast<unsigned long long*>(dst_row(row, acc_g) + wrap_index(z0 + iz, N)),
                          (unsigned long long)f);
            }
        }
        return;
    }
    // into g_coef: per tile row the brick's BZ nodes as BZ/4 aligned 16-byte vector atomics (z0 and N are
    // multiples of 4, so 4 consecutive z stay inside one period), then the EZ - BZ halo nodes one by one
    const float inv1 = ldexpf(1.f, -sc.e1), inv12 = ldexpf(1.f, -(sc.e1 + sc.e2));
    auto value = [&](int node) {
        return sc.fixed ? fmaf((float)(int)hi[node], inv1, (float)(int)lo[node] * inv12) : __uint_as_float(hi[node]);
    };
    constexpr int U = BZ / 4 + (EZ - BZ);
    for (int e = threadIdx.x; e < 3 * EX * EY * U; e += kFxThreads) {
        const int row = e / U, k = e - row * U;
        float* dst = dst_row(row, g_coef);
        if (k < BZ / 4) {
            const int nd = row * EZ + 4 * k;
            const float4 v = make_float4(value(nd), value(nd + 1), value(nd + 2), value(nd + 3));
            if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                atomicAdd(reinterpret_cast<float4*>(dst + wrap_index(z0 + 4 * k, N)), v);
        } else {
            const int iz = BZ + (k - BZ / 4);
            const float v = value(row * EZ + iz);
            if (v != 0.f) atomicAdd(dst + wrap_index(z0 + iz, N), v);
        }
    }
}

// g_coef += acc_g 2^-Ef, two nodes a thread (n is even: 3 N^3): each exact sum rounded once to FP32
// (the integer-to-float conversion; the power-of-two scale is exact), then added.  No FP64 arithmetic.
static __global__ void det_finish_kernel(const long long* __restrict__ acc_g, float* __restrict__ g_coef, long long n,
                                         float bound_factor, long long P, const unsigned* __restrict__ bound) {
    const FxScale sc = fx_det_scale(*bound, bound_factor, P);
    const float inv = ldexpf(1.f, -(sc.e1 + sc.e2));
    const longlong2* a2 = reinterpret_cast<const longlong2*>(acc_g);
    float2* g2 = reinterpret_cast<float2*>(g_coef);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n / 2;
         i += (long long)gridDim.x * blockDim.x) {
        const longlong2 a = a2[i];
        float2 g = g2[i];
        g.x += __ll2float_rn(a.x) * inv;
        g.y += __ll2float_rn(a.y) * inv;
        g2[i] = g;
    }
}

// Position gradient: one thread per particle of the work item, coefficients
// staged as in the forward evaluation.
template <int ORD, typename CT, typename TR, bool HESS>
__global__ void __launch_bounds__(kAdjThreads)
gx_kernel(const CT* __restrict__ coef, int N, BrickGrid bg, Ws<TR> w,
          const typename TileT<CT>::T* __restrict__ g_u, const typename TileT<CT>::T* __restrict__ g_grad,
          const float4* __restrict__ cot,
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
        // the particle's cotangents (FP32: from its sorted slot), requested before the contractions that
        // they multiply
        A gu[3], gg[9];
        if (sizeof(A) == 4 && cot) {
            const float4* cp4 = cot + 4 * (size_t)(beg + (kBucket ? (unsigned)s_order[q] : q));
            const float4 v0 = cp4[0], v1 = cp4[1], v2 = cp4[2];
            gu[0] = v0.x; gu[1] = v0.y; gu[2] = v0.z;
            gg[0] = v0.w; gg[1] = v1.x; gg[2] = v1.y; gg[3] = v1.z; gg[4] = v1.w;
            gg[5] = v2.x; gg[6] = v2.y; gg[7] = v2.z; gg[8] = v2.w;
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) gu[c] = g_u ? g_u[3 * idx + c] : A(0);
            if (HESS) {
#pragma unroll
                for (int e = 0; e < 9; ++e) gg[e] = g_grad[9 * idx + e];
            }
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
                const void* g_u, const void* g_grad, void* g_coef, double* g_x, const float4* cot) {
    using A = typename TileT<CT>::T;
    const A dscale = (A)((double)p->N / p->L);
    int rc;
    if constexpr (sizeof(A) == 4) {
        if (g_coef && !cot) g_coef = nullptr;           // no cotangents: nothing to add
        if (g_coef) {
            const size_t sm = fx_tile_bytes<ORD>();
            const unsigned grid = (unsigned)(items * FxShape<ORD>::XP);
            const float factor = g_grad ? 1.f + 3.f * (float)dscale : 1.f;   // |contribution| <= G factor
            if (p->deterministic) {
                // fixed-point accumulator [3][N][N][N] int64, then the bound word
                const long long nodes = 3LL * p->N * p->N * p->N;
                long long* acc_g = reinterpret_cast<long long*>(p->det.ptr);
                unsigned* bound = reinterpret_cast<unsigned*>(acc_g + nodes);
                cudaError_t e = cudaMemsetAsync(acc_g, 0, sizeof(long long) * nodes + 16, p->stream);
                if (e != cudaSuccess) return set_cuda_error(e);
                const long long want = (w.P + 255) / 256;
                const unsigned blocks = (unsigned)std::max(1LL, std::min(want, 8LL * p->sms));
                if (g_grad)
                    cotangent_bound_kernel<true><<<blocks, 256, 0, p->stream>>>((const float*)g_u,
                                                                                (const float*)g_grad, w.P, bound);
                else
                    cotangent_bound_kernel<false><<<blocks, 256, 0, p->stream>>>((const float*)g_u, nullptr, w.P,
                                                                                 bound);
                auto k = g_grad ? spread_fx_kernel<ORD, TR, true, true> : spread_fx_kernel<ORD, TR, false, true>;
                if ((rc = set_smem(k, sm))) return rc;
                k<<<grid, kFxThreads, sm, p->stream>>>(p->N, g, w, cot, (float*)g_coef, acc_g, bound, (float)dscale,
                                                       factor, p->d_status);
                const unsigned fb = (unsigned)std::max(1LL, std::min((nodes / 2 + 255) / 256, 16LL * p->sms));
                det_finish_kernel<<<fb, 256, 0, p->stream>>>(acc_g, (float*)g_coef, nodes, factor, w.P, bound);
            } else {
                auto k = g_grad ? spread_fx_kernel<ORD, TR, true, false> : spread_fx_kernel<ORD, TR, false, false>;
                if ((rc = set_smem(k, sm))) return rc;
                k<<<grid, kFxThreads, sm, p->stream>>>(p->N, g, w, cot, (float*)g_coef, nullptr, nullptr,
                                                       (float)dscale, factor, p->d_status);
            }
            g_coef = nullptr;                               // done
        }
    }
    if constexpr (sizeof(A) == 8) {
        if (g_coef) {
            const size_t sm = acc_bytes<ORD>();
            auto k = g_grad ? spread_kernel<ORD, TR, true> : spread_kernel<ORD, TR, false>;
            if ((rc = set_smem(k, sm))) return rc;
            k<<<(unsigned)items, kAdjThreads, sm, p->stream>>>(p->N, g, w, (const double*)g_u, (const double*)g_grad,
                                                                (double*)g_coef, (double)dscale, p->d_status);
        }
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
                                                            (const A*)g_grad, sizeof(A) == 4 ? cot : nullptr, g_x,
                                                            dscale, tmap, use_tma, p->d_status);
    }
    return BSPLINE_OK;
}

}  // namespace adjoint_impl

#define BS_ADJOINT_EXTERN(ORD, CT, TR)                                                                          \
    extern template int adjoint_impl::run_adjoint<ORD, CT, TR>(bspline_plan_s*, const void*,                   \
                                                                gather_impl::Ws<TR>, BrickGrid, long long,       \
                                                                const void*, const void*, void*, double*,        \
                                                                const float4*);
#define BS_ADJOINT_INSTANTIATE(ORD, CT, TR)                                                                     \
    template int adjoint_impl::run_adjoint<ORD, CT, TR>(bspline_plan_s*, const void*, gather_impl::Ws<TR>,      \
                                                         BrickGrid, long long, const void*, const void*,        \
                                                         void*, double*, const float4*);

}  // namespace bs

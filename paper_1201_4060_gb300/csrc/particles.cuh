// Shared definitions of the particle kernels: workspace layout, weights, gather.
// Included by particles.cu (binning, sort, dispatch) and by the gather_*.cu
// translation units that instantiate the gather for each coefficient type and
// order range (split only to compile in parallel).
#pragma once
#include "internal.h"

namespace bs {
namespace gather_impl {

constexpr int kAnchorBits = 10;          // N <= 1024

template <typename TR> struct Ws {
    unsigned* count;    // [NB + 1]  particles per brick; slot NB = invalid positions
    unsigned* offset;   // [NB + 2]  exclusive prefix sum of count
    unsigned* key;      // [P]
    unsigned* rank;     // [P]
    unsigned* cell;     // [P]       packed anchor node (ax << 20 | ay << 10 | az)
    TR* tf;             // [P][3]    local variable t per axis
    unsigned* s_cell;   // [P]       sorted copies
    TR* s_t;            // [P][3]
    unsigned* s_idx;    // [P]       original particle index
};

inline size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename TR> size_t carve(Ws<TR>* w, void* base, unsigned NB, int64_t P) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void* ptr = base ? (void*)((char*)base + off) : nullptr;
        off += align_up(bytes);
        return ptr;
    };
    w->count = (unsigned*)take(sizeof(unsigned) * (NB + 1));
    w->offset = (unsigned*)take(sizeof(unsigned) * (NB + 2));
    w->key = (unsigned*)take(sizeof(unsigned) * P);
    w->rank = (unsigned*)take(sizeof(unsigned) * P);
    w->cell = (unsigned*)take(sizeof(unsigned) * P);
    w->tf = (TR*)take(sizeof(TR) * 3 * P);
    w->s_cell = (unsigned*)take(sizeof(unsigned) * P);
    w->s_t = (TR*)take(sizeof(TR) * 3 * P);
    w->s_idx = (unsigned*)take(sizeof(unsigned) * P);
    return off;
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

template <typename C> __device__ __forceinline__ float ld_coef(const C* p);
template <> __device__ __forceinline__ float ld_coef<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld_coef<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <typename C, typename A> __device__ __forceinline__ A load_a(const C* p) {
    if constexpr (sizeof(A) == 8) return *p;
    else return ld_coef<C>(p);
}

// ------------------------------------------------------------------ gather
template <int ORD> constexpr int tile_edge() { return kBrick + ORD - 1; }

template <int ORD, typename CT, typename AT, typename TR, bool GRAD>
__global__ void __launch_bounds__(128)
gather_kernel(const CT* __restrict__ coef, int N, int nbx, Ws<TR> w, AT* __restrict__ out_u,
              AT* __restrict__ out_grad, AT dscale) {
    constexpr int E = tile_edge<ORD>();
    constexpr int E3 = E * E * E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT* tile = reinterpret_cast<CT*>(smem_raw);
    const unsigned brick = blockIdx.x;
    const unsigned beg = w.offset[brick], end = w.offset[brick + 1];
    if (beg == end) return;
    const int bx = brick / (nbx * nbx), by = (brick / nbx) % nbx, bz = brick % nbx;
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    const int msk = N - 1;
    for (int e = threadIdx.x; e < 3 * E3; e += blockDim.x) {
        const int c = e / E3, r = e - c * E3;
        const int ix = r / (E * E), iy = (r / E) % E, iz = r % E;
        const size_t g = (((size_t)c * N + ((x0 + ix) & msk)) * N + ((y0 + iy) & msk)) * N + ((z0 + iz) & msk);
        tile[e] = coef[g];
    }
    __syncthreads();
    for (unsigned i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const unsigned cp = w.s_cell[i];
        const int ox = (int)(cp >> (2 * kAnchorBits)) - x0;
        const int oy = (int)((cp >> kAnchorBits) & 1023u) - y0;
        const int oz = (int)(cp & 1023u) - z0;
        AT wx[ORD], dwx[ORD], wy[ORD], dwy[ORD], wz[ORD], dwz[ORD];
        bspline_weights<ORD, AT>((AT)w.s_t[3 * (size_t)i + 0], wx, dwx);
        bspline_weights<ORD, AT>((AT)w.s_t[3 * (size_t)i + 1], wy, dwy);
        bspline_weights<ORD, AT>((AT)w.s_t[3 * (size_t)i + 2], wz, dwz);
        const unsigned idx = w.s_idx[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const CT* tc = tile + c * E3 + (ox * E + oy) * E + oz;
            AT u = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll
            for (int jx = 0; jx < ORD; ++jx) {
                AT y00 = 0, y10 = 0, y01 = 0;
#pragma unroll
                for (int jy = 0; jy < ORD; ++jy) {
                    const CT* line = tc + (jx * E + jy) * E;
                    AT z0v = 0, z1v = 0;
#pragma unroll
                    for (int jz = 0; jz < ORD; ++jz) {
                        const AT a = load_a<CT, AT>(line + jz);
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
            out_u[3 * (size_t)idx + c] = u;
            if (GRAD) {
                out_grad[9 * (size_t)idx + 3 * c + 0] = gx * dscale;
                out_grad[9 * (size_t)idx + 3 * c + 1] = gy * dscale;
                out_grad[9 * (size_t)idx + 3 * c + 2] = gz * dscale;
            }
        }
    }
}

template <typename K> int set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return BSPLINE_OK;
}

template <int ORD, typename CT, typename AT, typename TR>
int run_gather(bspline_plan_s* p, const void* coeffs, Ws<TR> w, unsigned NB, int nbx, void* out_u, void* out_grad,
               bool grad) {
    constexpr int E = tile_edge<ORD>();
    const size_t sm = sizeof(CT) * 3 * (size_t)E * E * E;
    const AT dscale = (AT)((double)p->N / p->L);
    int rc;
    if (grad) {
        auto k = gather_kernel<ORD, CT, AT, TR, true>;
        if ((rc = set_smem(k, sm))) return rc;
        k<<<NB, 128, sm, p->stream>>>(reinterpret_cast<const CT*>(coeffs), p->N, nbx, w, (AT*)out_u, (AT*)out_grad,
                                      dscale);
    } else {
        auto k = gather_kernel<ORD, CT, AT, TR, false>;
        if ((rc = set_smem(k, sm))) return rc;
        k<<<NB, 128, sm, p->stream>>>(reinterpret_cast<const CT*>(coeffs), p->N, nbx, w, (AT*)out_u, nullptr,
                                      dscale);
    }
    return BSPLINE_OK;
}

}  // namespace gather_impl

#define BS_GATHER_EXTERN(ORD, CT, AT, TR)                                                                 \
    extern template int gather_impl::run_gather<ORD, CT, AT, TR>(bspline_plan_s*, const void*,               \
                                                                  gather_impl::Ws<TR>, unsigned, int, void*, \
                                                                  void*, bool);
#define BS_GATHER_INSTANTIATE(ORD, CT, AT, TR)                                                          \
    template int gather_impl::run_gather<ORD, CT, AT, TR>(bspline_plan_s*, const void*, gather_impl::Ws<TR>, \
                                                           unsigned, int, void*, void*, bool);

}  // namespace bs

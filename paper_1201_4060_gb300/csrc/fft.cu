// Prefilter + inverse real 3D FFT: u_hat (half spectrum) -> B-spline coefficients.
//
// Section 7: the coefficients follow from F_D[u_B](k) = c(kx) c(ky) c(kz) F_D[u](k)
// (Eq. B_spline_multiplication_3d) and one inverse transform; the multiply is
// negligible next to the transform (Section 8), so it is fused into the first
// pass's load.
//
// Two kernels, each one HBM read + write of the array:
//   X:  per (component, 16 batch columns): Stockham c2c along kx, prefilter on load;
//   YZ: per (component, x) plane: Stockham c2c along ky into an L2-resident
//       ring of planes, then c2r along kz via a half-length complex transform
//       (even/odd outputs packed as real/imaginary parts), output rounded to
//       the coefficient type on store.
// Each CTA holds a tile of lines in shared memory in a [position][line+1]
// layout (line index fastest, one complex of padding per row), so that global
// loads and stores are coalesced along contiguous lines and every butterfly
// read/write is bank-conflict free.  Radix-8/4/2 Stockham stages, fully
// unrolled per transform length; twiddles exp(+2 pi i m / N) from a table
// computed on the host in FP64.
#include <algorithm>

#include "internal.h"

namespace bs {
namespace {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename V> __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) { V r; r.x = a; r.y = b; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cmuli(V a) { return mk<V>(-a.y, a.x); }  // a * (+i)

// Inverse DFTs (exponent +2 pi i n k / R) in registers.
template <typename V> __device__ __forceinline__ void dft2(V& a, V& b) {
    V t = a;
    a = cadd(t, b);
    b = csub(t, b);
}
template <typename V> __device__ __forceinline__ void dft4(V& x0, V& x1, V& x2, V& x3) {
    V t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = cmuli(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}
template <typename V> __device__ __forceinline__ void dft8(V* x) {
    using R = decltype(V::x);
    V e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    V o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    const R s = (R)0.70710678118654752440084436210485;
    V w1 = mk<V>((o1.x - o1.y) * s, (o1.x + o1.y) * s);     // exp(i pi/4) o1
    V w2 = cmuli(o2);                                        // exp(i pi/2) o2
    V w3 = mk<V>((-o3.x - o3.y) * s, (o3.x - o3.y) * s);    // exp(3 i pi/4) o3
    x[0] = cadd(e0, o0);
    x[4] = csub(e0, o0);
    x[1] = cadd(e1, w1);
    x[5] = csub(e1, w1);
    x[2] = cadd(e2, w2);
    x[6] = csub(e2, w2);
    x[3] = cadd(e3, w3);
    x[7] = csub(e3, w3);
}
template <int R, typename V> __device__ __forceinline__ void butterfly(V* v) {
    if constexpr (R == 2) dft2(v[0], v[1]);
    else if constexpr (R == 4) dft4(v[0], v[1], v[2], v[3]);
    else dft8(v);
}

// One radix-R Stockham stage of NLINES inverse transforms of length L, in
// place in shared memory: element (line b, position q) at s[q * QS + b].
// Butterfly j of a line reads positions j + r L/R, multiplies by
// exp(2 pi i r (j mod NS) / (NS R)), and writes positions
// (j / NS) NS R + (j mod NS) + r NS.  All reads finish before any write.
template <typename V, int L, int NLINES, int T, int RADIX, int NS, int QS>
__device__ __forceinline__ void stage(V* s, const V* tw, int twstride) {
    constexpr int NB = (L / RADIX) * NLINES;
    constexpr int BPT = (NB + T - 1) / T;
    V v[BPT][RADIX];
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int u = t + i * T;
        if (NB % T == 0 || u < NB) {
            const int b = u % NLINES, j = u / NLINES, k = j % NS;
#pragma unroll
            for (int r = 0; r < RADIX; ++r) {
                V a = s[(j + r * (L / RADIX)) * QS + b];
                if (NS > 1 && r > 0) a = cmul(a, tw[(r * k * (L / (NS * RADIX))) * twstride]);
                v[i][r] = a;
            }
            butterfly<RADIX>(v[i]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int u = t + i * T;
        if (NB % T == 0 || u < NB) {
            const int b = u % NLINES, j = u / NLINES, k = j % NS;
            const int d = (j / NS) * NS * RADIX + k;
#pragma unroll
            for (int r = 0; r < RADIX; ++r) s[(d + r * NS) * QS + b] = v[i][r];
        }
    }
    __syncthreads();
}

template <typename V, int L, int NLINES, int T, int QS, int NS = 1>
__device__ __forceinline__ void fft_smem(V* s, const V* tw, int twstride) {
    if constexpr (NS < L) {
        constexpr int REM = L / NS;
        constexpr int RADIX = (REM % 8 == 0) ? 8 : ((REM % 4 == 0) ? 4 : 2);
        stage<V, L, NLINES, T, RADIX, NS, QS>(s, tw, twstride);
        fft_smem<V, L, NLINES, T, QS, NS * RADIX>(s, tw, twstride);
    }
}

template <int L, int NL> constexpr int threads_for() {
    return (L * NL / 16) < 32 ? 32 : (L * NL / 16);
}

// ---------------------------------------------------------------- pass X
// Lines along kx (stride N*H complex); batch index b = ky*H + kz contiguous.
template <typename R, int N, int NL>
__global__ void __launch_bounds__(threads_for<N, NL>())
fft_x_prefilter(const typename Cx<R>::T* __restrict__ in, typename Cx<R>::T* __restrict__ out,
                const R* __restrict__ c, const typename Cx<R>::T* __restrict__ tw, int H) {
    using V = typename Cx<R>::T;
    constexpr int T = threads_for<N, NL>();
    constexpr int QS = NL + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* s = tws + N;
    R* cyz = reinterpret_cast<R*>(s + N * QS);
    const int t = threadIdx.x;
    const long long NH = (long long)N * H;
    const long long tiles = (NH + NL - 1) / NL;
    const int comp = (int)(blockIdx.x / tiles);
    const long long b0 = (blockIdx.x % tiles) * NL;
    for (int m = t; m < N; m += T) tws[m] = tw[m];
    if (t < NL) {
        const long long bb = b0 + t;
        R f = 0;
        if (bb < NH) f = c[(int)(bb / H)] * c[(int)(bb % H)];
        cyz[t] = f;
    }
    __syncthreads();
    const V* src = in + (long long)comp * N * NH + b0;
    for (int e = t; e < N * NL; e += T) {
        const int q = e / NL, b = e % NL;
        V a = mk<V>(0, 0);
        if (b0 + b < NH) {
            a = src[(long long)q * NH + b];
            const R f = c[q] * cyz[b];
            a.x *= f;
            a.y *= f;
        }
        s[q * QS + b] = a;
    }
    __syncthreads();
    fft_smem<V, N, NL, T, QS>(s, tws, 1);
    V* dst = out + (long long)comp * N * NH + b0;
    for (int e = t; e < N * NL; e += T) {
        const int q = e / NL, b = e % NL;
        if (b0 + b < NH) dst[(long long)q * NH + b] = s[q * QS + b];
    }
}

template <typename OutT, typename V> __device__ __forceinline__ void store_pair(OutT* p, V z);
template <> __device__ __forceinline__ void store_pair<double, double2>(double* p, double2 z) {
    *reinterpret_cast<double2*>(p) = z;
}
template <> __device__ __forceinline__ void store_pair<float, float2>(float* p, float2 z) {
    *reinterpret_cast<float2*>(p) = z;
}
template <> __device__ __forceinline__ void store_pair<__nv_bfloat16, float2>(__nv_bfloat16* p, float2 z) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(z.x, z.y);
}


// c2r along kz (Z items below): with M = N/2 and X[M + k] = conj(X[M - k])
// (X[M] itself for k = 0), E[k] = X[k] + X[M + k] and
// O[k] = (X[k] - X[M + k]) exp(2 pi i k / N) have the even and odd outputs as
// their length-M inverse transforms; one complex transform of Z = E + i O
// gives z[m] = x[2m] + i x[2m + 1].  Only the real parts of X[0] and X[M]
// enter (real-to-complex semantics).

// ---------------------------------------------------------------- passes Y + Z fused
// One persistent kernel does the ky transform and the kz c2r of every
// (component, x) plane, handing each plane from one to the other through a
// ring of kRing plane buffers small enough to stay in L2 (kRing x N x H
// complex, 16.8 MB at N = 512 FP32), so the intermediate spectrum never makes
// a round trip through HBM.  Work items are taken in order from a global
// counter: per plane, ceil(H / NL) "Y" items (NL kz columns, all ky) then
// N / NR "Z" items (NR rows y, all kz).  A Z item waits until all Y items of
// its plane have been stored; a Y item waits until the Z items that last used
// its ring slot have read it.  Every dependency points to an earlier item,
// taken by a CTA that is already running, so the waits end; each wait is
// still bounded (about a second) and, if it runs out, sets the error word and
// the kernel returns.
constexpr int kRing = 16;
constexpr long long kWaitLimit = 1LL << 22;

// Counters of one launch (zeroed before it): [0] = work-item counter, then per
// plane the number of finished Y items, then per plane the finished Z items.

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits until *flag >= target (bounded); returns false for the whole CTA on error.
__device__ __forceinline__ bool cta_wait(const unsigned* flag, unsigned target, unsigned* error, unsigned* s_ok) {
    if (threadIdx.x == 0) {
        unsigned ok = 1;
        long long it = 0;
        while (ld_acquire(flag) < target) {
            if (ld_acquire(error) != 0u) { ok = 0; break; }
            if (++it > kWaitLimit) {
                atomicExch(error, 1u);
                ok = 0;
                break;
            }
            __nanosleep(200);
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0u;
}

template <typename V> __device__ __forceinline__ V ld_l2(const V* p) { return __ldcg(p); }

template <typename R, typename OutT, int N, int NL>
__global__ void __launch_bounds__(threads_for<N, NL>())
fft_yz_fused(const typename Cx<R>::T* __restrict__ w, OutT* __restrict__ out, typename Cx<R>::T* ring,
             const typename Cx<R>::T* __restrict__ tw, unsigned* ctr, unsigned* error, int drop_signals) {
    using V = typename Cx<R>::T;
    constexpr int T = threads_for<N, NL>();
    constexpr int H = N / 2 + 1;
    constexpr int M = N / 2;
    constexpr int NR = (2 * NL < N) ? 2 * NL : N;       // Z rows per item: same thread count as a Y item
    constexpr int QY = NL + 1, QZ = NR + 1;
    constexpr int TPZ = (H + NL - 1) / NL;              // Y items per plane
    constexpr int ZPP = N / NR;                         // Z items per plane
    constexpr int IPP = TPZ + ZPP;
    constexpr long long PLANES = 3LL * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* s = tws + N;
    __shared__ unsigned s_item, s_ok;
    unsigned* next = ctr;
    unsigned* done_y = ctr + 1;
    unsigned* done_z = ctr + 1 + PLANES;
    const int t = threadIdx.x;
    for (int m = t; m < N; m += T) tws[m] = tw[m];
    for (;;) {
        if (t == 0) s_item = (ld_acquire(error) != 0u) ? 0xffffffffu : atomicAdd(next, 1u);
        __syncthreads();
        const unsigned item = s_item;
        __syncthreads();
        if (item >= (unsigned)(PLANES * IPP)) return;
        const long long pl = item / IPP;
        const int r = (int)(item % IPP);
        V* slot = ring + (pl % kRing) * (long long)N * H;
        if (r < TPZ) {
            // ---- Y item: columns kz0..kz0+NL-1, all ky; into the ring slot
            if (pl >= kRing && !cta_wait(&done_z[pl - kRing], (unsigned)ZPP, error, &s_ok)) return;
            const int kz0 = r * NL;
            const V* src = w + pl * N * H + kz0;
            for (int e = t; e < N * NL; e += T) {
                const int q = e / NL, b = e % NL;
                s[q * QY + b] = (kz0 + b < H) ? src[(long long)q * H + b] : mk<V>(0, 0);
            }
            __syncthreads();
            fft_smem<V, N, NL, T, QY>(s, tws, 1);
            for (int e = t; e < N * NL; e += T) {
                const int q = e / NL, b = e % NL;
                if (kz0 + b < H) slot[(long long)q * H + kz0 + b] = s[q * QY + b];
            }
            __syncthreads();
            if (t == 0 && !drop_signals) {
                __threadfence();
                atomicAdd(&done_y[pl], 1u);
            }
        } else {
            // ---- Z item: rows y0..y0+NR-1 of the plane, c2r along kz (see fft_z_c2r)
            if (!cta_wait(&done_y[pl], (unsigned)TPZ, error, &s_ok)) return;
            const int y0 = (r - TPZ) * NR;
            for (int e = t; e < NR * M; e += T) {
                const int b = e / M, k = e % M;
                const V* row = slot + (long long)(y0 + b) * H;
                V z;
                if (k == 0) {
                    const R x0 = ld_l2(row).x, xm = ld_l2(row + M).x;
                    z = mk<V>(x0 + xm, x0 - xm);
                } else {
                    const V a = ld_l2(row + k);
                    const V c = ld_l2(row + M - k);
                    const V bb = mk<V>(c.x, -c.y);
                    const V E = cadd(a, bb);
                    const V O = cmul(csub(a, bb), tws[k]);
                    z = mk<V>(E.x - O.y, E.y + O.x);
                }
                s[k * QZ + b] = z;
            }
            __syncthreads();                            // the slot's rows are read: release it
            if (t == 0) {
                __threadfence();
                atomicAdd(&done_z[pl], 1u);
            }
            fft_smem<V, M, NR, T, QZ>(s, tws, 2);
            OutT* dst = out + (pl * N + y0) * (long long)N;
            for (int e = t; e < NR * M; e += T) {
                const int b = e / M, m = e % M;
                store_pair<OutT, V>(dst + (long long)b * N + 2 * m, s[m * QZ + b]);
            }
            __syncthreads();                            // s is reused by the next item
        }
    }
}

template <typename R> constexpr int lines_x() { return sizeof(R) == 4 ? 16 : 8; }

template <typename K> int set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return BSPLINE_OK;
}

template <typename R, typename OutT, int N>
int run_fft(bspline_plan_s* p, const void* u_hat, void* coeffs) {
    using V = typename Cx<R>::T;
    constexpr int NLX = lines_x<R>();
    const int H = N / 2 + 1;
    const R* c = nullptr;
    const V* tw = nullptr;
    if constexpr (sizeof(R) == 8) {
        c = p->d_c64;
        tw = p->d_tw64;
    } else {
        c = p->d_c32;
        tw = p->d_tw32;
    }
    V* w = reinterpret_cast<V*>(p->work.ptr);
    cudaStream_t st = p->stream;
    int rc;
    {
        auto k = fft_x_prefilter<R, N, NLX>;
        const size_t sm = sizeof(V) * (N + (size_t)N * (NLX + 1)) + sizeof(R) * NLX;
        if ((rc = set_smem(k, sm))) return rc;
        const long long tiles = ((long long)N * H + NLX - 1) / NLX;
        StageTimer tm(p, BSPLINE_STAGE_FFT_X);
        k<<<(unsigned)(3 * tiles), threads_for<N, NLX>(), sm, st>>>(reinterpret_cast<const V*>(u_hat), w, c, tw, H);
    }
    {
        auto k = fft_yz_fused<R, OutT, N, NLX>;
        constexpr int NR = (2 * NLX < N) ? 2 * NLX : N;
        constexpr int T = threads_for<N, NLX>();
        const size_t tile = std::max((size_t)N * (NLX + 1), (size_t)(N / 2) * (NR + 1));
        const size_t sm = sizeof(V) * (N + tile);
        if ((rc = set_smem(k, sm))) return rc;
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, T, sm);
        if (e != cudaSuccess) return set_cuda_error(e);
        const long long items = 3LL * N * ((H + NLX - 1) / NLX + N / NR);
        const long long grid = std::min<long long>(items, (long long)std::max(per_sm, 1) * p->sms);
        V* ring = w + 3LL * N * N * H;
        unsigned* ctr = reinterpret_cast<unsigned*>(ring + (long long)kRing * N * H);
        e = cudaMemsetAsync(ctr, 0, sizeof(unsigned) * (1 + 6LL * N), st);
        if (e != cudaSuccess) return set_cuda_error(e);
        StageTimer tm(p, BSPLINE_STAGE_FFT_YZ);
        k<<<(unsigned)grid, T, sm, st>>>(w, reinterpret_cast<OutT*>(coeffs), ring, tw, ctr,
                                         reinterpret_cast<unsigned*>(p->d_status + 1),
                                         (p->test_hooks & BSPLINE_TEST_DROP_TRANSFORM_SIGNALS) ? 1 : 0);
    }
    return set_cuda_error(cudaGetLastError());
}

// Workspace of the transform: the x-transformed spectrum, the plane ring and the counters.
template <typename V> size_t transform_workspace(int N) {
    const size_t H = N / 2 + 1;
    return sizeof(V) * (3ull * N * N * H + (size_t)kRing * N * H) + sizeof(unsigned) * (1 + 6ull * N);
}

template <int N> int run_n(bspline_plan_s* p, const void* u_hat, void* coeffs) {
    switch (p->dtype) {
        case BSPLINE_F64: return run_fft<double, double, N>(p, u_hat, coeffs);
        case BSPLINE_F32: return run_fft<float, float, N>(p, u_hat, coeffs);
        case BSPLINE_BF16: return run_fft<float, __nv_bfloat16, N>(p, u_hat, coeffs);
    }
    return BSPLINE_ERR_INVALID_ARG;
}

}  // namespace

int launch_coeffs(bspline_plan_s* p, const void* u_hat, void* coeffs) {
    const size_t need = p->dtype == BSPLINE_F64 ? transform_workspace<double2>(p->N) : transform_workspace<float2>(p->N);
    int rc = p->work.grow(need);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(p->d_status + 1, 0, sizeof(unsigned long long), p->stream);
    if (e != cudaSuccess) return set_cuda_error(e);
    switch (p->N) {
        case 8: return run_n<8>(p, u_hat, coeffs);
        case 16: return run_n<16>(p, u_hat, coeffs);
        case 32: return run_n<32>(p, u_hat, coeffs);
        case 64: return run_n<64>(p, u_hat, coeffs);
        case 128: return run_n<128>(p, u_hat, coeffs);
        case 256: return run_n<256>(p, u_hat, coeffs);
        case 512: return run_n<512>(p, u_hat, coeffs);
        case 1024: return run_n<1024>(p, u_hat, coeffs);
    }
    return BSPLINE_ERR_UNSUPPORTED_N;
}

}  // namespace bs

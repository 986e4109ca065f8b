// Prefilter + inverse real 3D FFT: u_hat (half spectrum) -> B-spline coefficients.
//
// Section 7: the coefficients follow from F_D[u_B](k) = c(kx) c(ky) c(kz) F_D[u](k)
// (Eq. B_spline_multiplication_3d) and one inverse transform; the multiply is
// negligible next to the transform (Section 8), so it is fused into the first
// pass's load.
//
// Three passes, each one HBM read + write of the array:
//   X: per (component, ky, kz-tile): Stockham c2c along kx, prefilter on load;
//   Y: per (component, x, kz-tile):  Stockham c2c along ky, in place;
//   Z: per (component, x, y) row:    c2r along kz via a half-length complex
//      transform (even/odd outputs packed as real/imaginary parts), output
//      rounded to the coefficient type on store.
// Each CTA holds a tile of lines in shared memory in a [position][line+1]
// layout (line index fastest, one complex of padding per row), so that global
// loads and stores are coalesced along contiguous lines and every butterfly
// read/write is bank-conflict free.  Radix-8/4/2 Stockham stages, fully
// unrolled per transform length; twiddles exp(+2 pi i m / N) from a table
// computed on the host in FP64.
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

// ---------------------------------------------------------------- pass Y
// Lines along ky (stride H); batch along kz (contiguous), ragged last tile.
template <typename R, int N, int NL>
__global__ void __launch_bounds__(threads_for<N, NL>())
fft_y(typename Cx<R>::T* __restrict__ data, const typename Cx<R>::T* __restrict__ tw, int H) {
    using V = typename Cx<R>::T;
    constexpr int T = threads_for<N, NL>();
    constexpr int QS = NL + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* s = tws + N;
    const int t = threadIdx.x;
    const int tpz = (H + NL - 1) / NL;
    const int kz0 = (int)(blockIdx.x % tpz) * NL;
    const long long line = blockIdx.x / tpz;                    // component * N + x
    V* base = data + line * N * H + kz0;
    for (int m = t; m < N; m += T) tws[m] = tw[m];
    for (int e = t; e < N * NL; e += T) {
        const int q = e / NL, b = e % NL;
        s[q * QS + b] = (kz0 + b < H) ? base[(long long)q * H + b] : mk<V>(0, 0);
    }
    __syncthreads();
    fft_smem<V, N, NL, T, QS>(s, tws, 1);
    for (int e = t; e < N * NL; e += T) {
        const int q = e / NL, b = e % NL;
        if (kz0 + b < H) base[(long long)q * H + b] = s[q * QS + b];
    }
}

// ---------------------------------------------------------------- pass Z
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

// c2r of rows of H = N/2 + 1 complex along kz.  With M = N/2 and
// X[M + k] = conj(X[M - k]) (X[M] itself for k = 0), E[k] = X[k] + X[M + k]
// and O[k] = (X[k] - X[M + k]) exp(2 pi i k / N) have the even and odd
// outputs as their length-M inverse transforms; one complex transform of
// Z = E + i O gives z[m] = x[2m] + i x[2m + 1].  Only the real parts of X[0]
// and X[M] enter (real-to-complex semantics).
template <typename R, typename OutT, int N, int NR>
__global__ void __launch_bounds__(threads_for<N / 2, NR>())
fft_z_c2r(const typename Cx<R>::T* __restrict__ in, OutT* __restrict__ out,
          const typename Cx<R>::T* __restrict__ tw, int H) {
    using V = typename Cx<R>::T;
    constexpr int M = N / 2;
    constexpr int T = threads_for<M, NR>();
    constexpr int QS = NR + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* s = tws + N;
    const int t = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * NR;
    for (int m = t; m < N; m += T) tws[m] = tw[m];
    __syncthreads();
    for (int e = t; e < NR * M; e += T) {
        const int b = e / M, k = e % M;
        const V* row = in + (r0 + b) * H;
        V z;
        if (k == 0) {
            const R x0 = row[0].x, xm = row[M].x;
            z = mk<V>(x0 + xm, x0 - xm);
        } else {
            const V a = row[k];
            const V c = row[M - k];
            const V bb = mk<V>(c.x, -c.y);
            const V E = cadd(a, bb);
            const V O = cmul(csub(a, bb), tws[k]);
            z = mk<V>(E.x - O.y, E.y + O.x);
        }
        s[k * QS + b] = z;
    }
    __syncthreads();
    fft_smem<V, M, NR, T, QS>(s, tws, 2);
    for (int e = t; e < NR * M; e += T) {
        const int b = e / M, m = e % M;
        store_pair<OutT, V>(out + (r0 + b) * N + 2 * m, s[m * QS + b]);
    }
}

template <typename R> constexpr int lines_x() { return sizeof(R) == 4 ? 16 : 8; }
constexpr int kRowsZ = 16;

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
        auto k = fft_y<R, N, NLX>;
        const size_t sm = sizeof(V) * (N + (size_t)N * (NLX + 1));
        if ((rc = set_smem(k, sm))) return rc;
        const long long blocks = 3LL * N * ((H + NLX - 1) / NLX);
        StageTimer tm(p, BSPLINE_STAGE_FFT_Y);
        k<<<(unsigned)blocks, threads_for<N, NLX>(), sm, st>>>(w, tw, H);
    }
    {
        auto k = fft_z_c2r<R, OutT, N, kRowsZ>;
        const size_t sm = sizeof(V) * (N + (size_t)(N / 2) * (kRowsZ + 1));
        if ((rc = set_smem(k, sm))) return rc;
        const long long rows = 3LL * N * N;
        StageTimer tm(p, BSPLINE_STAGE_FFT_Z);
        k<<<(unsigned)(rows / kRowsZ), threads_for<N / 2, kRowsZ>(), sm, st>>>(w, reinterpret_cast<OutT*>(coeffs), tw, H);
    }
    return set_cuda_error(cudaGetLastError());
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
    const size_t csz = p->dtype == BSPLINE_F64 ? sizeof(double2) : sizeof(float2);
    const size_t need = csz * 3 * (size_t)p->N * p->N * (p->N / 2 + 1);
    int rc = p->work.grow(need);
    if (rc) return rc;
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

// Building blocks of the shared-memory FFTs: complex helpers, radix-2/3/4/8
// butterflies of the inverse DFT (exponent +2 pi i n k / R), the Stockham
// stage and the tile loads.  Included by the forward path (fft.cu: prefilter
// + inverse real transform) and by its adjoint (adjoint_fft.cu: forward real
// transform + prefilter), which runs the inverse stages on conjugated data.
#pragma once
#include <algorithm>

#include "internal.h"

namespace bs {
namespace fftc {

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
// Length 3: with w = exp(2 pi i / 3) = -1/2 + i sqrt(3)/2, X1 and X2 are
// a - (b + c)/2 +- i (sqrt(3)/2) (b - c).
template <typename V> __device__ __forceinline__ void dft3(V& a, V& b, V& c) {
    using R = decltype(V::x);
    const R h = (R)0.86602540378443864676372317075294;   // sqrt(3) / 2
    const V s = cadd(b, c), d = csub(b, c);
    const V m = mk<V>(a.x - (R)0.5 * s.x, a.y - (R)0.5 * s.y);
    const V id = mk<V>(-h * d.y, h * d.x);
    a = cadd(a, s);
    b = cadd(m, id);
    c = csub(m, id);
}
template <int R, typename V> __device__ __forceinline__ void butterfly(V* v) {
    if constexpr (R == 2) dft2(v[0], v[1]);
    else if constexpr (R == 3) dft3(v[0], v[1], v[2]);
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

// Radix of the stage that has rem = L / NS points left: 8, 4 or 2 while the
// power of two lasts, then 3 (L = 2^a 3^b).
constexpr int radix_for(int rem) {
    return (rem % 8 == 0) ? 8 : ((rem % 4 == 0) ? 4 : ((rem % 2 == 0) ? 2 : 3));
}

template <typename V, int L, int NLINES, int T, int QS, int NS = 1>
__device__ __forceinline__ void fft_smem(V* s, const V* tw, int twstride) {
    if constexpr (NS < L) {
        constexpr int RADIX = radix_for(L / NS);
        stage<V, L, NLINES, T, RADIX, NS, QS>(s, tw, twstride);
        fft_smem<V, L, NLINES, T, QS, NS * RADIX>(s, tw, twstride);
    }
}

// ---- the same transform with its first stage fed from registers and its
// last stage written to registers, so the data make one trip through shared
// memory fewer at each end (and the prefilter or pre/post-processing ride
// along with the loads and stores).  The radix sequence is fixed by L:
// radix_for(L / NS) at each stage, as in fft_smem.

// NS of the last stage (NS * radix_for(L / NS) == L).
constexpr int ns_last(int L) {
    int ns = 1;
    while (ns * radix_for(L / ns) < L) ns *= radix_for(L / ns);
    return ns;
}

// First stage (NS = 1): butterfly j of line b takes positions j + r L/R from
// ld(position, line) and writes s[(j R + r) QS + b].  Ends with a barrier.
// IN_PLACE: ld reads the same shared memory, so a barrier separates every
// thread's reads from the first write.
template <typename V, int L, int NLINES, int T, int QS, bool IN_PLACE = false, typename Ld>
__device__ __forceinline__ void stage_first(V* s, Ld ld) {
    constexpr int RADIX = radix_for(L);
    constexpr int NB = (L / RADIX) * NLINES;
    constexpr int BPT = (NB + T - 1) / T;
    V v[BPT][RADIX];
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int u = t + i * T;
        if (NB % T == 0 || u < NB) {
            const int b = u % NLINES, j = u / NLINES;
#pragma unroll
            for (int r = 0; r < RADIX; ++r) v[i][r] = ld(j + r * (L / RADIX), b);
        }
    }
    if constexpr (IN_PLACE) __syncthreads();
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int u = t + i * T;
        if (NB % T == 0 || u < NB) {
            const int b = u % NLINES, j = u / NLINES;
            butterfly<RADIX>(v[i]);
#pragma unroll
            for (int r = 0; r < RADIX; ++r) s[(j * RADIX + r) * QS + b] = v[i][r];
        }
    }
    __syncthreads();
}

// Stages after the first, up to (not including) the last.
template <typename V, int L, int NLINES, int T, int QS, int NS>
__device__ __forceinline__ void stages_mid(V* s, const V* tw, int twstride) {
    if constexpr (NS < ns_last(L)) {
        constexpr int RADIX = radix_for(L / NS);
        stage<V, L, NLINES, T, RADIX, NS, QS>(s, tw, twstride);
        stages_mid<V, L, NLINES, T, QS, NS * RADIX>(s, tw, twstride);
    }
}

// Last stage (NS = L / R): butterfly j reads positions j + r NS, twiddles by
// exp(2 pi i r j / L), and hands output position j + r NS of line b to st.
// Consecutive threads take consecutive lines (JFAST = false) or consecutive
// butterflies of one line (JFAST = true: stores along a line coalesce).
template <typename V, int L, int NLINES, int T, int QS, bool JFAST, typename St>
__device__ __forceinline__ void stage_last(const V* s, const V* tw, int twstride, St st) {
    constexpr int NS = ns_last(L);
    constexpr int RADIX = L / NS;
    constexpr int NB = NS * NLINES;
    constexpr int BPT = (NB + T - 1) / T;
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int u = t + i * T;
        if (NB % T == 0 || u < NB) {
            const int b = JFAST ? u / NS : u % NLINES, j = JFAST ? u % NS : u / NLINES;
            V v[RADIX];
#pragma unroll
            for (int r = 0; r < RADIX; ++r) {
                V a = s[(j + r * NS) * QS + b];
                if (r > 0) a = cmul(a, tw[(r * j) * twstride]);
                v[r] = a;
            }
            butterfly<RADIX>(v);
#pragma unroll
            for (int r = 0; r < RADIX; ++r) st(j + r * NS, b, v[r]);
        }
    }
}

// A transform of length L = RADIX (one stage): registers only, no shared memory.
template <typename V, int L, int NLINES, int T, typename Ld, typename St>
__device__ __forceinline__ void stage_single(Ld ld, St st) {
    constexpr int NB = NLINES;
    constexpr int BPT = (NB + T - 1) / T;
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int b = t + i * T;
        if (NB % T == 0 || b < NB) {
            V v[L];
#pragma unroll
            for (int r = 0; r < L; ++r) v[r] = ld(r, b);
            butterfly<L>(v);
#pragma unroll
            for (int r = 0; r < L; ++r) st(r, b, v[r]);
        }
    }
}

template <int L, int NL> constexpr int threads_for() {
    return (L * NL / 16) < 32 ? 32 : (L * NL / 16);
}

// Lines per tile: 8 complex float (64-byte row segments), 4 complex double.
template <typename R> constexpr int tile_lines() { return sizeof(R) == 4 ? 8 : 4; }
// Row pitch (complex elements) of the x-transformed spectrum and of the ring:
// H = N/2 + 1 rounded up to a multiple of 8, so every row starts 64-byte aligned.
constexpr int row_pitch(int N) { return ((N / 2 + 1) + 7) & ~7; }

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
// 16 bytes, cached in L2 only: for data another CTA of the same launch wrote.
__device__ __forceinline__ void cp_async16_l2(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copy a tile of NL-element row segments (row stride `pitch` elements) into
// s[q * QS + b]; elements with b >= valid are zero.
template <typename V, int ROWS, int NL, int T, int QS>
__device__ __forceinline__ void load_tile(V* s, const V* __restrict__ src, long long pitch, int valid) {
#pragma unroll
    for (int e = threadIdx.x; e < ROWS * NL; e += T) {
        const int q = e / NL, b = e % NL;
        if (b < valid) {
            if constexpr (sizeof(V) == 8) cp_async8(&s[q * QS + b], src + q * pitch + b);
            else cp_async16(&s[q * QS + b], src + q * pitch + b);
        } else {
            s[q * QS + b] = mk<V>(0, 0);
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

}  // namespace fftc
}  // namespace bs

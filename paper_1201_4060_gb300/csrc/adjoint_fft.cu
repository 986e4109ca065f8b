// Adjoint of the coefficient transform: g_u_hat from g_coef.
//
// The forward map is u_hat -> inverse real transform of c(kx) c(ky) c(kz) u_hat
// (Section 7, Eq. B_spline_multiplication_3d and the coefficient transform).
// Its adjoint, for the real inner product on the coefficients and
// Re <a, b> on the half spectrum (the convention of real-to-complex
// gradients), is
//     g_u_hat(k) = c(kx) c(ky) c(kz) m(kz) sum_x g_coef(x) exp(-2 pi i k.x / N),
// m(kz) = 1 for kz = 0 and kz = N/2, else 2 (how often the inverse real
// transform counts a stored mode).  Three passes, each one HBM read + write:
//   Z:  real-to-complex along z via a half-length complex transform of
//       z[m] = g[2m] + i g[2m+1] (even/odd split, then the twiddle step);
//   Y:  complex along y, in place;
//   X:  complex along x, times c(kx) c(ky) c(kz) m(kz), into the half spectrum.
// The forward DFT is the inverse one read at reversed indices
// (X_fwd[k] = X_inv[(-k) mod L]), so the passes reuse the inverse Stockham
// stages of the forward path and reverse the index on the way out.
#include "fft_core.cuh"

namespace bs {
namespace {

using namespace fftc;

template <typename R> constexpr int zr_rows() { return sizeof(R) == 4 ? 16 : 8; }
template <typename R, int N> constexpr int z_rows_adj() { return zr_rows<R>() < N ? zr_rows<R>() : N; }

// ---------------------------------------------------------------- pass Z (r2c)
// NR consecutive rows (c, x, y) of N reals -> N/2 + 1 complex each, into the
// workspace [3][N][N][HP].  With T the inverse length-M transform of z and
// Z[k] = T[(M - k) mod M] its forward transform:
//   E[k] = (Z[k] + conj Z[M-k]) / 2,  O[k] = (Z[k] - conj Z[M-k]) / (2i),
//   G[k] = E[k] + exp(-2 pi i k / N) O[k],  k = 0..M (indices mod M).
template <typename R, int N>
__global__ void __launch_bounds__(threads_for<N / 2, z_rows_adj<R, N>()>())
fft_z_r2c(const R* __restrict__ g, typename Cx<R>::T* __restrict__ out, const typename Cx<R>::T* __restrict__ tw) {
    using V = typename Cx<R>::T;
    constexpr int M = N / 2, NR = z_rows_adj<R, N>(), QZ = NR + 1;
    constexpr int T = threads_for<M, NR>();
    constexpr int HP = row_pitch(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* trans = tws + N;
    const int t = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * NR;
    for (int m = t; m < N; m += T) tws[m] = tw[m];
    for (int e = t; e < NR * M; e += T) {
        const int b = e / M, m = e % M;
        const R* row = g + (r0 + b) * N;
        trans[m * QZ + b] = mk<V>(row[2 * m], row[2 * m + 1]);
    }
    __syncthreads();
    fft_smem<V, M, NR, T, QZ>(trans, tws, 2);
    constexpr int H = M + 1;
    for (int e = t; e < NR * H; e += T) {
        const int b = e / H, k = e % H;
        const V zk = trans[((M - k) % M) * QZ + b];      // Z[k]
        const V zm = trans[(k % M) * QZ + b];            // Z[M - k]
        const V cm = mk<V>(zm.x, -zm.y);
        const V E = mk<V>((zk.x + cm.x) * R(0.5), (zk.y + cm.y) * R(0.5));
        const V d = csub(zk, cm);
        const V O = mk<V>(d.y * R(0.5), -d.x * R(0.5));   // d / (2i)
        const V w = tws[k];                               // exp(+2 pi i k / N), k <= M < N
        const V wc = mk<V>(w.x, -w.y);
        out[(r0 + b) * HP + k] = cadd(E, cmul(wc, O));
    }
}

// ---------------------------------------------------------------- pass Y
// One (component, x) plane, NL columns kz0.., all y: forward c2c along y in place.
template <typename R, int N, int NL>
__global__ void __launch_bounds__(threads_for<N, NL>())
fft_y_fwd(typename Cx<R>::T* __restrict__ w, const typename Cx<R>::T* __restrict__ tw, int band) {
    using V = typename Cx<R>::T;
    constexpr int T = threads_for<N, NL>();
    constexpr int H = N / 2 + 1, HP = row_pitch(N);
    constexpr int TPZ = (H + NL - 1) / NL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* s = tws + N;
    const int t = threadIdx.x;
    const long long pl = blockIdx.x / TPZ;
    const int kz0 = (int)(blockIdx.x % TPZ) * NL;
    if (band && kz0 > band) return;                      // columns the band's last pass writes as zero
    const int valid = min(NL, H - kz0);
    V* base = w + pl * N * HP + kz0;
    load_tile<V, N, NL, T, NL>(s, base, HP, valid);
    for (int m = t; m < N; m += T) tws[m] = tw[m];
    cp_async_wait_all();
    __syncthreads();
    fft_smem<V, N, NL, T, NL>(s, tws, 1);
    for (int e = t; e < N * NL; e += T) {
        const int q = e / NL, b = e % NL;
        if (b < valid) base[(long long)q * HP + b] = s[((N - q) % N) * NL + b];
    }
}

// ---------------------------------------------------------------- pass X
// NL columns (ky, kz0..) of one component: forward c2c along x, times
// c(kx) c(ky) c(kz) m(kz), into the half spectrum [3][N][N][N/2+1].
template <typename R, int N, int NL>
__global__ void __launch_bounds__(threads_for<N, NL>())
fft_x_fwd_prefilter(const typename Cx<R>::T* __restrict__ w, typename Cx<R>::T* __restrict__ out,
                    const R* __restrict__ c, const typename Cx<R>::T* __restrict__ tw, int band) {
    using V = typename Cx<R>::T;
    constexpr int T = threads_for<N, NL>();
    constexpr int M = N / 2, H = M + 1, HP = row_pitch(N);
    constexpr int TPZ = (H + NL - 1) / NL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* s = tws + N;
    const int t = threadIdx.x;
    const int comp = (int)(blockIdx.x / ((long long)N * TPZ));
    const int rem = (int)(blockIdx.x % ((long long)N * TPZ));
    const int ky = rem / TPZ, kz0 = (rem % TPZ) * NL;
    const int valid = min(NL, H - kz0);
    // a band (bspline_plan_set_band): the forward path ignores every mode outside |kx|, |ky|, kz <= band,
    // so their gradient is zero; columns wholly outside it are written as zeros without a transform
    V* dst = out + (long long)comp * N * N * H;
    if (band && (kz0 > band || (ky > band && ky < N - band))) {
        for (int e = t; e < N * NL; e += T) {
            const int kx = e / NL, b = e % NL;
            if (b < valid) dst[((long long)kx * N + ky) * H + kz0 + b] = mk<V>(R(0), R(0));
        }
        return;
    }
    load_tile<V, N, NL, T, NL>(s, w + (long long)comp * N * N * HP + (long long)ky * HP + kz0, (long long)N * HP,
                               valid);
    for (int m = t; m < N; m += T) tws[m] = tw[m];
    cp_async_wait_all();
    __syncthreads();
    fft_smem<V, N, NL, T, NL>(s, tws, 1);
    const R cy = __ldg(&c[ky]);
    for (int e = t; e < N * NL; e += T) {
        const int kx = e / NL, b = e % NL;
        if (b < valid) {
            const int kz = kz0 + b;
            const R f = __ldg(&c[kx]) * cy * __ldg(&c[kz]) * ((kz == 0 || kz == M) ? R(1) : R(2));
            const V a = s[((N - kx) % N) * NL + b];
            const bool in = !band || (kz <= band && (kx <= band || kx >= N - band));
            dst[((long long)kx * N + ky) * H + kz] = in ? mk<V>(a.x * f, a.y * f) : mk<V>(R(0), R(0));
        }
    }
}

template <typename R, int N>
int run_adjoint_fft(bspline_plan_s* p, const void* g_coef, void* g_u_hat) {
    using V = typename Cx<R>::T;
    constexpr int NL = tile_lines<R>();
    constexpr int H = N / 2 + 1;
    constexpr int TPZ = (H + NL - 1) / NL;
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
    StageTimer tm(p, BSPLINE_STAGE_ADJ_FFT);
    {
        constexpr int NR = z_rows_adj<R, N>();
        constexpr int T = threads_for<N / 2, NR>();
        auto k = fft_z_r2c<R, N>;
        const size_t sm = sizeof(V) * (N + (size_t)(N / 2) * (NR + 1));
        if ((rc = set_smem(k, sm))) return rc;
        k<<<(unsigned)(3LL * N * N / NR), T, sm, st>>>(reinterpret_cast<const R*>(g_coef), w, tw);
    }
    {
        constexpr int T = threads_for<N, NL>();
        auto k = fft_y_fwd<R, N, NL>;
        const size_t sm = sizeof(V) * (N + (size_t)N * NL);
        if ((rc = set_smem(k, sm))) return rc;
        k<<<(unsigned)(3LL * N * TPZ), T, sm, st>>>(w, tw, p->band);
    }
    {
        constexpr int T = threads_for<N, NL>();
        auto k = fft_x_fwd_prefilter<R, N, NL>;
        const size_t sm = sizeof(V) * (N + (size_t)N * NL);
        if ((rc = set_smem(k, sm))) return rc;
        k<<<(unsigned)(3LL * N * TPZ), T, sm, st>>>(w, reinterpret_cast<V*>(g_u_hat), c, tw, p->band);
    }
    return set_cuda_error(cudaGetLastError());
}

template <int N> int adj_n(bspline_plan_s* p, const void* g_coef, void* g_u_hat) {
    if (p->dtype == BSPLINE_F64) return run_adjoint_fft<double, N>(p, g_coef, g_u_hat);
    return run_adjoint_fft<float, N>(p, g_coef, g_u_hat);
}

}  // namespace

// Workspace: the z/y-transformed spectrum [3][N][N][HP] (inside the forward
// transform's workspace, which the caller has grown).
int launch_adjoint_transform(bspline_plan_s* p, const void* g_coef, void* g_u_hat) {
    switch (p->N) {
        case 8: return adj_n<8>(p, g_coef, g_u_hat);
        case 16: return adj_n<16>(p, g_coef, g_u_hat);
        case 32: return adj_n<32>(p, g_coef, g_u_hat);
        case 64: return adj_n<64>(p, g_coef, g_u_hat);
        case 128: return adj_n<128>(p, g_coef, g_u_hat);
        case 256: return adj_n<256>(p, g_coef, g_u_hat);
        case 512: return adj_n<512>(p, g_coef, g_u_hat);
        case 1024: return adj_n<1024>(p, g_coef, g_u_hat);
        case 48: return adj_n<48>(p, g_coef, g_u_hat);
        case 96: return adj_n<96>(p, g_coef, g_u_hat);
        case 192: return adj_n<192>(p, g_coef, g_u_hat);
        case 384: return adj_n<384>(p, g_coef, g_u_hat);
        case 768: return adj_n<768>(p, g_coef, g_u_hat);
    }
    return BSPLINE_ERR_UNSUPPORTED_N;
}

}  // namespace bs

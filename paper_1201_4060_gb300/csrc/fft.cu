// Prefilter + inverse real 3D FFT: u_hat (half spectrum) -> B-spline coefficients.
//
// Section 7: the coefficients follow from F_D[u_B](k) = c(kx) c(ky) c(kz) F_D[u](k)
// (Eq. B_spline_multiplication_3d) and one inverse transform; the multiply is
// negligible next to the transform (Section 8), so it is fused into the first
// pass.
//
// Two kernels, each one HBM read + write of the array:
//   X:  per (component, NL batch columns): Stockham c2c along kx, prefilter
//       applied to the staged tile; output spectrum with rows padded to a
//       multiple of 8 complex (64 bytes);
//   YZ: per (component, x) plane: Stockham c2c along ky into a ring of plane
//       buffers small enough to stay in L2, then c2r along kz via a
//       half-length complex transform (even/odd outputs packed as real and
//       imaginary parts), rounded to the coefficient type on store.
// Tiles move between global and shared memory with cp.async, so the data in
// flight occupies shared memory rather than registers and several CTAs per SM
// keep loads outstanding while others compute.  In shared memory a kx/ky tile
// is [position][line] with 64-byte rows (line index fastest): a half-warp's
// 64-bit accesses cover two whole rows, so butterfly reads are bank-conflict
// free (only the first stage's scattered writes pair up); the kz transform
// uses [position][line + 1], conflict-free for its transposed fill.
// Global accesses are coalesced along contiguous lines.  Radix-8/4/2 Stockham stages, fully
// unrolled per transform length; twiddles exp(+2 pi i m / N) from a table
// computed on the host in FP64.
#include "fft_core.cuh"

namespace bs {
namespace {

using namespace fftc;

// ---------------------------------------------------------------- pass X
// Lines along kx (input stride N*H complex); batch index b = ky*H + kz is
// contiguous in the input.  Output: [3][N(x)][N(ky)][HP] with kz fastest.
// Several fields of one grid size in one launch (batches): in_fields[f] is
// field f's half spectrum, its x-transformed spectrum goes to out + f 3 N N HP,
// and the grid holds 3 * tiles CTAs per field.  in_fields = nullptr: one field.
// band > 0 (bspline_plan_set_band): modes with |kx|, |ky| or kz beyond band are
// zero; they are not read, and the columns (ky, kz) outside the band are not
// transformed or stored (the ky/kz pass never reads them).
template <typename R, int N, int NL>
__global__ void __launch_bounds__(threads_for<N, NL>())
fft_x_prefilter(const typename Cx<R>::T* __restrict__ in, typename Cx<R>::T* __restrict__ out,
                const R* __restrict__ c, const typename Cx<R>::T* __restrict__ tw, int comp0,
                const typename Cx<R>::T* const* __restrict__ in_fields, int band) {
    using V = typename Cx<R>::T;
    constexpr int T = threads_for<N, NL>();
    static_assert(T % NL == 0, "each thread stays on one line");
    constexpr int H = N / 2 + 1, HP = row_pitch(N);
    constexpr long long NH = (long long)N * H;
    constexpr long long TILES = (NH + NL - 1) / NL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* s = tws + N;
    const int t = threadIdx.x;
    unsigned bx = blockIdx.x;
    if (in_fields) {
        constexpr unsigned per = 3u * (unsigned)TILES;
        const unsigned f = bx / per;
        bx -= f * per;
        in = in_fields[f];
        out += (long long)f * 3 * N * N * HP;
    }
    const int comp = comp0 + (int)(bx / TILES);
    const long long b0 = (bx % TILES) * NL;
    const int valid = (int)std::min<long long>(NL, NH - b0);
    auto col_in_band = [&](int b) {                      // column b0 + b = ky H + kz inside the band
        const long long bb = b0 + b;
        const int ky = (int)(bb / H), kz = (int)(bb % H);
        return kz <= band && (ky <= band || ky >= N - band);
    };
    if (band) {                                          // a tile with no column in the band has nothing to do
        bool any = false;
        for (int b = 0; b < valid; ++b) any = any || col_in_band(b);
        if (!any) return;
    }
    for (int m = t; m < N; m += T) tws[m] = tw[m];
    // this thread's line: batch index b0 + bl = ky H + kz; prefilter c(ky) c(kz) of the line
    const int bl = t % NL;
    const long long bb = b0 + bl;
    const int ky = (int)(bb / H), kz = (int)(bb % H);
    const R cyz = (bl < valid) ? c[ky] * c[kz] : R(0);
    const V* src = in + (long long)comp * N * NH + b0;
    V* dst = out + (long long)comp * N * N * HP + (long long)ky * HP + kz;
    // this thread's line (every thread stays on its column bl: the b below is always bl)
    const bool col = bl < valid && (!band || col_in_band(bl));
    auto ld = [&](int q, int b) -> V {                   // prefilter c(kx) c(ky) c(kz) on load
        if (!col || (band && q > band && q < N - band)) return mk<V>(R(0), R(0));
        const V a = src[(long long)q * NH + b];
        const R f = __ldg(&c[q]) * cyz;
        return mk<V>(a.x * f, a.y * f);
    };
    auto st = [&](int q, int b, V v) {
        if (col) dst[(long long)q * N * HP] = v;
    };
    if constexpr (radix_for(N) == N) {
        stage_single<V, N, NL, T>(ld, st);
    } else {
        stage_first<V, N, NL, T, NL>(s, ld);            // its barrier also publishes the twiddles
        stages_mid<V, N, NL, T, NL, radix_for(N)>(s, tws, 1);
        stage_last<V, N, NL, T, NL, false>(s, tws, 1, st);
    }
}

template <typename OutT, typename V> __device__ __forceinline__ void store_pair(OutT* p, V z);
// Coefficient stores stream past L2 (evict first): the ring of plane buffers is what should stay there.
template <> __device__ __forceinline__ void store_pair<double, double2>(double* p, double2 z) {
    __stcs(reinterpret_cast<double2*>(p), z);
}
template <> __device__ __forceinline__ void store_pair<float, float2>(float* p, float2 z) {
    __stcs(reinterpret_cast<float2*>(p), z);
}
template <> __device__ __forceinline__ void store_pair<__nv_bfloat16, float2>(__nv_bfloat16* p, float2 z) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(z.x, z.y);
    __stcs(reinterpret_cast<unsigned*>(p), *reinterpret_cast<const unsigned*>(&v));
}

// ---------------------------------------------------------------- passes Y + Z fused
// One persistent kernel does the ky transform and the kz c2r of every
// (component, x) plane, handing each plane from one to the other through a
// ring of plane buffers small enough to stay in L2 (kRingMax planes, or up
// to 64 MB of them for small planes: fields_ring_slots), so the intermediate
// spectrum never makes a round trip through HBM.  Work items are taken in order from a global
// counter: per plane, ceil(H / NL) "Y" items (NL kz columns, all ky) then
// N / NR "Z" items (NR rows y, all kz).  A Z item waits until all Y items of
// its plane have been stored; a Y item waits until the Z items that last used
// its ring slot have read it.  Thread 0 checks an item's flag when it hands
// the item to its CTA: while the previous item runs it has already read that
// flag (relaxed), and if the read shows the dependency done an acquire fence
// is all the check costs; otherwise it waits on the flag with acquire loads.
// Every dependency points to an earlier item, taken by a CTA that is already
// running, so the waits end; each wait is still bounded (about a second) and,
// if it runs out, sets the error word and the CTA returns; every later wait
// of the launch sees the error word and returns at once, so the launch ends.
//
// c2r along kz: with M = N/2 and X[M + k] = conj(X[M - k]) (X[M] itself for
// k = 0), E[k] = X[k] + X[M + k] and O[k] = (X[k] - X[M + k]) exp(2 pi i k / N)
// have the even and odd outputs as their length-M inverse transforms; one
// complex transform of Z = E + i O gives z[m] = x[2m] + i x[2m + 1].  Only the
// real parts of X[0] and X[M] enter (real-to-complex semantics).
// Items are dequeued in super-steps: step s holds the Y items of plane s and
// then the Z items of plane s - lag, so a plane's consumers come lag planes
// after its producers.  The host picks lag from the number of planes the
// resident CTAs work on at once (plus a margin) and ring = 2 lag slots, so a
// Y item rarely waits for its slot either; lag < ring keeps every dependency
// pointing back.
constexpr int kRingMax = 32;
constexpr long long kWaitLimit = 1LL << 22;

// Item index -> (plane, index within the plane: < TPZ for Y items, else TPZ + Z index).
template <int TPZ, int ZPP>
__device__ __forceinline__ void item_to_plane(long long item, long long planes, int lag, long long* pl, int* r) {
    constexpr int IPP = TPZ + ZPP;
    const long long head = (long long)lag * TPZ;                   // steps 0..lag-1: Y items only
    const long long body = head + (planes - lag) * IPP;            // steps lag..planes-1: Y then Z
    if (item < head) {
        *pl = item / TPZ;
        *r = (int)(item % TPZ);
    } else if (item < body) {
        const long long j = item - head, s = lag + j / IPP;
        const int q = (int)(j % IPP);
        if (q < TPZ) {
            *pl = s;
            *r = q;
        } else {
            *pl = s - lag;
            *r = q;
        }
    } else {                                                       // steps planes..planes+lag-1: Z only
        const long long j = item - body;
        *pl = planes + j / ZPP - lag;
        *r = TPZ + (int)(j % ZPP);
    }
}

// Counters of one launch (zeroed before it): [0] = work-item counter, then per
// plane the number of finished Y items, then per plane the finished Z items.

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Count one finished item: a release reduction, so everything the CTA wrote or
// read before its last barrier happens before any acquire load that sees the count.
__device__ __forceinline__ void signal_release(unsigned* p) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

// Relaxed load at GPU scope: no ordering of its own; with fence_acq_rel after
// it (once it has seen a released count) it acts as an acquire.
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Thread 0 only: bounded acquire wait for *flag >= target; false (error word set) if it runs out.
__device__ __forceinline__ bool spin_acquire(const unsigned* flag, unsigned target, unsigned* error) {
    long long it = 0;
    while (ld_acquire(flag) < target) {
        if (ld_acquire(error) != 0u) return false;
        if (++it > kWaitLimit) {
            atomicExch(error, 1u);
            return false;
        }
        __nanosleep(200);
    }
    return true;
}

// Z rows per item: 2 NL (16 FP32 rows, 8 FP64 rows; all of them for small N).
// The rows are transformed in place (the staged ring rows and the transform
// buffer share memory), which keeps a CTA's shared memory small enough for
// four CTAs per SM in FP32 while halving the number of Z items and the fixed
// cost each one carries (its wait, its barriers, its signal).
template <typename R, int N, int NL> constexpr int z_rows() {
    return (2 * NL < N) ? 2 * NL : N;
}

// Row pitch of the staged ring rows of a Z item: HP plus 16 bytes of skew, so
// that the rows of one warp access spread over all banks (row stride an odd
// multiple of 16 bytes modulo 128).
template <typename V, int N> constexpr int z_row_pitch() { return row_pitch(N) + 16 / (int)sizeof(V); }

// The fused kernel runs threads_for<N, TL> threads (TL = tile_lines) on Y
// items of NLY columns and Z items of z_rows<R, N, TL> rows.
template <typename R, int N, int TL, int NLY>
constexpr size_t yz_smem_elems() {
    using V = typename Cx<R>::T;
    constexpr int NR = z_rows<R, N, TL>();
    constexpr size_t y = (size_t)N * NLY;
    constexpr size_t zr = (size_t)NR * z_row_pitch<V, N>(), zt = (size_t)(N / 2) * (NR + 1);
    constexpr size_t z = zr > zt ? zr : zt;
    return N + (y > z ? y : z);
}

// CTAs per SM the fused kernel is compiled for: 32 warps per SM (FP32), 24 (FP64).
template <typename R, int N, int NL> constexpr int yz_min_blocks() {
    constexpr int W = sizeof(R) == 4 ? 1024 : 768;
    return (W / threads_for<N, NL>()) < 1 ? 1 : (W / threads_for<N, NL>());
}

template <typename R, typename OutT, int N, int NL, int NLY>
__global__ void __launch_bounds__(threads_for<N, NL>(), yz_min_blocks<R, N, NL>())
fft_yz_fused(const typename Cx<R>::T* __restrict__ w, OutT* __restrict__ out, typename Cx<R>::T* ring,
             const typename Cx<R>::T* __restrict__ tw, unsigned* ctr, unsigned* error, int lag, int ring_slots,
             int drop_signals, long long plane0, long long planes, OutT* const* __restrict__ out_fields, int band) {
    using V = typename Cx<R>::T;
    constexpr int T = threads_for<N, NL>();
    constexpr int H = N / 2 + 1, HP = row_pitch(N);
    constexpr int M = N / 2;
    constexpr int NR = z_rows<R, N, NL>();              // Z rows per item: same thread count as a Y item
    constexpr int QY = NLY, QZ = NR + 1;
    constexpr int TPZ = (H + NLY - 1) / NLY;            // Y items per plane
    constexpr int ZPP = N / NR;                         // Z items per plane
    constexpr int IPP = TPZ + ZPP;
    constexpr int CHUNKS = HP * (int)sizeof(V) / 16;    // 16-byte pieces of one ring row
    constexpr int RP = z_row_pitch<V, N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tws = reinterpret_cast<V*>(smem_raw);
    V* buf = tws + N;                                   // Y: [N][QY] tile of NLY columns
    V* raw = buf;                                       // Z: NR ring rows, pitch RP
    V* trans = buf;                                     // Z: [M][QZ] transform buffer over them (in place)
    __shared__ unsigned s_item[2];
    unsigned* next = ctr;
    unsigned* done_y = ctr + 1;
    unsigned* done_z = ctr + 1 + planes;
    const int t = threadIdx.x;
    for (int m = t; m < N; m += T) tws[m] = tw[m];
    // thread 0 claims the following item while this one runs (its counter round trip overlaps the work);
    // a claimed item depends only on earlier items, so the smallest running item can always proceed
    unsigned claimed = (t == 0) ? atomicAdd(next, 1u) : 0u;
    const unsigned total = (unsigned)(planes * IPP);
    unsigned pre_item = 0xffffffffu, pre_val = 0;       // thread 0: relaxed read of the next item's flag
    // the flag an item waits for: a Z item its plane's Y items, a Y item its ring slot
    auto flag_of = [&](unsigned item, const unsigned** f, unsigned* target) {
        long long lp;
        int r;
        item_to_plane<TPZ, ZPP>(item, planes, lag, &lp, &r);
        *f = nullptr;
        if (r >= TPZ) {
            *f = &done_y[lp];
            *target = (unsigned)TPZ;
        } else if (lp >= ring_slots) {
            *f = &done_z[lp - ring_slots];
            *target = (unsigned)ZPP;
        }
    };
    auto prefetch_flag = [&]() {                        // thread 0, once the next claim has returned
        pre_item = claimed;
        const unsigned* f;
        unsigned target;
        if (pre_item < total) {
            flag_of(pre_item, &f, &target);
            pre_val = f ? ld_relaxed(f) : 0u;
        }
    };
    for (unsigned it = 0;; ++it) {
        // alternate slots: the slot written now was last read two items ago, before this item's barriers
        if (t == 0) {
            const unsigned item = claimed;
            claimed = atomicAdd(next, 1u);
            unsigned ok = 1;
            if (item < total) {
                const unsigned* f;
                unsigned target;
                flag_of(item, &f, &target);
                if (f) {
                    if (pre_item == item && pre_val >= target) { fence_acq_rel(); }
                    else ok = spin_acquire(f, target, error) ? 1u : 0u;
                }
            }
            s_item[it & 1u] = ok ? item : 0xfffffffeu;
        }
        __syncthreads();
        const unsigned item = s_item[it & 1u];
        if (item >= total) return;
        long long lp;                                   // plane within this launch; pl = plane0 + lp
        int r;
        item_to_plane<TPZ, ZPP>(item, planes, lag, &lp, &r);
        const long long pl = plane0 + lp;
        V* slot = ring + (lp % ring_slots) * (long long)N * HP;
        if (r < TPZ && band && r * NLY > band) {
            // ---- Y item beyond the band: its columns are zero, and the Z items never read them
            if (t == 0) prefetch_flag();
            __syncthreads();
            if (t == 0 && !drop_signals) signal_release(&done_y[lp]);
        } else if (r < TPZ) {
            // ---- Y item: columns kz0..kz0+NL-1, all ky; into the ring slot (rows ky beyond the band: zero)
            const int kz0 = r * NLY;
            const int valid = std::min(NLY, H - kz0);
            const V* src = w + pl * N * HP + kz0;
            V* dst = slot + kz0;
            auto ld = [&](int q, int b) -> V {
                return (b < valid && (!band || q <= band || q >= N - band)) ? __ldcs(&src[(long long)q * HP + b])
                                                                              : mk<V>(R(0), R(0));
            };
            auto st = [&](int q, int b, V v) {
                if (b < valid) dst[(long long)q * HP + b] = v;
            };
            if constexpr (radix_for(N) == N) {
                if (t == 0) prefetch_flag();
                stage_single<V, N, NLY, T>(ld, st);
            } else {
                stage_first<V, N, NLY, T, QY>(buf, ld);
                if (t == 0) prefetch_flag();
                stages_mid<V, N, NLY, T, QY, radix_for(N)>(buf, tws, 1);
                stage_last<V, N, NLY, T, QY, false>(buf, tws, 1, st);
            }
            __syncthreads();
            if (t == 0 && !drop_signals) {
                signal_release(&done_y[lp]);
            }
        } else {
            // ---- Z item: rows y0..y0+NR-1 of the plane, c2r along kz
            const int y0 = (r - TPZ) * NR;
            const unsigned char* src = reinterpret_cast<const unsigned char*>(slot + (long long)y0 * HP);
            unsigned char* dstb = reinterpret_cast<unsigned char*>(raw);
            // with a band only the row's first band + 1 modes are staged (the others are read as zero)
            const int nch = band ? std::min(CHUNKS, ((band + 1) * (int)sizeof(V) + 15) / 16) : CHUNKS;
            for (int j = t; j < NR * nch; j += T) {
                const int row = j / nch, k = j - row * nch;
                cp_async16_l2(dstb + (size_t)row * RP * sizeof(V) + 16 * k, src + (size_t)row * HP * sizeof(V) + 16 * k);
            }
            cp_async_wait_all();
            __syncthreads();                            // the slot's rows are read: release it
            if (t == 0) {
                signal_release(&done_z[lp]);
                prefetch_flag();
            }
            auto ld = [&](int k, int b) -> V {          // even/odd split of the half spectrum
                const V* row = raw + b * RP;
                const V zero = mk<V>(R(0), R(0));       // modes beyond the band
                const V a = (!band || k <= band) ? row[k] : zero;
                const V c = (!band || M - k <= band) ? row[M - k] : zero;   // k = 0: X[0] and X[M]
                if (k == 0) return mk<V>(a.x + c.x, a.x - c.x);
                const V bb = mk<V>(c.x, -c.y);
                const V E = cadd(a, bb);
                const V O = cmul(csub(a, bb), tws[k]);
                return mk<V>(E.x - O.y, E.y + O.x);
            };
            // planes of several fields (batches): field pl / 3N writes its own coefficients
            OutT* ob = out;
            long long lpl = pl;
            if (out_fields) {
                const long long f = pl / (3LL * N);
                ob = out_fields[f];
                lpl = pl - f * 3LL * N;
            }
            OutT* dst = ob + (lpl * N + y0) * (long long)N;
            auto st = [&](int m, int b, V z) { store_pair<OutT, V>(dst + (long long)b * N + 2 * m, z); };
            if constexpr (radix_for(M) == M) {
                stage_single<V, M, NR, T>(ld, st);
            } else {
                stage_first<V, M, NR, T, QZ, true>(trans, ld);
                stages_mid<V, M, NR, T, QZ, radix_for(M)>(trans, tws, 2);
                stage_last<V, M, NR, T, QZ, true>(trans, tws, 2, st);
            }
            __syncthreads();                            // smem is reused by the next item
        }
    }
}

// Ring slots of a transform over F fields of grid N: one launch keeps about 2 grid / (items per plane)
// planes in flight, far more than kRingMax for small planes, so the ring grows up to 64 MB of planes
// (L2-resident; 59 slots at 512^3 FP32, where 32 MB gave the same time within 2 %).
template <typename V> long long fields_ring_slots(int N, int F) {
    const long long plane = (long long)sizeof(V) * N * row_pitch(N);
    const long long fit = (64LL << 20) / plane;
    return std::max<long long>(kRingMax, std::min<long long>(3LL * N * F, fit));
}

// Workspace of the transform: the x-transformed spectrum, the plane ring and the counters.
template <typename V> size_t transform_workspace(int N) {
    const size_t HP = row_pitch(N);
    return sizeof(V) * (3ull * N * N * HP + (size_t)fields_ring_slots<V>(N, 1) * N * HP) +
           sizeof(unsigned) * (1 + 6ull * N);
}

// Y-item columns in units of tile_lines.
constexpr int kYCols = 1;

template <typename R, typename OutT, int N>
int run_fft(bspline_plan_s* p, const void* u_hat, void* coeffs, int c0, int c1) {
    using V = typename Cx<R>::T;
    constexpr int NL = tile_lines<R>();
    constexpr int T = threads_for<N, NL>();
    constexpr int H = N / 2 + 1, HP = row_pitch(N);
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
        // twice the lines of a y/z tile: 128-byte row segments per kx in HBM
        constexpr int NLX = 2 * NL;
        auto k = fft_x_prefilter<R, N, NLX>;
        const size_t sm = sizeof(V) * (N + (size_t)N * NLX);
        if ((rc = set_smem(k, sm))) return rc;
        const long long tiles = ((long long)N * H + NLX - 1) / NLX;
        StageTimer tm(p, BSPLINE_STAGE_FFT_X);
        k<<<(unsigned)((c1 - c0) * tiles), threads_for<N, NLX>(), sm, st>>>(reinterpret_cast<const V*>(u_hat), w, c,
                                                                             tw, c0, nullptr, p->band);
    }
    {
        auto k = fft_yz_fused<R, OutT, N, NL, kYCols * NL>;
        constexpr int NR = z_rows<R, N, NL>();
        const size_t sm = sizeof(V) * yz_smem_elems<R, N, NL, kYCols * NL>();
        if ((rc = set_smem(k, sm))) return rc;
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, T, sm);
        if (e != cudaSuccess) return set_cuda_error(e);
        const int ipp = (H + kYCols * NL - 1) / (kYCols * NL) + N / NR;
        const long long planes = (long long)(c1 - c0) * N;
        const long long items = planes * ipp;
        const long long grid = std::min<long long>(items, (long long)std::max(per_sm, 1) * p->sms);
        // planes in progress at once ~ 2 grid / items-per-plane (each CTA runs one item and has claimed
        // the next); consumers trail by that plus a margin
        const long long slots = fields_ring_slots<V>(N, 1);
        const int lag = (int)std::min<long long>(std::min<long long>(slots / 2, planes),
                                                 (2 * grid + ipp - 1) / ipp + 2);
        const int ring_slots = 2 * lag;
        V* ring = w + 3LL * N * N * HP;
        unsigned* ctr = reinterpret_cast<unsigned*>(ring + slots * N * HP);
        e = cudaMemsetAsync(ctr, 0, sizeof(unsigned) * (1 + 2 * planes), st);
        if (e != cudaSuccess) return set_cuda_error(e);
        StageTimer tm(p, BSPLINE_STAGE_FFT_YZ);
        k<<<(unsigned)grid, T, sm, st>>>(w, reinterpret_cast<OutT*>(coeffs), ring, tw, ctr,
                                         reinterpret_cast<unsigned*>(p->d_status + kStatusTransformTimeout), lag, ring_slots,
                                         (p->test_hooks & BSPLINE_TEST_DROP_TRANSFORM_SIGNALS) ? 1 : 0,
                                         (long long)c0 * N, planes, nullptr, p->band);
    }
    return set_cuda_error(cudaGetLastError());
}

// F fields of one grid size, order, prefilter and band (those of p) in one launch of each kernel:
// in_fields / out_fields are device arrays of F pointers; w is the group's workspace
// (fields_workspace<V>(N, F) bytes); a wait that runs out sets *error.
template <typename V> size_t fields_workspace(int N, int F) {
    const size_t HP = row_pitch(N);
    return sizeof(V) * (3ull * N * N * HP * (size_t)F + (size_t)fields_ring_slots<V>(N, F) * N * HP) +
           sizeof(unsigned) * (1 + 6ull * N * (size_t)F);
}

template <typename R, typename OutT, int N>
int run_fft_fields(const bspline_plan_s* p, int F, const void* const* in_fields, void* const* out_fields, void* work,
                   unsigned* error, cudaStream_t st) {
    using V = typename Cx<R>::T;
    constexpr int NL = tile_lines<R>();
    constexpr int T = threads_for<N, NL>();
    constexpr int H = N / 2 + 1, HP = row_pitch(N);
    const R* c = nullptr;
    const V* tw = nullptr;
    if constexpr (sizeof(R) == 8) {
        c = p->d_c64;
        tw = p->d_tw64;
    } else {
        c = p->d_c32;
        tw = p->d_tw32;
    }
    V* w = reinterpret_cast<V*>(work);
    int rc;
    {
        constexpr int NLX = 2 * NL;
        auto k = fft_x_prefilter<R, N, NLX>;
        const size_t sm = sizeof(V) * (N + (size_t)N * NLX);
        if ((rc = set_smem(k, sm))) return rc;
        const long long tiles = ((long long)N * H + NLX - 1) / NLX;
        k<<<(unsigned)(3LL * F * tiles), threads_for<N, NLX>(), sm, st>>>(
            nullptr, w, c, tw, 0, reinterpret_cast<const V* const*>(in_fields), p->band);
    }
    {
        auto k = fft_yz_fused<R, OutT, N, NL, kYCols * NL>;
        constexpr int NR = z_rows<R, N, NL>();
        const size_t sm = sizeof(V) * yz_smem_elems<R, N, NL, kYCols * NL>();
        if ((rc = set_smem(k, sm))) return rc;
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, T, sm);
        if (e != cudaSuccess) return set_cuda_error(e);
        const int ipp = (H + kYCols * NL - 1) / (kYCols * NL) + N / NR;
        const long long planes = 3LL * N * F;
        const long long items = planes * ipp;
        const long long grid = std::min<long long>(items, (long long)std::max(per_sm, 1) * p->sms);
        const long long slots = fields_ring_slots<V>(N, F);
        const int lag = (int)std::min<long long>(std::min<long long>(slots / 2, planes),
                                                 (2 * grid + ipp - 1) / ipp + 2);
        V* ring = w + 3LL * N * N * HP * F;
        unsigned* ctr = reinterpret_cast<unsigned*>(ring + slots * N * HP);
        e = cudaMemsetAsync(ctr, 0, sizeof(unsigned) * (1 + 2 * planes), st);
        if (e != cudaSuccess) return set_cuda_error(e);
        k<<<(unsigned)grid, T, sm, st>>>(w, nullptr, ring, tw, ctr, error, lag, 2 * lag, 0, 0LL, planes,
                                         reinterpret_cast<OutT* const*>(out_fields), p->band);
    }
    return set_cuda_error(cudaGetLastError());
}

template <int N>
int run_n_fields(const bspline_plan_s* p, int F, const void* const* in_fields, void* const* out_fields, void* work,
                 unsigned* error, cudaStream_t st) {
    switch (p->dtype) {
        case BSPLINE_F64: return run_fft_fields<double, double, N>(p, F, in_fields, out_fields, work, error, st);
        case BSPLINE_F32: return run_fft_fields<float, float, N>(p, F, in_fields, out_fields, work, error, st);
        case BSPLINE_BF16:
            return run_fft_fields<float, __nv_bfloat16, N>(p, F, in_fields, out_fields, work, error, st);
    }
    return BSPLINE_ERR_INVALID_ARG;
}

template <int N> int run_n(bspline_plan_s* p, const void* u_hat, void* coeffs, int c0, int c1) {
    switch (p->dtype) {
        case BSPLINE_F64: return run_fft<double, double, N>(p, u_hat, coeffs, c0, c1);
        case BSPLINE_F32: return run_fft<float, float, N>(p, u_hat, coeffs, c0, c1);
        case BSPLINE_BF16: return run_fft<float, __nv_bfloat16, N>(p, u_hat, coeffs, c0, c1);
    }
    return BSPLINE_ERR_INVALID_ARG;
}

}  // namespace

size_t coeffs_workspace_bytes(const bspline_plan_s* p) {
    return p->dtype == BSPLINE_F64 ? transform_workspace<double2>(p->N) : transform_workspace<float2>(p->N);
}

int launch_coeffs_range(bspline_plan_s* p, const void* u_hat, void* coeffs, int c0, int c1) {
    int rc = p->work.grow(coeffs_workspace_bytes(p));
    if (rc) return rc;
    if (c0 == 0) {
        cudaError_t e = cudaMemsetAsync(p->d_status + kStatusTransformTimeout, 0, sizeof(unsigned long long), p->stream);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    switch (p->N) {
        case 8: return run_n<8>(p, u_hat, coeffs, c0, c1);
        case 16: return run_n<16>(p, u_hat, coeffs, c0, c1);
        case 32: return run_n<32>(p, u_hat, coeffs, c0, c1);
        case 64: return run_n<64>(p, u_hat, coeffs, c0, c1);
        case 128: return run_n<128>(p, u_hat, coeffs, c0, c1);
        case 256: return run_n<256>(p, u_hat, coeffs, c0, c1);
        case 512: return run_n<512>(p, u_hat, coeffs, c0, c1);
        case 1024: return run_n<1024>(p, u_hat, coeffs, c0, c1);
        case 48: return run_n<48>(p, u_hat, coeffs, c0, c1);
        case 96: return run_n<96>(p, u_hat, coeffs, c0, c1);
        case 192: return run_n<192>(p, u_hat, coeffs, c0, c1);
        case 384: return run_n<384>(p, u_hat, coeffs, c0, c1);
        case 768: return run_n<768>(p, u_hat, coeffs, c0, c1);
    }
    return BSPLINE_ERR_UNSUPPORTED_N;
}

int launch_coeffs(bspline_plan_s* p, const void* u_hat, void* coeffs) { return launch_coeffs_range(p, u_hat, coeffs, 0, 3); }

size_t coeffs_fields_workspace_bytes(const bspline_plan_s* p, int F) {
    return p->dtype == BSPLINE_F64 ? fields_workspace<double2>(p->N, F) : fields_workspace<float2>(p->N, F);
}

int launch_coeffs_fields(const bspline_plan_s* p, int F, const void* const* in_fields, void* const* out_fields,
                         void* work, unsigned* error, cudaStream_t st) {
    switch (p->N) {
        case 8: return run_n_fields<8>(p, F, in_fields, out_fields, work, error, st);
        case 16: return run_n_fields<16>(p, F, in_fields, out_fields, work, error, st);
        case 32: return run_n_fields<32>(p, F, in_fields, out_fields, work, error, st);
        case 64: return run_n_fields<64>(p, F, in_fields, out_fields, work, error, st);
        case 128: return run_n_fields<128>(p, F, in_fields, out_fields, work, error, st);
        case 256: return run_n_fields<256>(p, F, in_fields, out_fields, work, error, st);
        case 512: return run_n_fields<512>(p, F, in_fields, out_fields, work, error, st);
        case 1024: return run_n_fields<1024>(p, F, in_fields, out_fields, work, error, st);
        case 48: return run_n_fields<48>(p, F, in_fields, out_fields, work, error, st);
        case 96: return run_n_fields<96>(p, F, in_fields, out_fields, work, error, st);
        case 192: return run_n_fields<192>(p, F, in_fields, out_fields, work, error, st);
        case 384: return run_n_fields<384>(p, F, in_fields, out_fields, work, error, st);
        case 768: return run_n_fields<768>(p, F, in_fields, out_fields, work, error, st);
    }
    return BSPLINE_ERR_UNSUPPORTED_N;
}

}  // namespace bs

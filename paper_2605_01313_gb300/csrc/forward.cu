// Coefficients from samples on the arrival grid (Sec. 3-4): the inverse of the
// evaluation at the grid points, so that values at the arrival grid can be
// carried to the departure points in one call.  The samples of Grid [0]
// (theta_j = (j + 1/2) pi / n_lat, phi_k = 2 pi k / n_lon) are extended to the
// doubled sphere by the field's parity (row 2 n_lat - 1 - j, half a turn in
// longitude, sign +1 for scalars and -1 for wind components), then
//   c_{n,m} = (1 / (N1 N2)) sum_{j,k} f_ext(phi_k, theta_j) e^{-i (m phi_k + n theta_j)}.
//
// Two passes on the FFT engine of the NUFFT (sign -1 by conjugation):
//  k_fwd_phi   the rows: two real rows of a field form one complex sequence,
//              whose transform splits into the two rows' spectra F_m(theta_j);
//  k_fwd_theta the columns m >= 0 (the rest by conjugate symmetry, the samples
//              being real): the doubled column (F_m(theta_j) for j < n_lat,
//              parity (-1)^m F_m(theta_{N2-1-j}) above, the half turn being the
//              factor (-1)^m), its transform, the half-cell phase e^{-i pi n / N2}
//              and the 1 / (N1 N2) scale, written in the centred layout of
//              dfsnufft_execute.
//
// FP64 plans run both passes in double-single arithmetic (df32.cuh), as their
// inverse passes do: each line's samples are scaled by the power of two that
// brings its largest into [1, 2) on load, and the coefficients, written in
// FP64, are scaled back.
#include <type_traits>

#include "df32.cuh"
#include "fft_core.cuh"

using namespace dfs_fft;

namespace {

template <typename C> __device__ __forceinline__ C conjc(C a) { return cmake(a.x, -a.y); }
template <typename C, typename R> __device__ __forceinline__ C cscale2(C a, R s) {
    return cmake(a.x * s, a.y * s);
}

// Storage types of a pass in arithmetic type R: samples In, coefficients Out.
template <typename R> struct FwdIO {
    typedef R In;
    typedef typename CxT<R>::type Out;
};
template <> struct FwdIO<df32> {
    typedef double In;
    typedef double2 Out;
};
// A sample as the pass's real type R (double-single: times 2^-sh, split).
template <typename R>
__device__ __forceinline__ R fwd_in(typename FwdIO<R>::In v, int) { return v; }
template <> __device__ __forceinline__ df32 fwd_in<df32>(double v, int sh) {
    return split_double(df_scale_down(v, sh));
}
// A coefficient to its storage (double-single: hi + lo in FP64, times 2^sh).
template <typename C> __device__ __forceinline__ C fwd_out(C v, int) { return v; }
__device__ __forceinline__ double2 fwd_out(dfc v, int sh) {
    const double s = df_pow2(sh);
    return make_double2(((double)v.x.hi + (double)v.x.lo) * s,
                        ((double)v.y.hi + (double)v.y.lo) * s);
}

struct FwdArgs {
    int n_lat, N1, N2;
    int log1, log2;           // log2 N1, log2 N2
    int tws1, tws2;           // twiddle strides: tw1[k << tws1] = e^{2 pi i k / N1}
    int F;                    // fields per member
    int CB, lcb;              // columns per CTA (theta pass), a power of two, and its log2
    int full;                 // 0: of the columns m < 0 only the Nyquist row is written
    int K;                    // Gauss-Legendre form: complex slots per line and class
    long long gpitch;         // and complex per class row (>= lines K)
};

// grid (n_lat / 2, lines); block N1 / E threads.  Rows 2r and 2r + 1 of line f.
// LOG > 0: length 2^LOG at compile time with the stage-ordered table stw.
// GL: the spectra go to the two parity classes of the Gauss-Legendre solve
// (gauss.cu): mode m of a field of parity s is in class 0 when s (-1)^m = +1
// (spec), else in class 1 (g1); row j, slot line * K + m / 2 of an n_lat x
// (lines K) complex matrix.
// emax (double-single passes): each line's largest sample exponent.
template <typename R, int E, int LOG, bool GL>
__global__ void __launch_bounds__(512) k_fwd_phi(FwdArgs a,
                                                 const typename FwdIO<R>::In *__restrict__ samples,
                                                 const typename CxT<R>::type *__restrict__ tw1,
                                                 const typename CxT<R>::type *__restrict__ stw,
                                                 typename CxT<R>::type *__restrict__ spec,
                                                 const int *__restrict__ parity,
                                                 typename CxT<R>::type *__restrict__ g1,
                                                 const int *__restrict__ emax) {
    typedef typename CxT<R>::type C;
    typedef typename FwdIO<R>::In In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    C *z = sm + region_len<C>(a.N1);                   // the pair's transform
    const int f = blockIdx.y;
    const int j = 2 * blockIdx.x;
    const int t = threadIdx.x;
    const In *x = samples + ((size_t)f * a.n_lat + j) * a.N1;
    const In *y = x + a.N1;
    const int sh = emax ? df_line_shift(emax[f]) : 0;
    // DFT_-(x + i y) = conj(DFT_+(conj(x + i y)))
    auto ld = [&](int i) -> C { return cmake(fwd_in<R>(x[i], sh), -fwd_in<R>(y[i], sh)); };
    auto st = [&](int k, C v) { z[k] = conjc(v); };
    if constexpr (LOG > 0) line_fft_ct<LOG, E>(stw, sm, t, ld, st);
    else line_fft<E>(a.log1, tw1, a.tws1, sm, t, ld, st);
    __syncthreads();
    // X_m = (Z_m + conj Z_{-m}) / 2,  Y_m = (Z_m - conj Z_{-m}) / (2i)
    if constexpr (GL) {
        const int pneg = parity[f % a.F] < 0;
        const size_t pitch = (size_t)a.gpitch;                    // complex per class row
        for (int m = t; m <= a.N1 / 2; m += blockDim.x) {
            const C zp = z[m], zm = conjc(z[(a.N1 - m) & (a.N1 - 1)]);
            C *g = (pneg == (m & 1)) ? spec : g1;
            const size_t o = (size_t)j * pitch + (size_t)f * a.K + (m >> 1);
            g[o] = cmake((R)0.5 * (zp.x + zm.x), (R)0.5 * (zp.y + zm.y));
            g[o + pitch] = cmake((R)0.5 * (zp.y - zm.y), (R)-0.5 * (zp.x - zm.x));
            if (m == a.N1 / 2) {           // the other class has no mode in this slot
                C *h = g == spec ? g1 : spec;
                h[o] = cmake((R)0, (R)0);
                h[o + pitch] = cmake((R)0, (R)0);
            }
        }
    } else {
        C *sx = spec + ((size_t)f * a.n_lat + j) * a.N1;
        C *sy = sx + a.N1;
        for (int m = t; m <= a.N1 / 2; m += blockDim.x) {      // the theta pass reads m <= N1/2
            const C zp = z[m], zm = conjc(z[(a.N1 - m) & (a.N1 - 1)]);
            sx[m] = cmake((R)0.5 * (zp.x + zm.x), (R)0.5 * (zp.y + zm.y));
            sy[m] = cmake((R)0.5 * (zp.y - zm.y), (R)-0.5 * (zp.x - zm.x));
        }
    }
}

// Persistent: grid = min(tasks, resident CTAs); a task is one block of CB
// adjacent columns of one line (tasks = ceil((N1/2 + 1) / CB) x lines), CTA i
// takes tasks i, i + gridDim.x, ...  Block CB * N2/E threads, thread = (t, c), c
// fastest.  The samples are real, so c_{-n,-m} = conj c_{n,m}: only the modes
// m = 0..N1/2 (DFT index) are transformed, and each column 0 < m < N1/2 also
// writes its mirror column -m.  LOG > 0: length 2^LOG at compile time.
// A task's n_lat x CB row spectra are staged in shared memory row by row (the CB
// columns of a row are one contiguous read of CB * sizeof(C) >= 16 bytes, a whole
// 32-byte sector for FP32 at CB = 4), by asynchronous 16-byte copies issued one
// task ahead into the other of two buffers, so that the next block's reads are
// in flight while this one is transformed; both halves of the doubled column are
// read from there, so each spectrum value leaves HBM once.  The copies of the
// block holding m = N1/2 also read the CB - 1 columns after it (inside the row,
// as N1 >= 16 > CB); their values are never used.
template <typename R, int E, int LOG>
__global__ void __launch_bounds__(sizeof(R) == 4 ? 1024 : 512) k_fwd_theta(FwdArgs a,
                                                   const typename CxT<R>::type *__restrict__ spec,
                                                   const int *__restrict__ parity,
                                                   const typename CxT<R>::type *__restrict__ tw2,
                                                   const typename CxT<R>::type *__restrict__ stw,
                                                   typename FwdIO<R>::Out *__restrict__ coef,
                                                   int nblk, int ntask,
                                                   const int *__restrict__ emax) {
    dfs_grid_wait();
    typedef typename CxT<R>::type C;
    typedef typename FwdIO<R>::Out CO;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *smem = reinterpret_cast<C *>(smem_raw);
    const int c = threadIdx.x & (a.CB - 1);
    const int t = threadIdx.x >> a.lcb;
    C *sm = smem + (size_t)c * region_stride<C>(a.N2, a.CB);
    C *stage = smem + (size_t)a.CB * region_len<C>(a.N2);   // 2 x (n_lat x CB), c fastest
    const int per_buf = a.n_lat << a.lcb;
    // 16-byte chunks of a staged row: CB * sizeof(C) / 16, a power of two
    const int lcpr = a.lcb + (sizeof(C) == 16 ? 0 : -1);
    auto prefetch = [&](int task, C *buf) {
        const int f = task / nblk;
        const int m0 = (task - f * nblk) * a.CB;
        const char *src = reinterpret_cast<const char *>(spec + (size_t)f * a.n_lat * a.N1 + m0);
        const size_t pitch = (size_t)a.N1 * sizeof(C);
        const int total = a.n_lat << lcpr;
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            const int r = q >> lcpr;
            cp_async_16(reinterpret_cast<char *>(buf) + (size_t)q * 16,
                        src + (size_t)r * pitch + (size_t)(q - (r << lcpr)) * 16);
        }
        cp_async_commit();
    };
    // 1 / (N1 N2), a power of two
    const R scale = R(ldexpf(1.f, -(a.log1 + a.log2)));
    // n2 = N2 << tws2 is a power of two: indices of tw2 are taken mod n2 by a mask
    const int tw_mask = (a.N2 << a.tws2) - 1;
    const int tw_step = 1 << (a.tws2 - 1);
    if ((int)blockIdx.x < ntask) prefetch(blockIdx.x, stage);
    int it = 0;
    for (int task = blockIdx.x; task < ntask; task += gridDim.x, ++it) {
        C *in = stage + (size_t)(it & 1) * per_buf;
        const int nxt = task + gridDim.x;
        if (nxt < ntask) {
            prefetch(nxt, stage + (size_t)((it + 1) & 1) * per_buf);
            cp_async_wait_group<1>();              // this task's copies have landed
        } else {
            cp_async_wait_group<0>();
        }
        __syncthreads();                           // everyone's have
        const int f = task / nblk;
        const int m = (task - f * nblk) * a.CB + c;          // DFT index of the phi mode
        const bool ok = m <= a.N1 / 2;
        // the upper half of the doubled column: parity (-1)^m times the mirrored row
        const R sgn = (R)(parity[f % a.F] < 0 ? -1 : 1) * ((m & 1) ? (R)-1 : (R)1);
        auto ld = [&](int i) -> C {
            if (!ok) return cmake((R)0, (R)0);
            const C v = i < a.n_lat ? in[(i << a.lcb) + c]
                                    : cscale2(in[((a.N2 - 1 - i) << a.lcb) + c], sgn);
            return conjc(v);
        };
        const int mc = m < a.N1 / 2 ? m + a.N1 / 2 : m - a.N1 / 2;   // centred column
        CO *out = coef + (size_t)f * a.N2 * a.N1 + mc;
        CO *mirror = coef + (size_t)f * a.N2 * a.N1 + (a.N1 - mc);   // column of -m
        const int sh = emax ? df_line_shift(emax[f]) : 0;
        const bool has_mirror = ok && m > 0 && m < a.N1 / 2;
        auto st = [&](int k, C v) {
            if (!ok) return;
            // mode n = k (k < N2/2) or k - N2; half-cell phase e^{-i pi n / N2}:
            // tw2 holds e^{+2 pi i k / n2} with n2 = N2 << tws2, so the phase is
            // conj(tw2[n << (tws2 - 1)]) taken mod n2
            const int n = k < a.N2 / 2 ? k : k - a.N2;
            const C ph = conjc(tw2[(n * tw_step) & tw_mask]);
            const C cv = cscale2(cmul(conjc(v), ph), scale);
            out[(size_t)(n + a.N2 / 2) * a.N1] = fwd_out(cv, sh);
            // c_{-n,-m} = conj c_{n,m}; the half-cell grid makes the sum antiperiodic
            // in n (c_{n+N2,m} = -c_{n,m}), so the row n = -N2/2 of column -m is
            // -conj c_{-N2/2,m}
            if (has_mirror) {
                if (n > -a.N2 / 2) {
                    if (a.full) mirror[(size_t)(a.N2 / 2 - n) * a.N1] = fwd_out(conjc(cv), sh);
                } else {
                    mirror[0] = fwd_out(cmake(-cv.x, cv.y), sh);
                }
            }
        };
        if constexpr (LOG > 0) line_fft_ct<LOG, E>(stw, sm, t, ld, st);
        else line_fft<E>(a.log2, tw2, a.tws2, sm, t, ld, st);
        __syncthreads();        // reads of this buffer and of sm end before they are refilled
    }
}

// The plan's tables for the pass's arithmetic: twiddles of lengths n1 and n2
// and the stage-ordered table of length n1/2 (double-single copies for df32).
template <typename R> struct FwdTables {
    const void *tw1, *tw2, *stw_phi, *stw_half;
    explicit FwdTables(dfsnufft_plan p) {
        const bool df = std::is_same<R, df32>::value;
        tw1 = df ? p->d_df_tw1 : p->d_tw1;
        tw2 = df ? p->d_df_tw2 : p->d_tw2;
        stw_phi = df ? p->d_df_stw_phi : p->d_stw_phi;
        stw_half = df ? p->d_df_stw_half : p->d_stw_theta;     // length n2 / 2
    }
};

template <typename R, int LOG>
cudaError_t run_fwd_phi(dfsnufft_plan p, const FwdArgs &a, const void *samples, void *spec,
                        int lines, const int *d_parity = nullptr, void *g1 = nullptr,
                        const int *emax = nullptr) {
    typedef typename CxT<R>::type C;
    typedef typename FwdIO<R>::In In;
    constexpr int E = DFS_FFT_E;
    const FwdTables<R> tb(p);
    const int threads = a.N1 / E;
    const size_t smem = sizeof(C) * (size_t)(region_len<C>(a.N1) + a.N1);
    const dim3 grid(a.n_lat / 2, lines);
    cudaError_t e;
    if (g1) {
        e = allow_smem(k_fwd_phi<R, E, LOG, true>, smem);
        if (e) return e;
        k_fwd_phi<R, E, LOG, true><<<grid, threads, smem, p->stream>>>(
            a, (const In *)samples, (const C *)tb.tw1, (const C *)tb.stw_phi, (C *)spec,
            d_parity, (C *)g1, emax);
    } else {
        e = allow_smem(k_fwd_phi<R, E, LOG, false>, smem);
        if (e) return e;
        k_fwd_phi<R, E, LOG, false><<<grid, threads, smem, p->stream>>>(
            a, (const In *)samples, (const C *)tb.tw1, (const C *)tb.stw_phi, (C *)spec,
            nullptr, nullptr, emax);
    }
    return cudaGetLastError();
}

template <typename R, int LOG>
cudaError_t run_fwd_theta(dfsnufft_plan p, const FwdArgs &a, const void *spec,
                          const int *d_parity, void *coeffs, int lines,
                          const int *emax = nullptr) {
    typedef typename CxT<R>::type C;
    typedef typename FwdIO<R>::Out CO;
    constexpr int E = DFS_FFT_E;
    const FwdTables<R> tb(p);
    const int T = a.N2 / E;
    const size_t smem = sizeof(C) * (size_t)a.CB * (region_len<C>(a.N2) + 2 * (size_t)a.n_lat);
    cudaError_t e = allow_smem(k_fwd_theta<R, E, LOG>, smem);
    if (e) return e;
    const int nblk = (a.N1 / 2 + 1 + a.CB - 1) / a.CB;
    const int ntask = nblk * lines;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fwd_theta<R, E, LOG>, a.CB * T,
                                                      smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    const long long want = (long long)p->num_sms * occ;
    const int ctas = (int)(want < ntask ? want : ntask);
    return dfs_launch_dependent(k_fwd_theta<R, E, LOG>, dim3(ctas), dim3(a.CB * T), smem,
                                p->stream, a, (const C *)spec, d_parity, (const C *)tb.tw2,
                                (const C *)tb.stw_half, (CO *)coeffs, nblk, ntask, emax);
}

template <typename R>
cudaError_t launch_forward(dfsnufft_plan p, const void *samples, const int *d_parity,
                           void *coeffs, void *spec, bool full) {
    constexpr int E = DFS_FFT_E;
    const dfsnufft_params &q = p->prm;
    FwdArgs a;
    memset(&a, 0, sizeof(a));
    a.n_lat = q.n_lat;
    a.N1 = q.N1;
    a.N2 = q.N2;
    a.log1 = ilog2(q.N1);
    a.log2 = ilog2(q.N2);
    a.tws1 = ilog2(q.n1) - a.log1;
    a.tws2 = ilog2(q.n2) - a.log2;
    a.F = p->n_fields;
    a.full = full ? 1 : 0;
    // columns per CTA: CTAs of 1024 threads for FP32 (four FP32 columns of a row
    // fill a 32-byte sector), of 512 for FP64 (two columns do)
    const int T = q.N2 / E;
    int cb = (sizeof(R) == 4 ? 1024 : 512) / T;
    if (cb < 1) cb = 1;
    if (cb > 8) cb = 8;
    a.CB = cb;
    a.lcb = ilog2(cb);
    const int lines = p->n_members * p->n_fields;
    constexpr bool df = std::is_same<R, df32>::value;
    const FwdTables<R> tb(p);
    // the plan's stage-ordered tables are for lengths n1/2 and n2/2: they serve
    // the compile-time drivers when the fine grid is twice the modes
    const bool ct1 = tb.stw_phi && q.n1 == 2 * q.N1 && a.log1 >= 9 && a.log1 <= 11;
    const bool ct2 = tb.stw_half && q.n2 == 2 * q.N2 && a.log2 >= 9 && a.log2 <= 11;
    cudaError_t e;
    const int *emax = nullptr;
    if (df) {
        // each line's largest sample (n_lat x N1 reals, read as pairs)
        e = dfs_launch_line_maxexp(p, samples, q.n_lat * q.N1 / 2, q.n_lat, 0, 0, lines);
        if (e) return e;
        emax = p->d_emax;
    }
    switch (ct1 ? a.log1 : 0) {
        case 9: e = run_fwd_phi<R, 9>(p, a, samples, spec, lines, nullptr, nullptr, emax); break;
        case 10: e = run_fwd_phi<R, 10>(p, a, samples, spec, lines, nullptr, nullptr, emax); break;
        case 11: e = run_fwd_phi<R, 11>(p, a, samples, spec, lines, nullptr, nullptr, emax); break;
        default: e = run_fwd_phi<R, 0>(p, a, samples, spec, lines, nullptr, nullptr, emax); break;
    }
    if (e) return e;
    switch (ct2 ? a.log2 : 0) {
        case 9: return run_fwd_theta<R, 9>(p, a, spec, d_parity, coeffs, lines, emax);
        case 10: return run_fwd_theta<R, 10>(p, a, spec, d_parity, coeffs, lines, emax);
        case 11: return run_fwd_theta<R, 11>(p, a, spec, d_parity, coeffs, lines, emax);
        default: return run_fwd_theta<R, 0>(p, a, spec, d_parity, coeffs, lines, emax);
    }
}

}  // namespace

// The sizes the forward transform takes: N1 = n_lon and N2 = 2 n_lat powers of
// two with 16 <= N <= 4096 (one line of at most 512 threads at E = 8), n_lat even.
bool dfs_forward_supported(const dfsnufft_params &q) {
    auto ok = [](int n) { return (n & (n - 1)) == 0 && n >= 16 && n <= 4096; };
    return ok(q.N1) && ok(q.N2) && (q.n_lat % 2) == 0;
}

cudaError_t dfs_launch_forward(dfsnufft_plan p, const void *samples, const int *d_parity,
                               void *coeffs, bool full) {
    // the row spectra (lines x n_lat x N1 complex) fit in the theta-pass buffer,
    // which the execute that follows overwrites only later in stream order
    // FP64 plans whose inverse passes run in double-single run these too
    if (p->gdf) return launch_forward<df32>(p, samples, d_parity, coeffs, p->d_T, full);
    return p->prm.dtype == DFSNUFFT_F64
               ? launch_forward<double>(p, samples, d_parity, coeffs, p->d_T, full)
               : launch_forward<float>(p, samples, d_parity, coeffs, p->d_T, full);
}

// The longitude pass of the Gauss-Legendre form (gauss.cu): the row spectra of
// every line into the two parity classes g0 and g1 (n_lat x (lines K) complex).
template <typename R>
static cudaError_t launch_fwd_phi_gl(dfsnufft_plan p, const void *samples, const int *d_parity,
                                     void *g0, void *g1, int K, long long pitch) {
    const dfsnufft_params &q = p->prm;
    FwdArgs a;
    memset(&a, 0, sizeof(a));
    a.n_lat = q.n_lat;
    a.N1 = q.N1;
    a.N2 = q.N2;
    a.log1 = ilog2(q.N1);
    a.log2 = ilog2(q.N2);
    a.tws1 = ilog2(q.n1) - a.log1;
    a.tws2 = ilog2(q.n2) - a.log2;
    a.F = p->n_fields;
    a.K = K;
    a.gpitch = pitch;
    const int lines = p->n_members * p->n_fields;
    const bool ct1 = p->d_stw_phi && q.n1 == 2 * q.N1 && a.log1 >= 9 && a.log1 <= 11;
    switch (ct1 ? a.log1 : 0) {
        case 9: return run_fwd_phi<R, 9>(p, a, samples, g0, lines, d_parity, g1);
        case 10: return run_fwd_phi<R, 10>(p, a, samples, g0, lines, d_parity, g1);
        case 11: return run_fwd_phi<R, 11>(p, a, samples, g0, lines, d_parity, g1);
        default: return run_fwd_phi<R, 0>(p, a, samples, g0, lines, d_parity, g1);
    }
}

cudaError_t dfs_launch_fwd_phi_gl(dfsnufft_plan p, const void *samples, const int *d_parity,
                                  void *g0, void *g1, int K, long long pitch) {
    return p->prm.dtype == DFSNUFFT_F64
               ? launch_fwd_phi_gl<double>(p, samples, d_parity, g0, g1, K, pitch)
               : launch_fwd_phi_gl<float>(p, samples, d_parity, g0, g1, K, pitch);
}

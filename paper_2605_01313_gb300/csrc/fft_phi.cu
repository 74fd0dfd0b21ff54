// phi pass: the row FFTs of the oversampled 2-D inverse FFT (sign +1), the
// last FFT stage of the type-2 NUFFT evaluating Eq. 5.3 (Sec. 5).
//
// Only the real part of the fine grid is needed (the interpolation weights are
// real and the values are Re v), so each row is a complex-to-real transform:
// Re g(j) = sum_k H_k e^{2 pi i k j / n1} with H_k = (T_k + conj T_{-k}) / 2
// Hermitian.  With M = n1 / 2 and Z_k = (H_k + H_{k+M}) + i e^{2 pi i k / n1}
// (H_k - H_{k+M}), the length-M inverse FFT z of Z gives
// Re g(2j) = Re z_j and Re g(2j+1) = Im z_j.  T_k is the theta-pass value at
// phi-mode k mod n1 (zero outside the N1 modes).  A real-field plan's theta
// pass already transformed the Hermitian part of the coefficients, so its row
// holds H_k itself for k = 0..N1/2, and H_{-k} = conj H_k.  Each CTA handles CB
// rows inside the plan's needed row range; the row's values are staged in
// shared memory first, since every one of them enters two Z_k.
#include <type_traits>

#include "fft_core.cuh"
#include "df32.cuh"

using namespace dfs_fft;

namespace {

struct PhiArgs {
    int N1, n1, logm, n2;     // logm = log2(n1 / 2)
    int CB;                   // rows per CTA (divides DFS_ROW_BLOCK)
    int F;                    // fields per member (line f belongs to member f / F)
    int tcols, tpitch;        // theta-pass columns per row and row pitch
    int line0;                // first line (blockIdx.y = line - line0)
};

// grid (n2 / CB, lines); block CB * M/E threads, thread = (t, c) with t fastest.
// LOGM > 0 fixes the transform length at compile time; 0 takes it from a.logm.
// DF (FP64 plans): each fine-grid value is written as the double-single pair
// (hi, lo) of df32.cuh, the input of the double-single interpolation.
template <typename R, int E, int MAXT, int MINB, int LOGM, bool HERM, bool DF = false>
__global__ void __launch_bounds__(MAXT, MINB)
    k_phi_pass(PhiArgs a, const typename CxT<R>::type *__restrict__ in,
               const typename CxT<R>::type *__restrict__ tw,
               const typename CxT<R>::type *__restrict__ stw, const int2 *__restrict__ rowrange,
               R *__restrict__ grid) {
    dfs_grid_wait();
    typedef typename CxT<R>::type C;
    const int row0 = blockIdx.x * a.CB;
    const int2 rr = rowrange[(a.line0 + blockIdx.y) / a.F];
    // whole CTA (within one row block): no stencil touches these rows
    if (((row0 - rr.x) & (a.n2 - 1)) >= rr.y) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *smem = reinterpret_cast<C *>(smem_raw);
    const int M = LOGM ? (1 << LOGM) : (1 << a.logm);
    const int T = M / E;
    const int t = threadIdx.x % T;
    const int c = threadIdx.x / T;
    const int row = row0 + c;
    const int f = a.line0 + blockIdx.y;
    const C *src = in + ((size_t)f * a.n2 + row) * a.tpitch;
    R *dst = grid + ((size_t)f * a.n2 + row) * a.n1;
    const int half = a.N1 / 2;
    const int nmask = a.n1 - 1;
    C *sm = smem + (size_t)c * region_len<C>(M);
    C *srow = smem + (size_t)a.CB * region_len<C>(M) + (size_t)c * a.tcols;
    for (int i = t; i < a.tcols; i += T) srow[i] = src[i];
    __syncthreads();
    auto hval = [&](int k) -> C {              // real-field rows: H_k, k taken mod n1
        k &= nmask;
        if (k <= half) return srow[k];
        if (k >= a.n1 - half) {
            const C v = srow[a.n1 - k];
            return cmake(v.x, -v.y);
        }
        return cmake((R)0, (R)0);
    };
    auto tval = [&](int k) -> C {              // T_k, k taken mod n1
        k &= nmask;
        int m;
        if (k < half) m = k;
        else if (k >= a.n1 - half) m = k - a.n1;
        else return cmake((R)0, (R)0);
        return srow[m + half];
    };
    auto ld = [&](int k) -> C {
        if constexpr (HERM) {
            const C h0 = hval(k), h1 = hval(k + M);
            const C d = cmul(cmake(h0.x - h1.x, h0.y - h1.y), ldt(&tw[k]));
            return cmake(h0.x + h1.x - d.y, h0.y + h1.y + d.x);
        }
        const C t0 = tval(k), t1 = tval(-k), t2 = tval(k + M), t3 = tval(M - k);
        // 2 H_k = T_k + conj T_{-k},  2 H_{k+M} = T_{k+M} + conj T_{M-k}
        const C h0 = cmake(t0.x + t1.x, t0.y - t1.y);
        const C h1 = cmake(t2.x + t3.x, t2.y - t3.y);
        const C d = cmul(cmake(h0.x - h1.x, h0.y - h1.y), ldt(&tw[k]));
        // (h0 + h1 + i d) / 2
        return cmake((R)0.5 * (h0.x + h1.x - d.y), (R)0.5 * (h0.y + h1.y + d.x));
    };
    auto st = [&](int j, C z) {
        if constexpr (std::is_same<R, df32>::value) {       // already double-single
            reinterpret_cast<float4 *>(dst)[j] = make_float4(z.x.hi, z.x.lo, z.y.hi, z.y.lo);
        } else if constexpr (DF) {
            const df32 h0 = split_double(z.x), h1 = split_double(z.y);
            reinterpret_cast<float4 *>(dst)[j] = make_float4(h0.hi, h0.lo, h1.hi, h1.lo);
        } else {
            reinterpret_cast<C *>(dst)[j] = z;
        }
    };
    if constexpr (LOGM > 0) line_fft_ct<LOGM, E>(stw, sm, t, ld, st);
    else line_fft<E>(a.logm, tw, 1, sm, t, ld, st);
}

// FP32 rows at compile-time lengths: each thread group transforms two rows
// at once (line_fft_ct2: the twiddles, the index arithmetic and the barriers
// serve both).  grid (n2 / CB, lines), CB = 2 x threads / (M/E) rows a CTA.
template <int E, int MAXT, int MINB, int LOGM, bool HERM>
__global__ void __launch_bounds__(MAXT, MINB)
    k_phi_pass2(PhiArgs a, const float2 *__restrict__ in, const float2 *__restrict__ tw,
                const float2 *__restrict__ stw, const int2 *__restrict__ rowrange,
                float *__restrict__ grid) {
    dfs_grid_wait();
    typedef float2 C;
    const int row0 = blockIdx.x * a.CB;
    const int2 rr = rowrange[(a.line0 + blockIdx.y) / a.F];
    if (((row0 - rr.x) & (a.n2 - 1)) >= rr.y) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *smem = reinterpret_cast<C *>(smem_raw);
    constexpr int M = 1 << LOGM;
    constexpr int T = M / E;
    const int t = threadIdx.x % T;
    const int c = threadIdx.x / T;                 // row pair
    const int row = row0 + 2 * c;
    const int f = a.line0 + blockIdx.y;
    const int half = a.N1 / 2;
    const int nmask = a.n1 - 1;
    const C *src = in + ((size_t)f * a.n2 + row) * a.tpitch;
    float *dst = grid + ((size_t)f * a.n2 + row) * a.n1;
    C *sm0 = smem + (size_t)(2 * c) * region_len<C>(M);
    C *sm1 = sm0 + region_len<C>(M);
    C *srow0 = smem + (size_t)a.CB * region_len<C>(M) + (size_t)(2 * c) * a.tcols;
    C *srow1 = srow0 + a.tcols;
    for (int i = t; i < a.tcols; i += T) {
        srow0[i] = src[i];
        srow1[i] = src[a.tpitch + i];
    }
    __syncthreads();
    // H_k of a row (k mod n1): real-field rows hold H_k, k = 0..N1/2; general
    // rows hold T_k and H_k = (T_k + conj T_{-k}) / 2
    auto hval = [&](const C *sr, int k) -> C {
        k &= nmask;
        if constexpr (HERM) {
            if (k <= half) return sr[k];
            if (k >= a.n1 - half) {
                const C v = sr[a.n1 - k];
                return cmake(v.x, -v.y);
            }
            return cmake(0.f, 0.f);
        } else {
            auto tv = [&](int kk) -> C {
                kk &= nmask;
                if (kk < half) return sr[kk + half];
                if (kk >= a.n1 - half) return sr[kk - a.n1 + half];
                return cmake(0.f, 0.f);
            };
            const C p = tv(k), m = tv(-k);
            return cmake(0.5f * (p.x + m.x), 0.5f * (p.y - m.y));
        }
    };
    auto ld2 = [&](int k, C &z0, C &z1) {
        const C w = __ldg(&tw[k]);
        const C a0 = hval(srow0, k), b0 = hval(srow0, k + M);
        const C a1 = hval(srow1, k), b1 = hval(srow1, k + M);
        const C d0 = cmul(cmake(a0.x - b0.x, a0.y - b0.y), w);
        const C d1 = cmul(cmake(a1.x - b1.x, a1.y - b1.y), w);
        z0 = cmake(a0.x + b0.x - d0.y, a0.y + b0.y + d0.x);
        z1 = cmake(a1.x + b1.x - d1.y, a1.y + b1.y + d1.x);
    };
    auto st2 = [&](int j, C z0, C z1) {
        reinterpret_cast<C *>(dst)[j] = z0;
        reinterpret_cast<C *>(dst + a.n1)[j] = z1;
    };
    auto none = [] {};
    line_fft_ct2<LOGM, E>(stw, sm0, sm1, t, ld2, st2, none);
}

// Per precision: elements per thread E, threads per CTA at most MAXT with MINB
// resident CTAs (MINBH for the rows of real-field plans); rows longer than
// E x MAXT complex values (FP32 fine grids of 8192 columns) use the wide form of
// MAXTW threads.  Double-single rows of real-field plans fit 64 registers a
// thread without spills, so two CTAs share an SM (C3 FP64 phi pass 305 -> 256
// us); the general rows would spill there and keep one.
template <typename R> struct PhiCfg;
template <> struct PhiCfg<float> {
    static const int E = DFS_FFT_E, MAXT = 256, MINB = 3, MINBH = 3, MAXTW = 512;
};
template <> struct PhiCfg<double> {
    static const int E = DFS_FFT_E, MAXT = 512, MINB = 1, MINBH = 1, MAXTW = 512;
};
template <> struct PhiCfg<df32> {
    static const int E = DFS_FFT_E, MAXT = 512, MINB = 1, MINBH = 2, MAXTW = 512;
};

template <typename R, int MAXT, int MINB, int LOGM, bool HERM, bool DF>
cudaError_t run_phi_df(dfsnufft_plan p, const PhiArgs &a, size_t smem, dim3 grid, int threads) {
    typedef typename CxT<R>::type C;
    constexpr int E = PhiCfg<R>::E;
    cudaError_t e = allow_smem(k_phi_pass<R, E, MAXT, MINB, LOGM, HERM, DF>, smem);
    if (e) return e;
    const bool dfr = std::is_same<R, df32>::value;     // double-single tables
    return dfs_launch_dependent(k_phi_pass<R, E, MAXT, MINB, LOGM, HERM, DF>, grid,
                                dim3(threads), smem, p->stream, a, (const C *)p->d_T,
                                (const C *)(dfr ? p->d_df_tw1 : p->d_tw1),
                                (const C *)(dfr ? p->d_df_stw_phi : p->d_stw_phi),
                                (const int2 *)p->d_rowrange, (R *)p->d_G);
}

// FP64 plans whose interpolation runs in double-single (p->gdf) take the DF form.
template <typename R, int MAXT, int MINB, int LOGM, bool HERM>
cudaError_t run_phi(dfsnufft_plan p, const PhiArgs &a, size_t smem, dim3 grid, int threads) {
    if constexpr (std::is_same<R, double>::value) {
        if (p->gdf) return run_phi_df<R, MAXT, MINB, LOGM, HERM, true>(p, a, smem, grid, threads);
    }
    return run_phi_df<R, MAXT, MINB, LOGM, HERM, false>(p, a, smem, grid, threads);
}

template <typename R, bool HERM>
cudaError_t dispatch_phi(dfsnufft_plan p, const PhiArgs &a, size_t smem, dim3 grid, int threads) {
    constexpr int MAXT = PhiCfg<R>::MAXT, MAXTW = PhiCfg<R>::MAXTW;
    constexpr int MINB = HERM ? PhiCfg<R>::MINBH : PhiCfg<R>::MINB;
    if (threads > MAXT) return run_phi<R, MAXTW, 1, 0, HERM>(p, a, smem, grid, threads);
    // compile-time lengths need the plan's stage-ordered table (double-single
    // for df32)
    if (std::is_same<R, df32>::value ? !p->d_df_stw_phi : !p->d_stw_phi)
        return run_phi<R, MAXT, MINB, 0, HERM>(p, a, smem, grid, threads);
    switch (a.logm) {
        case 9: return run_phi<R, MAXT, MINB, 9, HERM>(p, a, smem, grid, threads);
        case 10: return run_phi<R, MAXT, MINB, 10, HERM>(p, a, smem, grid, threads);
        case 11: return run_phi<R, MAXT, MINB, 11, HERM>(p, a, smem, grid, threads);
        default: return run_phi<R, MAXT, MINB, 0, HERM>(p, a, smem, grid, threads);
    }
}

// Four CTAs of 256 threads an SM (at most 64 registers a thread; about 51 KB of
// shared memory each for rows of 2048): the row loads at the start of each CTA
// are latency-bound, and the fourth CTA hides more of them than the registers
// a thread gives up cost (2 us of 64 on the 2048 x 1024 rows).
template <int LOGM, bool HERM>
cudaError_t run_phi2(dfsnufft_plan p, const PhiArgs &a, size_t smem, dim3 grid, int threads) {
    constexpr int E = PhiCfg<float>::E;
    cudaError_t e = allow_smem(k_phi_pass2<E, 256, 4, LOGM, HERM>, smem);
    if (e) return e;
    return dfs_launch_dependent(k_phi_pass2<E, 256, 4, LOGM, HERM>, grid, dim3(threads), smem,
                                p->stream, a, (const float2 *)p->d_T, (const float2 *)p->d_tw1,
                                (const float2 *)p->d_stw_phi, (const int2 *)p->d_rowrange,
                                (float *)p->d_G);
}

template <typename R>
cudaError_t launch_phi(dfsnufft_plan p) {
    typedef typename CxT<R>::type C;
    constexpr int E = PhiCfg<R>::E, MAXT = PhiCfg<R>::MAXT;
    const dfsnufft_params &q = p->prm;
    PhiArgs a;
    a.N1 = q.N1;
    a.n1 = q.n1;
    a.logm = ilog2(q.n1) - 1;
    a.n2 = q.n2;
    a.F = p->n_fields;
    a.tcols = dfs_tcols(p->herm, q.N1);
    a.tpitch = dfs_tpitch(p->herm, q.N1);
    int lines;
    dfs_lines(p, a.line0, lines);
    const int M = q.n1 / 2;
    const int T = M / E;
    if (sizeof(R) == 4 && p->d_stw_phi && a.logm >= 9 && a.logm <= 11) {
        // two rows a thread group, 256 threads a CTA
        a.CB = 2 * (256 / T);
        const size_t smem = sizeof(C) * (size_t)a.CB * (region_len<C>(M) + a.tcols);
        const dim3 grid(q.n2 / a.CB, lines);
        const int threads = (a.CB / 2) * T;
        switch (a.logm) {
            case 9: return p->herm ? run_phi2<9, true>(p, a, smem, grid, threads)
                                   : run_phi2<9, false>(p, a, smem, grid, threads);
            case 10: return p->herm ? run_phi2<10, true>(p, a, smem, grid, threads)
                                    : run_phi2<10, false>(p, a, smem, grid, threads);
            default: return p->herm ? run_phi2<11, true>(p, a, smem, grid, threads)
                                    : run_phi2<11, false>(p, a, smem, grid, threads);
        }
    }
    int cb = MAXT / T;
    if (cb < 1) cb = 1;
    if (cb > DFS_ROW_BLOCK) cb = DFS_ROW_BLOCK;
    const size_t per_row = sizeof(C) * (size_t)(region_len<C>(M) + a.tcols);
    while (cb > 1 && per_row * cb > 160 * 1024) cb >>= 1;
    a.CB = cb;
    const size_t smem = per_row * cb;
    const dim3 grid(q.n2 / cb, lines);
    if (p->herm) return dispatch_phi<R, true>(p, a, smem, grid, cb * T);
    return dispatch_phi<R, false>(p, a, smem, grid, cb * T);
}

}  // namespace

cudaError_t dfs_launch_phi_pass(dfsnufft_plan p) {
    if (p->gdf) return launch_phi<df32>(p);           // FP64 plans in double-single
    return p->prm.dtype == DFSNUFFT_F64 ? launch_phi<double>(p) : launch_phi<float>(p);
}

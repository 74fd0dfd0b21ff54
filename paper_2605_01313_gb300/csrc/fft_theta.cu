// theta pass: deconvolve-and-pad fused with the column FFTs of the oversampled
// 2-D inverse FFT (sign +1, unnormalised), a middle stage of the type-2 NUFFT
// evaluating Eq. 5.3 (Sec. 5).  For each phi-mode column (m), the theta modes
// of that column, each divided by phihat2(n) phihat1(m), are placed at fine
// index n mod n2 (zeros elsewhere) and transformed along the column; only the
// fine rows inside the plan's needed row range are stored: T[f][row][column].
//
// General plans transform every column m = -N1/2 .. N1/2-1 (column q of the
// array, m = q - N1/2).  Plans for real fields (DFSNUFFT_REAL_FIELDS) transform
// only m = 0 .. N1/2 (column k of T is m = k): the values are Re v, which only
// depend on the Hermitian part h_{n,m} = (c_{n,m} + conj c_{-n,-m}) / 2 of the
// coefficients, and the phi pass rebuilds the columns m < 0 from
// H_{-m} = conj H_m.  For a real field h = c at every pair of entries that are
// both in the array; the entries whose mirror lies outside it (the Nyquist
// row n = -N2/2 and column m = -N1/2) are split exactly into their two halves
// c/2 at (n, m) and conj(c)/2 at (-n, -m), so they are evaluated literally as in
// a general plan.  Column m = 0 takes its Hermitian part in full (its mirror is
// the same column).  This halves the column transforms and the T buffer.
//
// Main kernel (k_theta_tma): persistent CTAs take blocks of CB columns (16- or
// 32-byte row segments).  The block's N2 coefficient rows arrive in shared memory by
// 2-D TMA boxes, double-buffered so that the next block streams in while this
// one is transformed.  Each column's length-n2 transform is done as two
// length-n2/2 transforms: output row 2q + s = sum_n c_n e^{2 pi i n s / n2}
// e^{2 pi i n q / (n2/2)}, s = 0, 1 (the modes fit in n2/2; when n2 = 2 N2 the
// two Nyquist modes n = -N2/2 and n = +N2/2 of a real-field plan share index
// N2/2 and are added there).  k_theta_pass is the plain-load version for shapes
// the TMA kernel does not take (unaligned coefficient pointer, CTA or
// shared-memory limits).
#include <type_traits>

#include "coef_map.cuh"
#include "fft_core.cuh"
#include "tma.cuh"

using namespace dfs_fft;
using namespace dfs_coef;

namespace {

// A coefficient as the pass's complex type: itself, or (double-single passes of
// FP64 plans) the FP64 value times 2^-sh (the line's exponent shift, df32.cuh)
// split into double-single parts.
template <typename C, typename CIn> __device__ __forceinline__ C in_value(CIn v, int) { return v; }
template <> __device__ __forceinline__ dfc in_value<dfc, double2>(double2 v, int sh) {
    return to_dfc_scaled(v, sh);
}
// Complex coefficient c_{n,m} (m >= 0, |n| <= N) of a field given by its
// partial-regularity DFS coefficients (Sec. 4): col[k] = f^c_{k,m} + i f^s_{k,m},
// k = 0..N, for this m.  First the standard coefficient S = f~^c + i f~^s at |n|
// (the product-to-sum stencil of Sec. 4 for the case of m; f~_{0,m} = f_{1,m}/2
// for even m >= 2, which the identity gives in place of the printed 0), then
// Eq. 5.4: c = S/2 (m = 0, n != 0; S for n = 0), conj(S)/2 or /4 (even m), and
// -sign(n) i conj(S)/4 (odd m).  The stencils are linear with real weights, so
// they act on the cosine and sine parts at once.
template <typename C, typename CIn>
__device__ __forceinline__ C pr_coef(int n, int m, int N, const CIn *__restrict__ col,
                                     int sh = 0) {
    typedef decltype(C().x) R;
    const int na = n < 0 ? -n : n;
    // f_{k,m} on the case's index range, zero elsewhere
    auto f = [&](int k, int lo, int hi) -> C {
        return (k >= lo && k <= hi) ? in_value<C>(col[k], sh) : cmake((R)0, (R)0);
    };
    C S;
    if (m == 0) {
        if (na > N) return cmake((R)0, (R)0);
        const R v = in_value<C>(col[na], sh).x;            // no sine part at m = 0
        return cmake(na == 0 ? v : (R)0.5 * v, (R)0);
    } else if (m == 1) {
        if (na == 0) return cmake((R)0, (R)0);
        // sin t cos k t = (sin (k+1) t - sin (k-1) t) / 2, k = 0..N-1
        S = cscale(f(na - 1, 0, N - 1) - f(na + 1, 0, N - 1), (R)0.5);
        if (na == 1) S = S + cscale(f(0, 0, N - 1), (R)0.5);
    } else if ((m & 1) == 0) {
        // sin t sin k t = (cos (k-1) t - cos (k+1) t) / 2, k = 1..N-1
        S = na == 0 ? cscale(f(1, 1, N - 1), (R)0.5)
                    : cscale(f(na + 1, 1, N - 1) - f(na - 1, 1, N - 1), (R)0.5);
    } else {
        if (na == 0) return cmake((R)0, (R)0);
        // sin^2 t sin k t = (2 sin k t - sin (k-2) t - sin (k+2) t) / 4, k = 1..N-2
        S = cscale(cscale(f(na, 1, N - 2), (R)2) - f(na - 2, 1, N - 2) - f(na + 2, 1, N - 2),
                   (R)0.25);
        if (na == 1) S = S + cscale(f(1, 1, N - 2), (R)0.25);
    }
    const C cs = cmake(S.x, -S.y);                         // conj(S) = f~^c - i f~^s
    if ((m & 1) == 0) return cscale(cs, na == 0 ? (R)0.5 : (R)0.25);
    // -sign(n) i conj(S) / 4
    const R g = n > 0 ? (R)-0.25 : (R)0.25;
    return cmake(-g * cs.y, g * cs.x);
}

// Largest biased FP64 exponent of each line's coefficients (emax[line], zeroed
// before the launch; the double-single passes scale the line by it, df32.cuh),
// over the entries the theta pass reads: the whole N2 x N1 array (general
// plans), the Nyquist column 0 and the columns m >= 0 (array columns
// N1/2 .. N1-1) of every row plus the rest of the Nyquist row 0 (real-field
// plans), or all line_elems entries (partial-regularity input).  grid
// (blocks, lines).
__global__ void __launch_bounds__(256) k_coef_maxexp(const double2 *__restrict__ coef,
                                                     int line_elems, int rows, int N1, int herm,
                                                     int *__restrict__ emax) {
    const double2 *c = coef + (size_t)blockIdx.y * line_elems;
    const int K = N1 / 2 + 1;
    const int n = herm ? rows * K + (N1 / 2 - 1) : line_elems;
    unsigned m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int off = i;
        if (herm) {
            if (i < rows * K) {
                const int r = i / K;
                const int j = i - r * K;
                off = r * N1 + (j == 0 ? 0 : N1 / 2 - 1 + j);
            } else {
                off = i - rows * K + 1;                  // row 0, columns 1 .. N1/2 - 1
            }
        }
        const double2 v = c[off];
        const unsigned ex = (unsigned)(__double_as_longlong(v.x) >> 52) & 0x7ffu;
        const unsigned ey = (unsigned)(__double_as_longlong(v.y) >> 52) & 0x7ffu;
        m = max(m, max(ex, ey));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&emax[blockIdx.y], (int)m);
}

struct ThetaArgs {
    int N1, N2, n2, logn2;
    int CB;                   // columns per CTA
    int F;                    // fields per member (line f belongs to member f / F)
    int tcols, tpitch;        // transformed columns, row pitch of T
    int prM, prN;             // partial-regularity input: truncation (prM < 0: complex input)
    int line0;                // first line (blockIdx.y = line - line0)
};

// grid (ceil(tcols / CB), lines); block CB * n2/E threads, thread = (t, c) with c fastest.
// PRIN (real-field plans): the input is partial-regularity DFS coefficients,
// lines x (prM + 1) x (prN + 1) complex, converted on the fly by pr_coef.
// LOGN > 0: length n2 = 2^LOGN at compile time with the stage-ordered table stw.
// emax (double-single passes): each line's largest coefficient exponent, from
// k_coef_maxexp; the line is transformed at the scale of df_line_shift.
template <typename R, int E, int MAXT, int MINB, bool HERM, bool PRIN = false,
          typename CIn = typename CxT<R>::type, int LOGN = 0>
__global__ void __launch_bounds__(MAXT, MINB)
    k_theta_pass(ThetaArgs a, const CIn *__restrict__ coef,
                 const R *__restrict__ inv1, const R *__restrict__ inv2,
                 const typename CxT<R>::type *__restrict__ tw,
                 const typename CxT<R>::type *__restrict__ stw,
                 const int2 *__restrict__ rowrange, typename CxT<R>::type *__restrict__ out,
                 const int *__restrict__ emax) {
    dfs_grid_wait();
    typedef typename CxT<R>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *smem = reinterpret_cast<C *>(smem_raw);
    const int c = threadIdx.x % a.CB;
    const int t = threadIdx.x / a.CB;
    const int q = blockIdx.x * a.CB + c;           // column of T
    const int f = a.line0 + blockIdx.y;
    const int2 rr = rowrange[f / a.F];
    const bool col_ok = q < a.tcols;
    const CIn *cf0 = coef + (size_t)f * a.N2 * a.N1;
    C *dst = out + (size_t)f * a.n2 * a.tpitch + q;
    const int half = a.N2 / 2;
    const int qa = HERM ? a.N1 / 2 + q : q;        // array column
    const R sq = col_ok ? inv1[qa < a.N1 ? qa : 0] : (R)0;
    C *sm = smem + (size_t)c * region_stride<C>(a.n2, a.CB);
    const int sh = emax ? df_line_shift(emax[f]) : 0;
    auto cf = [&](int r, int col) -> C {
        return (r < a.N2 && col < a.N1) ? in_value<C>(cf0[(size_t)r * a.N1 + col], sh)
                                        : cmake((R)0, (R)0);
    };
    auto ld = [&](int i) -> C {
        if (!col_ok) return cmake((R)0, (R)0);
        int n;
        if (i < half) n = i;
        else if (i >= a.n2 - half) n = i - a.n2;
        else if (HERM && i == half) n = half;
        else return cmake((R)0, (R)0);
        const int r = n + half;
        const R s = sq * inv2[r < a.N2 ? r : 0];
        if constexpr (PRIN) {
            if (q > a.prM || n > a.prN || n < -a.prN) return cmake((R)0, (R)0);
            const CIn *col = coef + ((size_t)f * (a.prM + 1) + q) * (a.prN + 1);
            return cscale(pr_coef<C>(n, q, a.prN, col, sh), s);
        } else if constexpr (HERM) {
            return cscale(herm_coef<C>(n, q, half, a.N1, cf), s);
        } else {
            return cscale(cf(r, qa), s);
        }
    };
    auto st = [&](int i, C v) {
        if (col_ok && ((i - rr.x) & (a.n2 - 1)) < rr.y) dst[(size_t)i * a.tpitch] = v;
    };
    if constexpr (LOGN > 0) line_fft_ct<LOGN, E>(stw, sm, t, ld, st);
    else line_fft<E>(a.logn2, tw, 0, sm, t, ld, st);
}

struct ThetaTmaArgs {
    int N1, N2, n2, logh;     // logh = log2(n2 / 2)
    int nbq;                  // column blocks per line, ceil(tcols / CB)
    int total;                // nbq * lines (members x fields)
    int F;                    // fields per member (line f belongs to member f / F)
    int nbox, box_rows;       // TMA boxes per block and rows per box
    int in_elems;             // complex elements delivered per block
    int nbuf;                 // input buffers (2: prefetch the next block)
    unsigned tx_bytes;        // bytes delivered per block
    int tcols, tpitch;        // transformed columns, row pitch of T
    int col_base;             // array column of transformed column 0
    int prM, prN;             // partial-regularity input: truncation (prM < 0: complex input)
    int line0;                // first line of the launch (blocks cover lines line0 ..)
};

// LOGH > 0: half length 2^LOGH fixed at compile time (unrolled transform);
// LOGH == 0: taken from the arguments.  DUAL (FP32 at compile-time lengths):
// the two half-length transforms of a column run together in the same threads
// (line_fft_ct2: twiddles, index arithmetic and barriers shared), which needs
// one input buffer only: the next block's boxes are issued as soon as every
// thread has read its inputs (after the transforms' first barrier), so they
// land while this block is transformed.  Otherwise the halves run one after
// the other and the next block streams into a second buffer when one fits.
// PRIN (real-field plans): the input is partial-regularity DFS coefficients,
// lines x (prM + 1) x (prN + 1) complex, whose column m is contiguous; a block's
// CB columns are staged by 8-byte asynchronous copies of every thread instead of
// TMA boxes (the columns are not 16-byte aligned), completing on the same
// mbarrier, and converted on the fly by pr_coef.
template <typename R, int E, int CB, int MAXT, int MINB, int LOGH, bool HERM, bool PRIN = false>
__global__ void __launch_bounds__(MAXT, MINB)
    k_theta_tma(ThetaTmaArgs a, const __grid_constant__ CUtensorMap tmap,
                const typename CxT<R>::type *__restrict__ coef,
                const R *__restrict__ inv1, const R *__restrict__ inv2,
                const typename CxT<R>::type *__restrict__ tw,
                const typename CxT<R>::type *__restrict__ stw, const int2 *__restrict__ rowrange,
                typename CxT<R>::type *__restrict__ out, int *__restrict__ status) {
    dfs_grid_wait();
    typedef typename CxT<R>::type C;
    constexpr bool DUAL = LOGH > 0 && sizeof(R) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // TMA destinations start on 128-byte boundaries (base rounded up here;
    // buffer and box sizes are multiples of 128 bytes by construction)
    unsigned char *base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base);
    C *inb = reinterpret_cast<C *>(base + 128);
    C *ex = inb + (size_t)a.nbuf * a.in_elems;
    const int H = LOGH ? (1 << LOGH) : (a.n2 >> 1);
    constexpr int NREG = DUAL ? 2 : 1;             // exchange regions per column
    R *f2 = reinterpret_cast<R *>(ex + (size_t)NREG * CB * region_len<C>(H));   // 1 / phihat2
    C *nyq = reinterpret_cast<C *>(f2 + ((a.N2 + 3) & ~3));   // real-field plans: CB values
    const int c = threadIdx.x % CB;
    const int t = threadIdx.x / CB;
    const int half = a.N2 / 2;
    // column c's regions c and (DUAL: its odd-row transform) CB + c, region_stride
    // apart (the columns of a warp on different bank pairs)
    C *sm = ex + (size_t)c * region_stride<C>(H, CB);
    C *sm1 = ex + (size_t)(CB + c) * region_stride<C>(H, CB);
    for (int i = threadIdx.x; i < a.N2; i += blockDim.x) f2[i] = inv2[i];
    if (threadIdx.x == 0) {
        // PRIN: every thread arrives once a phase, when its copies have landed
        mbar_init(&bar[0], PRIN ? blockDim.x : 1);
        mbar_init(&bar[1], PRIN ? blockDim.x : 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int prs = a.prN + 1;                     // PRIN: staged elements a column
    // issued by thread 0 (TMA boxes), or by every thread (PRIN)
    auto issue = [&](int blk, int b) {
        const int f = a.line0 + blk / a.nbq;
        const int qb = blk - (f - a.line0) * a.nbq;
        C *dst = inb + (size_t)b * a.in_elems;
        if constexpr (PRIN) {
            for (int cc = 0; cc < CB; ++cc) {
                const int q = qb * CB + cc;
                if (q > a.prM) break;
                const C *src = coef + ((size_t)f * (a.prM + 1) + q) * prs;
                for (int k = threadIdx.x; k < prs; k += blockDim.x)
                    cp_async_8(dst + (size_t)cc * prs + k, src + k);
            }
            cp_async_mbar_arrive_noinc(&bar[b]);
            return;
        }
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[b], a.tx_bytes);
        const int x = (a.col_base + qb * CB) * (int)(sizeof(C) / 8);
        for (int i = 0; i < a.nbox; ++i)
            tma_load_2d(dst + (size_t)i * a.box_rows * CB, &tmap, x, f * a.N2 + i * a.box_rows,
                        &bar[b]);
    };
    uint32_t phase0 = 0, phase1 = 0;
    int it = 0;
    const bool issuer = PRIN || threadIdx.x == 0;
    if (issuer && (int)blockIdx.x < a.total) issue(blockIdx.x, 0);
    for (int blk = blockIdx.x; blk < a.total; blk += gridDim.x, ++it) {
        const int cur = a.nbuf == 2 ? (it & 1) : 0;
        const int nxt = blk + gridDim.x;
        const bool pre = a.nbuf == 2 && nxt < a.total;
        if (pre && issuer) issue(nxt, cur ^ 1);
        if (HERM && !PRIN && threadIdx.x < CB) {
            // conj c_{-N2/2,-m} of each column (the mirror of the Nyquist row),
            // fetched while the block's boxes land
            const int f = a.line0 + blk / a.nbq;
            const int q = (blk - (f - a.line0) * a.nbq) * CB + threadIdx.x;
            const int qa = a.col_base + q;
            C v = cmake((R)0, (R)0);
            if (q < a.tcols) v = coef[(size_t)f * a.N2 * a.N1 + (a.N1 - qa)];
            nyq[threadIdx.x] = cconj(v);
        }
        const bool ok = mbar_wait_bounded(&bar[cur], cur ? phase1 : phase0);
        if (cur) phase1 ^= 1;
        else phase0 ^= 1;
        if (__syncthreads_or(!ok)) {
            // give up on this launch; let copies still in flight land first
            if constexpr (PRIN) {
                cp_async_wait_all();
                if (threadIdx.x == 0) atomicExch(status, DFS_STATUS_TIMEOUT);
            } else if (threadIdx.x == 0) {
                atomicExch(status, DFS_STATUS_TIMEOUT);
                mbar_wait_bounded(&bar[cur], cur ? phase1 ^ 1 : phase0 ^ 1);
                if (pre) mbar_wait_bounded(&bar[cur ^ 1], cur ? phase0 : phase1);
            }
            __syncthreads();
            return;
        }
        const int f = a.line0 + blk / a.nbq;
        const int2 rr = rowrange[f / a.F];
        const int q = (blk - (f - a.line0) * a.nbq) * CB + c;      // column of T
        const int qa = a.col_base + q;                 // array column
        const bool col_ok = q < a.tcols;
        const R sq = col_ok ? inv1[qa < a.N1 ? qa : 0] : (R)0;
        const C *in = inb + (size_t)cur * a.in_elems;
        const C *cf0 = coef + (size_t)f * a.N2 * a.N1;
        C *dst = out + (size_t)f * a.n2 * a.tpitch + q;
        const bool k_zero = HERM && q == 0;            // m = 0: its own mirror
        const bool k_nyq = HERM && qa == a.N1;         // m = N1/2: mirror of the Nyquist column
        const C nyq_row = HERM ? nyq[c] : cmake((R)0, (R)0);
        // h_{n,m} (real-field plans, see herm_coef) or c_{n,m}, deconvolved
        auto coef_nm = [&](int n) -> C {
            const int r = n + half;
            if constexpr (PRIN) {
                if (q > a.prM || n > a.prN || n < -a.prN) return cmake((R)0, (R)0);
                return cscale(pr_coef<C>(n, q, a.prN, in + (size_t)c * prs), sq * f2[r]);
            }
            C v;
            if constexpr (HERM) {
                if (k_nyq) {                           // one column per line: global loads
                    v = n == -half ? cmake((R)0, (R)0)
                                   : cscale(cconj(cf0[(size_t)(half - n) * a.N1]), (R)0.5);
                } else if (n == half) {
                    v = cscale(nyq_row, (R)0.5);
                } else {
                    v = in[r * CB + c];
                    if (n == -half) {
                        v = cscale(v, (R)0.5);
                    } else if (k_zero) {
                        const C mirror = in[(a.N2 - r) * CB + c];
                        v = cscale(cmake(v.x + mirror.x, v.y - mirror.y), (R)0.5);
                    }
                }
            } else {
                v = in[r * CB + c];
            }
            return cscale(v, sq * f2[r < a.N2 ? r : 0]);
        };
        auto row_needed = [&](int row) { return ((row - rr.x) & (a.n2 - 1)) < rr.y; };
        if constexpr (DUAL) {
            // input i = t + e H/E of both halves: y_n and y_n e^{2 pi i n / n2}.
            // With n2 = 2H the twiddle is e^{2 pi i t / n2} e^{i pi e / E}, negated
            // for n = i - H: one table read a thread, the rest rotations by
            // multiples of pi/8 that are constants once the loop over e unrolls.
            constexpr int TT = (1 << LOGH) / E;
            const C wt = ldt(&tw[t]);
            auto ld2 = [&](int i, C &y0, C &y1) {
                y0 = y1 = cmake((R)0, (R)0);
                if (!col_ok) return;
                const int e = (i - t) / TT;
                const C wi = cmul(wt, cmake((R)c16(e * (8 / E)), (R)s16(e * (8 / E))));
                if (i < half) {
                    const C y = coef_nm(i);
                    y0 = y0 + y;
                    y1 = y1 + cmul(y, wi);
                } else if (i >= H - half) {
                    const C y = coef_nm(i - H);
                    y0 = y0 + y;
                    y1 = y1 - cmul(y, wi);
                }
                if (HERM && i == half) {
                    const C y = coef_nm(half);
                    y0 = y0 + y;
                    y1 = y1 + cmul(y, ldt(&tw[half]));
                }
            };
            auto st2 = [&](int qq, C z0, C z1) {
                if (!col_ok) return;
                if (row_needed(2 * qq)) dst[(size_t)(2 * qq) * a.tpitch] = z0;
                if (row_needed(2 * qq + 1)) dst[(size_t)(2 * qq + 1) * a.tpitch] = z1;
            };
            auto refill = [&]() {
                if (issuer && a.nbuf == 1 && nxt < a.total) issue(nxt, 0);
            };
            line_fft_ct2<LOGH, E>(stw, sm, sm1, t, ld2, st2, refill);
            __syncthreads();
        } else {
#pragma unroll 1
            for (int s = 0; s < 2; ++s) {
                auto term = [&](int n) -> C {
                    C y = coef_nm(n);
                    if (s) y = cmul(y, ldt(&tw[n & (a.n2 - 1)]));
                    return y;
                };
                auto ld = [&](int i) -> C {
                    C y = cmake((R)0, (R)0);
                    if (!col_ok) return y;
                    if (i < half) y = term(i);
                    else if (i >= H - half) y = term(i - H);
                    if (HERM && i == half) y = y + term(half);
                    return y;
                };
                auto st = [&](int qq, C v) {
                    const int row = 2 * qq + s;
                    if (col_ok && row_needed(row)) dst[(size_t)row * a.tpitch] = v;
                };
                if constexpr (LOGH > 0) line_fft_ct<LOGH, E>(stw, sm, t, ld, st);
                else line_fft<E>(a.logh, tw, 1, sm, t, ld, st);
                __syncthreads();
            }
            if (a.nbuf == 1 && issuer && nxt < a.total) issue(nxt, 0);
        }
    }
}

// Per precision: elements per thread E, threads per CTA at most MAXT, resident
// CTAs MINB the register budget is set for (plain kernel); for the TMA kernel
// columns per block CB, threads at most TMAXT and TMINB resident CTAs per SM
// (two CTAs of two columns each keep an SM busy while either waits at a
// barrier of its transform).
template <typename R> struct ThetaCfg;
template <> struct ThetaCfg<float> {
    static const int E = DFS_FFT_E, MAXT = 1024, MINB = 1, CB = 2, TMAXT = 512, TMINB = 2;
};
template <> struct ThetaCfg<double> {
    static const int E = DFS_FFT_E, MAXT = 512, MINB = 1, CB = 2, TMAXT = 512, TMINB = 1;
};
// Double-single: two CTAs of one column each per SM (64 registers a thread, a
// few bytes spilled; 70 KB of shared memory each), which hides the latency of
// the strided coefficient loads better than one CTA at 101 registers (C3 FP64
// theta pass 413 -> 342 us).
template <> struct ThetaCfg<df32> {
    static const int E = DFS_FFT_E, MAXT = 512, MINB = 2, CB = 1, TMAXT = 512, TMINB = 1;
};

template <typename R, int CB, int LOGH, bool HERM, bool PRIN>
cudaError_t run_theta_tma(dfsnufft_plan p, const ThetaTmaArgs &a, const CUtensorMap &tmap,
                          const void *coeffs, size_t smem, int grid, int threads) {
    typedef typename CxT<R>::type C;
    constexpr int E = ThetaCfg<R>::E, MAXT = ThetaCfg<R>::TMAXT, MINB = ThetaCfg<R>::TMINB;
    cudaError_t e = allow_smem(k_theta_tma<R, E, CB, MAXT, MINB, LOGH, HERM, PRIN>, smem);
    if (e) return e;
    return dfs_launch_dependent(
        k_theta_tma<R, E, CB, MAXT, MINB, LOGH, HERM, PRIN>, dim3(grid), dim3(threads), smem,
        p->stream, a, tmap, (const C *)coeffs, (const R *)p->d_inv1, (const R *)p->d_inv2,
        (const C *)p->d_tw2, (const C *)p->d_stw_theta, (const int2 *)p->d_rowrange, (C *)p->d_T,
        p->d_status);
}

template <typename R, int CB, bool HERM, bool PRIN = false>
cudaError_t dispatch_theta_tma(dfsnufft_plan p, const ThetaTmaArgs &a, const CUtensorMap &tmap,
                               const void *coeffs, size_t smem, int grid, int threads) {
    if (!p->d_stw_theta)
        return run_theta_tma<R, CB, 0, HERM, PRIN>(p, a, tmap, coeffs, smem, grid, threads);
    switch (a.logh) {
        case 9: return run_theta_tma<R, CB, 9, HERM, PRIN>(p, a, tmap, coeffs, smem, grid, threads);
        case 10:
            return run_theta_tma<R, CB, 10, HERM, PRIN>(p, a, tmap, coeffs, smem, grid, threads);
        case 11:
            return run_theta_tma<R, CB, 11, HERM, PRIN>(p, a, tmap, coeffs, smem, grid, threads);
        default: return run_theta_tma<R, CB, 0, HERM, PRIN>(p, a, tmap, coeffs, smem, grid, threads);
    }
}

// Launch the TMA theta pass with CB columns per block; returns
// cudaErrorNotSupported (without launching) when the shape or the coefficient
// pointer does not suit it.  prM >= 0: partial-regularity input (real-field
// plans), staged by asynchronous 8-byte copies (no tensor map).
template <typename R, int CB>
cudaError_t launch_theta_tma_cb(dfsnufft_plan p, const void *coeffs, int prM, int prN) {
    typedef typename CxT<R>::type C;
    constexpr int E = ThetaCfg<R>::E, MAXT = ThetaCfg<R>::TMAXT, MINB = ThetaCfg<R>::TMINB;
    static_assert(CB * sizeof(C) >= 16, "a TMA box row spans at least 16 bytes");
    const dfsnufft_params &q = p->prm;
    const bool pr = prM >= 0;
    if (pr && (!p->herm || ((uintptr_t)coeffs & (sizeof(C) - 1)) != 0))
        return cudaErrorNotSupported;
    if ((!pr && ((uintptr_t)coeffs & 15) != 0) || !p->d_status) return cudaErrorNotSupported;
    const int H = q.n2 / 2;
    if (H < E || CB * (H / E) > MAXT) return cudaErrorNotSupported;
    ThetaTmaArgs a;
    a.N1 = q.N1;
    a.N2 = q.N2;
    a.n2 = q.n2;
    a.logh = ilog2(H);
    a.tcols = dfs_tcols(p->herm, q.N1);
    a.tpitch = dfs_tpitch(p->herm, q.N1);
    a.col_base = p->herm ? q.N1 / 2 : 0;
    a.prM = prM;
    a.prN = prN;
    // the box's first column must sit on a 16-byte boundary
    if ((a.col_base * sizeof(C)) % 16 != 0) return cudaErrorNotSupported;
    a.nbq = (a.tcols + CB - 1) / CB;
    int line0, lines;
    dfs_lines(p, line0, lines);
    a.line0 = line0;
    a.total = a.nbq * lines;
    a.F = p->n_fields;
    // boxes of CB columns x box_rows rows, each a multiple of 128 bytes (box
    // destinations stay 128-byte aligned): box_rows a multiple of ra rows
    constexpr int ra = 128 / (CB * (int)sizeof(C));
    a.box_rows = q.N2 < 256 ? ((q.N2 + ra - 1) / ra * ra) : 256;
    a.nbox = (q.N2 + a.box_rows - 1) / a.box_rows;
    a.in_elems = a.nbox * a.box_rows * CB;
    a.tx_bytes = (unsigned)(sizeof(C) * a.in_elems);
    if (pr && (long long)CB * (prN + 1) > a.in_elems) return cudaErrorNotSupported;
    // compile-time lengths in FP32 run both halves at once (see k_theta_tma)
    const bool dual = sizeof(R) == 4 && p->d_stw_theta && a.logh >= 9 && a.logh <= 11;
    const size_t ex_bytes = sizeof(C) * (size_t)(dual ? 2 : 1) * CB * region_len<C>(H);
    const size_t f2_bytes = sizeof(R) * (size_t)((q.N2 + 3) & ~3) + sizeof(C) * CB;
    const size_t limit = (MINB > 1 ? 226 / MINB : 220) * 1024;
    const size_t in_bytes = sizeof(C) * (size_t)a.in_elems;
    a.nbuf = !dual && 256 + 2 * in_bytes + ex_bytes + f2_bytes <= limit ? 2 : 1;
    const size_t smem = 256 + a.nbuf * in_bytes + ex_bytes + f2_bytes;
    if (smem > limit) return cudaErrorNotSupported;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));             // unused by the partial-regularity form
    if (!pr) {
        cudaError_t e = dfs_encode_tensor_map_2d(&tmap, coeffs, (uint64_t)q.N1 * (sizeof(C) / 8),
                                                 (uint64_t)q.N2 * (line0 + lines),
                                                 sizeof(C) * (uint64_t)q.N1,
                                                 (uint32_t)(CB * (sizeof(C) / 8)),
                                                 (uint32_t)a.box_rows);
        if (e) return e;
    }
    int grid = (p->num_sms > 0 ? p->num_sms : 1) * MINB;
    if (grid > a.total) grid = a.total;
    const int threads = CB * (H / E);
    if (pr) return dispatch_theta_tma<R, CB, true, true>(p, a, tmap, coeffs, smem, grid, threads);
    if (p->herm) return dispatch_theta_tma<R, CB, true>(p, a, tmap, coeffs, smem, grid, threads);
    return dispatch_theta_tma<R, CB, false>(p, a, tmap, coeffs, smem, grid, threads);
}

// The configured block width, else (FP64 columns of 8192 fine rows) one column.
template <typename R>
cudaError_t launch_theta_tma(dfsnufft_plan p, const void *coeffs, int prM, int prN) {
    cudaError_t e = launch_theta_tma_cb<R, ThetaCfg<R>::CB>(p, coeffs, prM, prN);
    if constexpr (sizeof(R) == 8) {
        if (e == cudaErrorNotSupported) e = launch_theta_tma_cb<R, 1>(p, coeffs, prM, prN);
    }
    return e;
}

template <typename R, int E, int MAXT, int MINB, bool HERM, bool PRIN, int LOGN>
cudaError_t run_theta_df(dfsnufft_plan p, const ThetaArgs &a, const void *coeffs, size_t smem,
                         dim3 grid, int threads) {
    typedef typename CxT<R>::type C;
    cudaError_t e = allow_smem(k_theta_pass<R, E, MAXT, MINB, HERM, PRIN, double2, LOGN>, smem);
    if (e) return e;
    return dfs_launch_dependent(
        k_theta_pass<R, E, MAXT, MINB, HERM, PRIN, double2, LOGN>, grid, dim3(threads), smem,
        p->stream, a, (const double2 *)coeffs, (const R *)p->d_df_inv1,
        (const R *)p->d_df_inv2, (const C *)p->d_df_tw2, (const C *)p->d_df_stw_theta,
        (const int2 *)p->d_rowrange, (C *)p->d_T, (const int *)p->d_emax);
}

template <typename R, int E, bool HERM, bool PRIN = false>
cudaError_t run_theta_plain(dfsnufft_plan p, const ThetaArgs &a, const void *coeffs, size_t smem,
                            dim3 grid, int threads) {
    typedef typename CxT<R>::type C;
    constexpr int MAXT = ThetaCfg<R>::MAXT, MINB = ThetaCfg<R>::MINB;
    if constexpr (std::is_same<R, df32>::value) {
        // FP64 coefficients, double-single factors and twiddles; lengths 2^10 ..
        // 2^12 at compile time with the double-single stage-ordered table
        if constexpr (E == DFS_FFT_E) {
            switch (p->d_df_stw_theta ? a.logn2 : 0) {
                case 10:
                    return run_theta_df<R, E, MAXT, MINB, HERM, PRIN, 10>(p, a, coeffs, smem,
                                                                          grid, threads);
                case 11:
                    return run_theta_df<R, E, MAXT, MINB, HERM, PRIN, 11>(p, a, coeffs, smem,
                                                                          grid, threads);
                case 12:
                    return run_theta_df<R, E, MAXT, MINB, HERM, PRIN, 12>(p, a, coeffs, smem,
                                                                          grid, threads);
                default: break;
            }
        }
        return run_theta_df<R, E, MAXT, MINB, HERM, PRIN, 0>(p, a, coeffs, smem, grid, threads);
    } else {
        cudaError_t e = allow_smem(k_theta_pass<R, E, MAXT, MINB, HERM, PRIN>, smem);
        if (e) return e;
        return dfs_launch_dependent(
            k_theta_pass<R, E, MAXT, MINB, HERM, PRIN>, grid, dim3(threads), smem, p->stream, a,
            (const C *)coeffs, (const R *)p->d_inv1, (const R *)p->d_inv2, (const C *)p->d_tw2,
            (const C *)nullptr, (const int2 *)p->d_rowrange, (C *)p->d_T, (const int *)nullptr);
    }
}

template <typename R>
cudaError_t launch_theta(dfsnufft_plan p, const void *coeffs, int prM, int prN) {
    typedef typename CxT<R>::type C;
    if constexpr (!std::is_same<R, df32>::value) {
        cudaError_t e = launch_theta_tma<R>(p, coeffs, prM, prN);
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();
    }
    constexpr int MAXT = ThetaCfg<R>::MAXT;
    const dfsnufft_params &q = p->prm;
    // columns longer than E x MAXT values (FP64, 8192 fine rows): 16 a thread
    const bool wide = q.n2 / ThetaCfg<R>::E > MAXT;
    const int E = wide ? 16 : ThetaCfg<R>::E;
    ThetaArgs a;
    a.N1 = q.N1;
    a.N2 = q.N2;
    a.n2 = q.n2;
    a.logn2 = ilog2(q.n2);
    a.F = p->n_fields;
    a.tcols = dfs_tcols(p->herm, q.N1);
    a.tpitch = dfs_tpitch(p->herm, q.N1);
    a.prM = prM;
    a.prN = prN;
    int line0, lines;
    dfs_lines(p, line0, lines);
    a.line0 = line0;
    const int T = q.n2 / E;
    int cb = MAXT / T;
    if (cb < 1) cb = 1;
    int ncp = 1;
    while (ncp < a.tcols) ncp <<= 1;
    if (cb > ncp) cb = ncp;
    const size_t per_col = sizeof(C) * (size_t)region_len<C>(q.n2);
    while (cb > 1 && per_col * cb > 160 * 1024) cb >>= 1;
    a.CB = cb;
    const size_t smem = per_col * cb;
    const dim3 grid((a.tcols + cb - 1) / cb, lines);
    if (prM >= 0) {
        if (!p->herm) return cudaErrorInvalidValue;
        if (wide) return run_theta_plain<R, 16, true, true>(p, a, coeffs, smem, grid, cb * T);
        return run_theta_plain<R, ThetaCfg<R>::E, true, true>(p, a, coeffs, smem, grid, cb * T);
    }
    if (wide) {
        if (p->herm) return run_theta_plain<R, 16, true>(p, a, coeffs, smem, grid, cb * T);
        return run_theta_plain<R, 16, false>(p, a, coeffs, smem, grid, cb * T);
    }
    if (p->herm) return run_theta_plain<R, ThetaCfg<R>::E, true>(p, a, coeffs, smem, grid, cb * T);
    return run_theta_plain<R, ThetaCfg<R>::E, false>(p, a, coeffs, smem, grid, cb * T);
}

}  // namespace

cudaError_t dfs_launch_line_maxexp(dfsnufft_plan p, const void *data, int line_elems, int rows,
                                   int herm, int line0, int lines) {
    const dfsnufft_params &q = p->prm;
    cudaError_t e = cudaMemsetAsync(p->d_emax + line0, 0, sizeof(int) * lines, p->stream);
    if (e) return e;
    const int n = herm ? rows * (q.N1 / 2 + 1) + q.N1 / 2 - 1 : line_elems;
    int blocks = (n + 2047) / 2048;
    if (blocks > 1024) blocks = 1024;
    k_coef_maxexp<<<dim3(blocks, lines), 256, 0, p->stream>>>(
        (const double2 *)data + (size_t)line0 * line_elems, line_elems, rows, q.N1, herm,
        p->d_emax + line0);
    return cudaGetLastError();
}

// Each line's exponent maximum for the double-single passes (k_coef_maxexp).
static cudaError_t launch_coef_maxexp(dfsnufft_plan p, const void *coeffs, int prM, int prN) {
    const dfsnufft_params &q = p->prm;
    int line0, lines;
    dfs_lines(p, line0, lines);
    const bool pr = prM >= 0;
    const int line_elems = pr ? (prM + 1) * (prN + 1) : q.N2 * q.N1;
    return dfs_launch_line_maxexp(p, coeffs, line_elems, q.N2, (!pr && p->herm) ? 1 : 0, line0,
                                  lines);
}

cudaError_t dfs_launch_theta_pass(dfsnufft_plan p, const void *coeffs, int prM, int prN) {
    if (p->gdf) {                                  // FP64 in double-single
        cudaError_t e = launch_coef_maxexp(p, coeffs, prM, prN);
        if (e) return e;
        return launch_theta<df32>(p, coeffs, prM, prN);
    }
    return p->prm.dtype == DFSNUFFT_F64 ? launch_theta<double>(p, coeffs, prM, prN)
                                        : launch_theta<float>(p, coeffs, prM, prN);
}

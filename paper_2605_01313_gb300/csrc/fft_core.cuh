// FFT engine shared by the theta and phi passes: in-register radix-2/4/8/16
// decimation-in-frequency butterflies inside Stockham autosort stages, with
// padded shared-memory exchanges between stages.  Two drivers: line_fft
// (length known at run time) and line_fft_ct (length and radix sequence fixed
// at compile time, fully unrolled; used for the large transforms).
#pragma once

#include "common.cuh"
#include "df32.cuh"
#include "tma.cuh"

namespace dfs_fft {

// cos(2 pi k / 16) from the values of cos and sin at pi/8 and pi/4.
__host__ __device__ constexpr double c16(int k) {
    constexpr double C1 = 0.92387953251128675613;   // cos(pi/8)
    constexpr double S1 = 0.38268343236508977173;   // sin(pi/8)
    constexpr double H = 0.70710678118654752440;    // sqrt(2)/2
    k &= 15;
    return k == 0 ? 1.0 : k == 1 ? C1 : k == 2 ? H : k == 3 ? S1 : k == 4 ? 0.0
         : k == 5 ? -S1 : k == 6 ? -H : k == 7 ? -C1 : k == 8 ? -1.0 : k == 9 ? -C1
         : k == 10 ? -H : k == 11 ? -S1 : k == 12 ? 0.0 : k == 13 ? S1 : k == 14 ? H : C1;
}
__host__ __device__ constexpr double s16(int k) { return c16(k - 4); }

// a * e^{+2 pi i K / 16}, exact for the multiples of pi/2.
template <int K, typename C>
__device__ __forceinline__ C tw16(C a) {
    constexpr int k = K & 15;
    if constexpr (k == 0) {
        return a;
    } else if constexpr (k == 4) {
        return cmake(-a.y, a.x);
    } else if constexpr (k == 8) {
        return cmake(-a.x, -a.y);
    } else if constexpr (k == 12) {
        return cmake(a.y, -a.x);
    } else {
        typedef decltype(a.x) R;
        constexpr R c = (R)c16(k), s = (R)s16(k);
        return cmake(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

// In-place DFT of size R (power of two <= 16), sign +1, on the registers
// v[K + r S] (r = 0..R-1): radix-2 decimation in frequency, so that afterwards
// v[K + r S] holds output bitrev_R(r).  Every index is a compile-time constant.
template <int R, int K, int S, int H, int B, int P, typename C>
__device__ __forceinline__ void dif_step(C *v) {
    // block B of size 2H, pair P: (a, c) -> (a + c, (a - c) e^{+2 pi i P / (2H)})
    if constexpr (B < R / (2 * H)) {
        if constexpr (P < H) {
            constexpr int i = K + (B * 2 * H + P) * S;
            constexpr int j = i + H * S;
            const C a = v[i], c = v[j];
            v[i] = a + c;
            v[j] = tw16<P * (8 / H)>(a - c);
            dif_step<R, K, S, H, B, P + 1>(v);
        } else {
            dif_step<R, K, S, H, B + 1, 0>(v);
        }
    }
}

template <int R, int K, int S, int H, typename C>
__device__ __forceinline__ void dif_levels(C *v) {
    if constexpr (H >= 1) {
        dif_step<R, K, S, H, 0, 0>(v);
        dif_levels<R, K, S, H / 2>(v);
    }
}

__host__ __device__ constexpr int bitrev(int r, int R) {
    int out = 0;
    for (int b = 1; b < R; b <<= 1) {
        out = (out << 1) | (r & 1);
        r >>= 1;
    }
    return out;
}

// Shared-memory exchange layout.  FP32 lines (8-byte elements, a bank pair
// each, 16 pairs a row of banks): element i sits at i ^ ((i >> 3) & 15), a
// permutation of [0, n) for every power of two n that XORs the bank pair with
// the 8-element group, so that neither the unit-stride reads nor the
// Ns-strided Stockham writes of a half-warp meet twice on one pair.  When the
// lanes of a warp interleave cb lines (lane = t cb + c), line c's region starts
// c region_stride(n, cb) elements in, n + 16 / cb apart, which puts the lines'
// pairs evenly apart; region_len(n) = n + 16 bounds every stride, for sizing.
// 16-byte elements: one padding element after every 128 bytes.
template <typename C> __host__ __device__ constexpr int pad_shift() {
    return sizeof(C) == 8 ? 4 : 3;
}
template <typename C> __device__ __forceinline__ int spad(int i) {
    if constexpr (sizeof(C) == 8) return i ^ ((i >> 3) & 15);
    else return i + (i >> pad_shift<C>());
}
template <typename C> __host__ __device__ constexpr int region_len(int n) {
    return sizeof(C) == 8 ? n + 16 : n + (n >> pad_shift<C>());
}
template <typename C> __host__ __device__ constexpr int region_stride(int n, int cb) {
    return sizeof(C) == 8 ? n + (cb >= 16 ? 1 : 16 / cb) : region_len<C>(n);
}

// One radix-R Stockham stage over the E register elements of thread t.  Thread
// t owns butterflies j = t + k T (k < E/R) whose inputs are
// x[j + r N/R] = v[k + r (E/R)]; output r of butterfly j goes to index
// (j - j mod Ns) R + j mod Ns + r Ns.
template <int R, int E, int K, typename C, class St>
__device__ __forceinline__ void stockham_butterfly(C *v, int t, int T, int Ns, int tsh,
                                                   const C *__restrict__ tw, bool last, C *sm,
                                                   St &st) {
    // tsh = log2(N / (Ns R)) + twiddle-table stride shift: twiddle of input r is
    // tw[(r jm) << tsh] = e^{+2 pi i r jm / (Ns R)}
    constexpr int G = E / R;
    if constexpr (K < G) {
        const int j = t + K * T;
        const int jm = j & (Ns - 1);
        if (Ns > 1) {
            const int d = jm << tsh;
#pragma unroll
            for (int r = 1; r < R; ++r) v[K + r * G] = cmul(v[K + r * G], ldt(&tw[r * d]));
        }
        dif_levels<R, K, G, R / 2>(v);
        const int base = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int o = base + bitrev(r, R) * Ns;
            if (last) st(o, v[K + r * G]);
            else sm[spad<C>(o)] = v[K + r * G];
        }
        stockham_butterfly<R, E, K + 1>(v, t, T, Ns, tsh, tw, last, sm, st);
    }
}

// Length-N (N = 2^logN, E <= N <= 8192) inverse FFT of one line held by the
// N/E threads t = 0..N/E-1, E elements each; every thread of the CTA must call
// it (it synchronises the CTA between stages).  ld(i) gives input element i,
// st(i, value) receives output element i.  Stages are radix E, then one stage
// for the remaining factor.  tw[k << tws] = e^{+2 pi i k / N}.
template <int E, typename C, class Ld, class St>
__device__ __forceinline__ void line_fft(int logN, const C *__restrict__ tw, int tws, C *sm,
                                         int t, Ld &ld, St &st) {
    constexpr int LE = E == 16 ? 4 : E == 8 ? 3 : 2;
    const int N = 1 << logN;
    const int T = N / E;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = ld(t + e * T);
    int Ns = 1, lns = 0;
    int rem = logN;
    bool first = true;
    while (rem > 0) {
        const int lr = rem >= LE ? LE : rem;
        rem -= lr;
        const bool last = rem == 0;
        const int tsh = (logN - lns - lr) + tws;
        if (!first) {
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = sm[spad<C>(t + e * T)];
            __syncthreads();
        }
        switch (lr) {
            case 4:
                if constexpr (E >= 16) stockham_butterfly<16, E, 0>(v, t, T, Ns, tsh, tw, last, sm, st);
                break;
            case 3:
                if constexpr (E >= 8) stockham_butterfly<8, E, 0>(v, t, T, Ns, tsh, tw, last, sm, st);
                break;
            case 2: stockham_butterfly<4, E, 0>(v, t, T, Ns, tsh, tw, last, sm, st); break;
            default: stockham_butterfly<2, E, 0>(v, t, T, Ns, tsh, tw, last, sm, st); break;
        }
        first = false;
        Ns <<= lr;
        lns += lr;
    }
}



// ---- compile-time-length driver
//
// Its twiddles come from a stage-ordered table: for every stage after the
// first (Ns = product of the earlier radices, radix R) a block of (R - 1) Ns
// entries, entry (r - 1) Ns + jm = e^{+2 pi i r jm / (Ns R)}.  Consecutive
// threads have consecutive jm, so each table read is coalesced.

// Offset of the stage starting at log2(Ns) = LNS in the stage-ordered table.
__host__ __device__ constexpr int stage_table_offset(int logn, int e, int lns) {
    const int le = e == 16 ? 4 : e == 8 ? 3 : 2;
    int off = 0, l = 0;
    while (l < lns) {
        const int lr = (logn - l) >= le ? le : (logn - l);
        if (l > 0) off += ((1 << lr) - 1) << l;
        l += lr;
    }
    return off;
}

// Entries of the stage-ordered table of a length-2^logn transform.
__host__ __device__ constexpr int stage_table_size(int logn, int e) {
    return stage_table_offset(logn, e, logn);
}

template <int R, int E, int K, int NS, int OFF, int T, bool LAST, typename C, class St>
__device__ __forceinline__ void ct_butterfly(C *v, int t, const C *__restrict__ stw, C *sm,
                                             St &st) {
    constexpr int G = E / R;
    if constexpr (K < G) {
        const int j = t + K * T;
        const int jm = j & (NS - 1);
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r)
                v[K + r * G] = cmul(v[K + r * G], ldt(&stw[OFF + (r - 1) * NS + jm]));
        }
        dif_levels<R, K, G, R / 2>(v);
        const int base = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int o = base + bitrev(r, R) * NS;
            if constexpr (LAST) st(o, v[K + r * G]);
            else sm[spad<C>(o)] = v[K + r * G];
        }
        ct_butterfly<R, E, K + 1, NS, OFF, T, LAST>(v, t, stw, sm, st);
    }
}

template <int LOGN, int E, int LNS, typename C, class St>
__device__ __forceinline__ void ct_stages(C *v, int t, const C *__restrict__ stw, C *sm,
                                          St &st) {
    constexpr int LE = E == 16 ? 4 : E == 8 ? 3 : 2;
    constexpr int REM = LOGN - LNS;
    if constexpr (REM > 0) {
        constexpr int LR = REM >= LE ? LE : REM;
        constexpr int T = (1 << LOGN) / E;
        if constexpr (LNS > 0) {
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = sm[spad<C>(t + e * T)];
            __syncthreads();
        }
        ct_butterfly<(1 << LR), E, 0, (1 << LNS), stage_table_offset(LOGN, E, LNS), T,
                     REM == LR>(v, t, stw, sm, st);
        ct_stages<LOGN, E, LNS + LR>(v, t, stw, sm, st);
    }
}

// Length 2^LOGN inverse FFT of one line (see line_fft), everything unrolled;
// stw is the stage-ordered twiddle table of this length and E.
template <int LOGN, int E, typename C, class Ld, class St>
__device__ __forceinline__ void line_fft_ct(const C *__restrict__ stw, C *sm, int t, Ld &ld,
                                            St &st) {
    constexpr int T = (1 << LOGN) / E;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = ld(t + e * T);
    ct_stages<LOGN, E, 0>(v, t, stw, sm, st);
}

// ---- two lines at once (compile-time length)
//
// The same transform applied to two register sets v0 and v1 (for instance the
// two half-length transforms of one column): twiddle loads, index arithmetic
// and barriers are shared, and each set exchanges through its own region.
// after_first_barrier() runs on every thread right after the first barrier,
// when no thread reads the inputs any more (the caller may refill them).

template <int R, int E, int K, int NS, int OFF, int T, bool LAST, typename C, class St>
__device__ __forceinline__ void ct_butterfly2(C *v0, C *v1, int t, const C *__restrict__ stw,
                                              C *sm0, C *sm1, St &st) {
    constexpr int G = E / R;
    if constexpr (K < G) {
        const int j = t + K * T;
        const int jm = j & (NS - 1);
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const C w = ldt(&stw[OFF + (r - 1) * NS + jm]);
                v0[K + r * G] = cmul(v0[K + r * G], w);
                v1[K + r * G] = cmul(v1[K + r * G], w);
            }
        }
        dif_levels<R, K, G, R / 2>(v0);
        dif_levels<R, K, G, R / 2>(v1);
        const int base = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int o = base + bitrev(r, R) * NS;
            if constexpr (LAST) {
                st(o, v0[K + r * G], v1[K + r * G]);
            } else {
                sm0[spad<C>(o)] = v0[K + r * G];
                sm1[spad<C>(o)] = v1[K + r * G];
            }
        }
        ct_butterfly2<R, E, K + 1, NS, OFF, T, LAST>(v0, v1, t, stw, sm0, sm1, st);
    }
}

template <int LOGN, int E, int LNS, typename C, class St, class Hook>
__device__ __forceinline__ void ct_stages2(C *v0, C *v1, int t, const C *__restrict__ stw,
                                           C *sm0, C *sm1, St &st, Hook &after_first_barrier) {
    constexpr int LE = E == 16 ? 4 : E == 8 ? 3 : 2;
    constexpr int REM = LOGN - LNS;
    if constexpr (REM > 0) {
        constexpr int LR = REM >= LE ? LE : REM;
        constexpr int T = (1 << LOGN) / E;
        if constexpr (LNS > 0) {
            __syncthreads();
            if constexpr (LNS == LE) after_first_barrier();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                v0[e] = sm0[spad<C>(t + e * T)];
                v1[e] = sm1[spad<C>(t + e * T)];
            }
            __syncthreads();
        }
        ct_butterfly2<(1 << LR), E, 0, (1 << LNS), stage_table_offset(LOGN, E, LNS), T,
                      REM == LR>(v0, v1, t, stw, sm0, sm1, st);
        ct_stages2<LOGN, E, LNS + LR>(v0, v1, t, stw, sm0, sm1, st, after_first_barrier);
    }
}

// Two length-2^LOGN inverse FFTs (LOGN > LE: at least two stages) held by the
// same threads: ld(i, a, b) gives input i of both, st(i, a, b) takes output i.
template <int LOGN, int E, typename C, class Ld, class St, class Hook>
__device__ __forceinline__ void line_fft_ct2(const C *__restrict__ stw, C *sm0, C *sm1, int t,
                                             Ld &ld, St &st, Hook &after_first_barrier) {
    constexpr int T = (1 << LOGN) / E;
    C v0[E], v1[E];
#pragma unroll
    for (int e = 0; e < E; ++e) ld(t + e * T, v0[e], v1[e]);
    ct_stages2<LOGN, E, 0>(v0, v1, t, stw, sm0, sm1, st, after_first_barrier);
}

__host__ __device__ __forceinline__ int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    return dfs_allow_smem((const void *)kernel, bytes);
}

}  // namespace dfs_fft

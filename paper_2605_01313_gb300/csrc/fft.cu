// Deconvolve-and-pad plus the two passes of the oversampled 2-D inverse FFT
// (sign +1, unnormalised), the middle stages of the type-2 NUFFT that
// evaluates Eq. 5.3 (Sec. 5).
//
//   theta pass: for each phi-mode column q (m = q - N1/2), place the N2 theta
//     modes, each divided by phihat2(n) phihat1(m), at fine index n mod n2
//     (zeros elsewhere), inverse-FFT the length-n2 column, and store the fine
//     rows that some point's stencil touches:  T[f][row][q].
//   phi pass: for each needed fine row, the real part of the inverse FFT of the
//     N1 values placed at m mod n1: a complex-to-real transform of length n1
//     done as a complex FFT of length n1 / 2, into the real fine grid
//     G[f][row][:].
//
// The transforms are Stockham autosort FFTs (radix-16 stages, a radix 2/4/8
// stage for the remainder): each thread keeps 16 elements in registers, does
// its butterflies there, and exchanges through padded shared memory between
// stages, so each element crosses shared memory once per stage after the
// first.  Zero inputs of the pruned (half-empty) transforms are never read.
#include "common.cuh"

namespace {

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

__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

// One radix-R Stockham stage over the E register elements of thread t.  Thread
// t owns butterflies j = t + k T (k < E/R) whose inputs are
// x[j + r N/R] = v[k + r (E/R)]; output r of butterfly j goes to index
// (j - j mod Ns) R + j mod Ns + r Ns.
template <int R, int E, int K, typename C, class St>
__device__ __forceinline__ void stockham_butterfly(C *v, int t, int T, int N, int Ns,
                                                   const C *__restrict__ tw, int tws, bool last,
                                                   C *sm, St &st) {
    constexpr int G = E / R;
    if constexpr (K < G) {
        const int j = t + K * T;
        const int jm = j & (Ns - 1);
        if (Ns > 1) {
            const int step = (N / (Ns * R)) * jm;
#pragma unroll
            for (int r = 1; r < R; ++r)
                v[K + r * G] = cmul(v[K + r * G], __ldg(&tw[(r * step) << tws]));
        }
        dif_levels<R, K, G, R / 2>(v);
        const int base = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int o = base + bitrev(r, R) * Ns;
            if (last) st(o, v[K + r * G]);
            else sm[spad(o)] = v[K + r * G];
        }
        stockham_butterfly<R, E, K + 1>(v, t, T, N, Ns, tw, tws, last, sm, st);
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
    int Ns = 1;
    int rem = logN;
    bool first = true;
    while (rem > 0) {
        const int lr = rem >= LE ? LE : rem;
        rem -= lr;
        const bool last = rem == 0;
        if (!first) {
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = sm[spad(t + e * T)];
            __syncthreads();
        }
        switch (lr) {
            case 4:
                if constexpr (E >= 16) stockham_butterfly<16, E, 0>(v, t, T, N, Ns, tw, tws, last, sm, st);
                break;
            case 3:
                if constexpr (E >= 8) stockham_butterfly<8, E, 0>(v, t, T, N, Ns, tw, tws, last, sm, st);
                break;
            case 2: stockham_butterfly<4, E, 0>(v, t, T, N, Ns, tw, tws, last, sm, st); break;
            default: stockham_butterfly<2, E, 0>(v, t, T, N, Ns, tw, tws, last, sm, st); break;
        }
        first = false;
        Ns <<= lr;
    }
}

__host__ __device__ __forceinline__ int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

struct ThetaArgs {
    int N1, N2, n2, logn2;
    int CB;                   // columns per CTA
};

// grid (ceil(N1 / CB), n_fields); block CB * n2/E threads, thread = (t, c) with c fastest.
template <typename R, int E, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
    k_theta_pass(ThetaArgs a, const typename CxT<R>::type *__restrict__ coef,
                 const R *__restrict__ inv1, const R *__restrict__ inv2,
                 const typename CxT<R>::type *__restrict__ tw,
                 const unsigned char *__restrict__ rowmask, typename CxT<R>::type *__restrict__ out) {
    typedef typename CxT<R>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *smem = reinterpret_cast<C *>(smem_raw);
    const int c = threadIdx.x % a.CB;
    const int t = threadIdx.x / a.CB;
    const int q = blockIdx.x * a.CB + c;
    const int f = blockIdx.y;
    const bool col_ok = q < a.N1;
    const C *src = coef + (size_t)f * a.N2 * a.N1 + q;
    C *dst = out + (size_t)f * a.n2 * a.N1 + q;
    const int half = a.N2 / 2;
    const R sq = col_ok ? inv1[q] : (R)0;
    C *sm = smem + (size_t)c * (a.n2 + (a.n2 >> 4));
    auto ld = [&](int i) -> C {
        int n;
        if (i < half) n = i;
        else if (i >= a.n2 - half) n = i - a.n2;
        else return cmake((R)0, (R)0);
        if (!col_ok) return cmake((R)0, (R)0);
        const int r = n + half;
        const C v = src[(size_t)r * a.N1];
        const R s = sq * inv2[r];
        return cmake(v.x * s, v.y * s);
    };
    auto st = [&](int i, C v) {
        if (col_ok && rowmask[i / DFS_ROW_BLOCK]) dst[(size_t)i * a.N1] = v;
    };
    line_fft<E>(a.logn2, tw, 0, sm, t, ld, st);
}

struct PhiArgs {
    int N1, n1, logm, n2;     // logm = log2(n1 / 2)
    int CB;                   // rows per CTA (divides DFS_ROW_BLOCK)
};

// Only the real part of the fine grid is needed (the interpolation weights are
// real and the values are Re v), so each row is a complex-to-real transform:
// Re g(j) = sum_k H_k e^{2 pi i k j / n1} with H_k = (T_k + conj T_{-k}) / 2
// Hermitian.  With M = n1 / 2 and Z_k = (H_k + H_{k+M}) + i e^{2 pi i k / n1}
// (H_k - H_{k+M}), the length-M inverse FFT z of Z gives
// Re g(2j) = Re z_j and Re g(2j+1) = Im z_j.  T_k is the theta-pass value at
// phi-mode k mod n1 (zero outside the N1 modes).
//
// grid (n2 / CB, n_fields); block CB * M/E threads, thread = (t, c) with t fastest.
template <typename R, int E, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
    k_phi_pass(PhiArgs a, const typename CxT<R>::type *__restrict__ in,
               const typename CxT<R>::type *__restrict__ tw,
               const unsigned char *__restrict__ rowmask, R *__restrict__ grid) {
    typedef typename CxT<R>::type C;
    const int row0 = blockIdx.x * a.CB;
    if (!rowmask[row0 / DFS_ROW_BLOCK]) return;     // whole CTA: no stencil touches these rows
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *smem = reinterpret_cast<C *>(smem_raw);
    const int M = 1 << a.logm;
    const int T = M / E;
    const int t = threadIdx.x % T;
    const int c = threadIdx.x / T;
    const int row = row0 + c;
    const int f = blockIdx.y;
    const C *src = in + ((size_t)f * a.n2 + row) * a.N1;
    R *dst = grid + ((size_t)f * a.n2 + row) * a.n1;
    const int half = a.N1 / 2;
    const int nmask = a.n1 - 1;
    C *sm = smem + (size_t)c * (M + (M >> 4));
    auto tval = [&](int k) -> C {              // T_k, k taken mod n1
        k &= nmask;
        int m;
        if (k < half) m = k;
        else if (k >= a.n1 - half) m = k - a.n1;
        else return cmake((R)0, (R)0);
        return src[m + half];
    };
    auto ld = [&](int k) -> C {
        const C t0 = tval(k), t1 = tval(-k), t2 = tval(k + M), t3 = tval(M - k);
        // 2 H_k = T_k + conj T_{-k},  2 H_{k+M} = T_{k+M} + conj T_{M-k}
        const C h0 = cmake(t0.x + t1.x, t0.y - t1.y);
        const C h1 = cmake(t2.x + t3.x, t2.y - t3.y);
        const C d = cmul(cmake(h0.x - h1.x, h0.y - h1.y), __ldg(&tw[k]));
        // (h0 + h1 + i d) / 2
        return cmake((R)0.5 * (h0.x + h1.x - d.y), (R)0.5 * (h0.y + h1.y + d.x));
    };
    auto st = [&](int j, C z) { reinterpret_cast<C *>(dst)[j] = z; };
    line_fft<E>(a.logm, tw, 1, sm, t, ld, st);
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Per precision and pass: elements per thread E, threads per CTA at most MAXT,
// and the resident CTAs MINB the register budget (65536 / (MAXT MINB)) is set for.
template <typename R> struct ThetaCfg;
template <> struct ThetaCfg<float> { static const int E = 8, MAXT = 1024, MINB = 1; };
template <> struct ThetaCfg<double> { static const int E = 8, MAXT = 512, MINB = 1; };
template <typename R> struct PhiCfg;
template <> struct PhiCfg<float> { static const int E = 8, MAXT = 256, MINB = 3; };
template <> struct PhiCfg<double> { static const int E = 8, MAXT = 512, MINB = 1; };

template <typename R>
cudaError_t launch_theta(dfsnufft_plan p, const void *coeffs) {
    typedef typename CxT<R>::type C;
    constexpr int E = ThetaCfg<R>::E, MAXT = ThetaCfg<R>::MAXT, MINB = ThetaCfg<R>::MINB;
    const dfsnufft_params &q = p->prm;
    ThetaArgs a;
    a.N1 = q.N1;
    a.N2 = q.N2;
    a.n2 = q.n2;
    a.logn2 = ilog2(q.n2);
    const int T = q.n2 / E;
    int cb = MAXT / T;
    if (cb < 1) cb = 1;
    int n1p = 1;
    while (n1p < q.N1) n1p <<= 1;
    if (cb > n1p) cb = n1p;
    const size_t per_col = sizeof(C) * (size_t)(q.n2 + (q.n2 >> 4));
    while (cb > 1 && per_col * cb > 160 * 1024) cb >>= 1;
    a.CB = cb;
    const size_t smem = per_col * cb;
    cudaError_t e = allow_smem(k_theta_pass<R, E, MAXT, MINB>, smem);
    if (e) return e;
    dim3 grid((q.N1 + cb - 1) / cb, p->n_fields);
    k_theta_pass<R, E, MAXT, MINB><<<grid, cb * T, smem, p->stream>>>(
        a, (const C *)coeffs, (const R *)p->d_inv1, (const R *)p->d_inv2, (const C *)p->d_tw2,
        p->d_rowmask, (C *)p->d_T);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_phi(dfsnufft_plan p) {
    typedef typename CxT<R>::type C;
    constexpr int E = PhiCfg<R>::E, MAXT = PhiCfg<R>::MAXT, MINB = PhiCfg<R>::MINB;
    const dfsnufft_params &q = p->prm;
    PhiArgs a;
    a.N1 = q.N1;
    a.n1 = q.n1;
    a.logm = ilog2(q.n1) - 1;
    a.n2 = q.n2;
    const int M = q.n1 / 2;
    const int T = M / E;
    int cb = MAXT / T;
    if (cb < 1) cb = 1;
    if (cb > DFS_ROW_BLOCK) cb = DFS_ROW_BLOCK;
    const size_t per_row = sizeof(C) * (size_t)(M + (M >> 4));
    while (cb > 1 && per_row * cb > 160 * 1024) cb >>= 1;
    a.CB = cb;
    const size_t smem = per_row * cb;
    cudaError_t e = allow_smem(k_phi_pass<R, E, MAXT, MINB>, smem);
    if (e) return e;
    dim3 grid(q.n2 / cb, p->n_fields);
    k_phi_pass<R, E, MAXT, MINB><<<grid, cb * T, smem, p->stream>>>(
        a, (const C *)p->d_T, (const C *)p->d_tw1, p->d_rowmask, (R *)p->d_G);
    return cudaGetLastError();
}

}  // namespace

cudaError_t dfs_launch_theta_pass(dfsnufft_plan p, const void *coeffs) {
    return p->prm.dtype == DFSNUFFT_F64 ? launch_theta<double>(p, coeffs)
                                        : launch_theta<float>(p, coeffs);
}

cudaError_t dfs_launch_phi_pass(dfsnufft_plan p) {
    return p->prm.dtype == DFSNUFFT_F64 ? launch_phi<double>(p) : launch_phi<float>(p);
}

// Deconvolve-and-pad plus the two passes of the oversampled 2-D inverse FFT
// (sign +1, unnormalised), the middle stages of the type-2 NUFFT that
// evaluates Eq. 5.3 (Sec. 5).
//
//   theta pass: for each phi-mode column q (m = q - N1/2), place the N2 theta
//     modes, each divided by phihat2(n) phihat1(m), at fine index n mod n2
//     (zeros elsewhere), inverse-FFT the length-n2 column, and store the fine
//     rows that some point's stencil touches:  T[f][row][q].
//   phi pass: for each needed fine row, place the N1 values at m mod n1 and
//     inverse-FFT the length-n1 row into the fine grid G[f][row][:].
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

// In-register DFT of size R (power of two <= 16), sign +1, natural order,
// by recursive radix-2 decimation in time; all indices resolve at compile time.
template <int R>
struct Dft {
    template <typename C>
    static __device__ __forceinline__ void run(C *v) {
        C e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        Dft<R / 2>::run(e);
        Dft<R / 2>::run(o);
        combine<0>(v, e, o);
    }
    template <int K, typename C>
    static __device__ __forceinline__ void combine(C *v, const C *e, const C *o) {
        if constexpr (K < R / 2) {
            C t = tw16<K * (16 / R)>(o[K]);
            v[K] = e[K] + t;
            v[K + R / 2] = e[K] - t;
            combine<K + 1>(v, e, o);
        }
    }
};
template <>
struct Dft<1> {
    template <typename C>
    static __device__ __forceinline__ void run(C *) {}
};

__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

// One radix-R Stockham stage over the 16 register elements of thread t.
// Thread t owns butterflies j = t + k T (k < 16/R) whose inputs are
// x[j + r N/R] = v[k + r (16/R)].
template <int R, typename C, class St>
__device__ __forceinline__ void stockham_stage(C *v, int t, int T, int N, int Ns,
                                               const C *__restrict__ tw, bool last, C *sm,
                                               St &st) {
    constexpr int G = 16 / R;
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const int j = t + k * T;
        const int jm = j & (Ns - 1);
        C u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = v[k + r * G];
        if (Ns > 1) {
            const int step = (N / (Ns * R)) * jm;
#pragma unroll
            for (int r = 1; r < R; ++r) u[r] = cmul(u[r], __ldg(&tw[r * step]));
        }
        Dft<R>::run(u);
        const int base = (j - jm) * R + jm;
        if (last) {
#pragma unroll
            for (int r = 0; r < R; ++r) st(base + r * Ns, u[r]);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) sm[spad(base + r * Ns)] = u[r];
        }
    }
}

// Length-N (N = 2^logN, 16 <= N <= 8192) inverse FFT of one line held by the
// N/16 threads t = 0..N/16-1; every thread of the CTA must call it (it
// synchronises the CTA between stages).  ld(i) gives input element i,
// st(i, value) receives output element i.
template <typename C, class Ld, class St>
__device__ __forceinline__ void line_fft(int logN, const C *__restrict__ tw, C *sm, int t,
                                         Ld &ld, St &st) {
    const int N = 1 << logN;
    const int T = N >> 4;
    C v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = ld(t + e * T);
    int Ns = 1;
    int rem = logN;
    bool first = true;
    while (rem > 0) {
        const int lr = rem >= 4 ? 4 : rem;
        rem -= lr;
        const bool last = rem == 0;
        if (!first) {
            __syncthreads();
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = sm[spad(t + e * T)];
            __syncthreads();
        }
        switch (lr) {
            case 4: stockham_stage<16>(v, t, T, N, Ns, tw, last, sm, st); break;
            case 3: stockham_stage<8>(v, t, T, N, Ns, tw, last, sm, st); break;
            case 2: stockham_stage<4>(v, t, T, N, Ns, tw, last, sm, st); break;
            default: stockham_stage<2>(v, t, T, N, Ns, tw, last, sm, st); break;
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
    int n_row_blocks;
};

// grid (ceil(N1 / CB), n_fields); block CB * n2/16 threads, thread = (t, c) with c fastest.
template <typename R>
__global__ void __launch_bounds__(512) k_theta_pass(ThetaArgs a,
                                                    const typename CxT<R>::type *__restrict__ coef,
                                                    const double *__restrict__ inv1,
                                                    const double *__restrict__ inv2,
                                                    const typename CxT<R>::type *__restrict__ tw,
                                                    const unsigned char *__restrict__ rowmask,
                                                    typename CxT<R>::type *__restrict__ out) {
    typedef typename CxT<R>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *smem = reinterpret_cast<C *>(smem_raw);
    const int c = threadIdx.x % a.CB;
    const int t = threadIdx.x / a.CB;
    const int q = blockIdx.x * a.CB + c;
    const int f = blockIdx.y;
    const bool col_ok = q < a.N1;
    const size_t fofs = (size_t)f * a.N2 * a.N1;
    const size_t oofs = (size_t)f * a.n2 * a.N1;
    const int half = a.N2 / 2;
    const double sq = col_ok ? inv1[q] : 0.0;
    C *sm = smem + (size_t)c * (a.n2 + (a.n2 >> 4));
    auto ld = [&](int i) -> C {
        int n;
        if (i < half) n = i;
        else if (i >= a.n2 - half) n = i - a.n2;
        else return cmake((R)0, (R)0);
        if (!col_ok) return cmake((R)0, (R)0);
        const int r = n + half;
        C v = coef[fofs + (size_t)r * a.N1 + q];
        const double s = sq * inv2[r];
        return cmake((R)((double)v.x * s), (R)((double)v.y * s));
    };
    auto st = [&](int i, C v) {
        if (col_ok && rowmask[i / DFS_ROW_BLOCK]) out[oofs + (size_t)i * a.N1 + q] = v;
    };
    line_fft(a.logn2, tw, sm, t, ld, st);
}

struct PhiArgs {
    int N1, n1, logn1, n2;
    int CB;                   // rows per CTA (divides DFS_ROW_BLOCK)
};

// grid (n2 / CB, n_fields); block CB * n1/16 threads, thread = (t, c) with t fastest.
template <typename R>
__global__ void __launch_bounds__(512) k_phi_pass(PhiArgs a,
                                                  const typename CxT<R>::type *__restrict__ in,
                                                  const typename CxT<R>::type *__restrict__ tw,
                                                  const unsigned char *__restrict__ rowmask,
                                                  typename CxT<R>::type *__restrict__ grid) {
    typedef typename CxT<R>::type C;
    const int row0 = blockIdx.x * a.CB;
    if (!rowmask[row0 / DFS_ROW_BLOCK]) return;     // whole CTA: no stencil touches these rows
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *smem = reinterpret_cast<C *>(smem_raw);
    const int T = a.n1 >> 4;
    const int t = threadIdx.x % T;
    const int c = threadIdx.x / T;
    const int row = row0 + c;
    const int f = blockIdx.y;
    const C *src = in + ((size_t)f * a.n2 + row) * a.N1;
    C *dst = grid + ((size_t)f * a.n2 + row) * a.n1;
    const int half = a.N1 / 2;
    C *sm = smem + (size_t)c * (a.n1 + (a.n1 >> 4));
    auto ld = [&](int i) -> C {
        int m;
        if (i < half) m = i;
        else if (i >= a.n1 - half) m = i - a.n1;
        else return cmake((R)0, (R)0);
        return src[m + half];
    };
    auto st = [&](int i, C v) { dst[i] = v; };
    line_fft(a.logn1, tw, sm, t, ld, st);
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R>
cudaError_t launch_theta(dfsnufft_plan p, const void *coeffs) {
    typedef typename CxT<R>::type C;
    const dfsnufft_params &q = p->prm;
    ThetaArgs a;
    a.N1 = q.N1;
    a.N2 = q.N2;
    a.n2 = q.n2;
    a.logn2 = ilog2(q.n2);
    const int T = q.n2 >> 4;
    int cb = 512 / T;
    if (cb < 1) cb = 1;
    int n1p = 1;
    while (n1p < q.N1) n1p <<= 1;
    if (cb > n1p) cb = n1p;
    const size_t per_col = sizeof(C) * (size_t)(q.n2 + (q.n2 >> 4));
    while (cb > 1 && per_col * cb > 160 * 1024) cb >>= 1;
    a.CB = cb;
    a.n_row_blocks = p->n_row_blocks;
    const size_t smem = per_col * cb;
    cudaError_t e = allow_smem(k_theta_pass<R>, smem);
    if (e) return e;
    dim3 grid((q.N1 + cb - 1) / cb, p->n_fields);
    k_theta_pass<R><<<grid, cb * T, smem, p->stream>>>(a, (const C *)coeffs, p->d_inv1, p->d_inv2,
                                                       (const C *)p->d_tw2, p->d_rowmask,
                                                       (C *)p->d_T);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_phi(dfsnufft_plan p) {
    typedef typename CxT<R>::type C;
    const dfsnufft_params &q = p->prm;
    PhiArgs a;
    a.N1 = q.N1;
    a.n1 = q.n1;
    a.logn1 = ilog2(q.n1);
    a.n2 = q.n2;
    const int T = q.n1 >> 4;
    int cb = 512 / T;
    if (cb < 1) cb = 1;
    if (cb > DFS_ROW_BLOCK) cb = DFS_ROW_BLOCK;
    const size_t per_row = sizeof(C) * (size_t)(q.n1 + (q.n1 >> 4));
    while (cb > 1 && per_row * cb > 160 * 1024) cb >>= 1;
    a.CB = cb;
    const size_t smem = per_row * cb;
    cudaError_t e = allow_smem(k_phi_pass<R>, smem);
    if (e) return e;
    dim3 grid(q.n2 / cb, p->n_fields);
    k_phi_pass<R><<<grid, cb * T, smem, p->stream>>>(a, (const C *)p->d_T, (const C *)p->d_tw1,
                                                     p->d_rowmask, (C *)p->d_G);
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

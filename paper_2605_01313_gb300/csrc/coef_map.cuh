// Coefficient helpers shared by the column passes of the inverse FFT (the
// theta pass and the persistent ensemble step): conjugation, scaling and the
// Hermitian part a real-field plan transforms (Sec. 5 evaluation of Eq. 5.3 for
// real fields, whose values depend on that part only).
#pragma once

#include "common.cuh"

namespace dfs_coef {

template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake(a.x, -a.y); }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) {
    return cmake(a.x * s, a.y * s);
}

// The Hermitian part h_{n,k} = (c_{n,k} + conj c_{-n,-k}) / 2 that a real-field
// plan transforms, for -half <= n <= half and 0 <= k <= N1/2, from a reader
// cf(row, col) of the centred coefficient array that returns zero outside it
// (half = N2/2).  Entries whose mirror lies outside the even-sized array (the
// Nyquist row n = -N2/2 and column m = -N1/2) are split exactly into c/2 at
// (n, m) and conj(c)/2 at (-n, -m); column k = 0 is its own mirror.
template <typename C, class Rd>
__device__ __forceinline__ C herm_coef(int n, int k, int half, int N1, Rd &cf) {
    typedef decltype(C().x) R;
    const int N1h = N1 / 2;
    const int qa = N1h + k;                        // array column of m = k (N1 if k = N1/2)
    if (k == N1h)                                  // mirror of the Nyquist column
        return n == -half ? cmake((R)0, (R)0) : cscale(cconj(cf(half - n, 0)), (R)0.5);
    if (n == half) return cscale(cconj(cf(0, N1 - qa)), (R)0.5);   // mirror of the Nyquist row
    const C c = cf(n + half, qa);
    if (n == -half) return cscale(c, (R)0.5);
    if (k == 0) {
        const C mirror = cf(half - n, qa);
        return cscale(cmake(c.x + mirror.x, c.y - mirror.y), (R)0.5);
    }
    return c;
}

}  // namespace dfs_coef

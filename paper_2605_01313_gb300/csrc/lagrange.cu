// Tensor-product cubic and quintic Lagrange interpolation of Grid [0] samples
// at arbitrary points: the interpolation of the paper's baseline model (cubic
// for the scalar forcing, quintic for the vector one; Sec. 1-2), here as a
// comparator for the spectral path.
//
// One thread per point, all fields.  The colatitude is reduced to [-pi, pi);
// a negative one is the point (phi + pi, -theta) of the doubled sphere, where a
// field is its parity times its value (Sec. 4).  The stencil is the (ORD + 1)^2
// nodes around the point in grid-index space, x = phi n_lon / (2 pi),
// y = theta n_lat / pi - 1/2; rows beyond a pole come from the same extension
// (the row mirrored about the pole, half a turn away, times the parity).
// Positions are reduced exactly in integer arithmetic (fractions of a turn in
// Q0.64, turns.cuh), so no FP64 arithmetic runs in the FP32 form; weights and
// sums run in the precision R.  A coordinate that is not finite or of
// magnitude 2^53 rad or more gives NaN values.
#include "common.cuh"
#include "turns.cuh"

namespace {

struct LagArgs {
    int n_lon, n_lat, F;
    long long n_points;
    unsigned vec_mask;        // bit f: field f is a wind component (parity -1)
};

// A Q0.64 fraction as a value in [0, 1) of precision R.
__device__ __forceinline__ float q64_unit(unsigned long long q, float) {
    return (float)(unsigned)(q >> 40) * 0x1p-24f;
}
__device__ __forceinline__ double q64_unit(unsigned long long q, double) {
    return (double)(q >> 11) * 0x1p-53;
}

// Weights of the Lagrange interpolant through the nodes -H .. ORD - H at t.
template <typename R, int ORD>
__device__ __forceinline__ void weights(R t, R *L) {
    constexpr int H = (ORD - 1) / 2;
#pragma unroll
    for (int a = 0; a <= ORD; ++a) {
        R num = 1;
        double den = 1;
#pragma unroll
        for (int b = 0; b <= ORD; ++b) {
            if (b == a) continue;
            num *= t - (R)(b - H);
            den *= (double)(a - b);
        }
        L[a] = num * (R)(1.0 / den);
    }
}

// grid ceil(n_points / 256); block 256.  samples: F x n_lat x n_lon; values:
// F x n_points.
template <typename R, int ORD>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_lagrange(LagArgs a, const double *__restrict__ lon,
                                                  const double *__restrict__ colat,
                                                  const R *__restrict__ samples,
                                                  R *__restrict__ values) {
    constexpr int NP = ORD + 1, H = (ORD - 1) / 2;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_points) return;
    const int n = a.n_lon, nl = a.n_lat;
    // fractions of a turn: theta in [-1/2, 1/2) read signed; a negative one is
    // the point (phi + 1/2 turn, -theta)
    unsigned long long ux = 0, uy = 0;
    const bool ok = turns_q64(lon[p], ux) & turns_q64(colat[p], uy);
    const bool neg = (long long)uy < 0;
    if (neg) {
        uy = 0ULL - uy;                                            // in (0, 2^63]
        ux += 1ULL << 63;
    }
    // x = phi n / (2 pi) = ux n / 2^64: cell i and offset, exactly
    const int i = (int)__umul64hi(ux, (unsigned long long)n);      // in [0, n)
    const unsigned long long xf = ux * (unsigned long long)n;
    // y = theta n_lat / pi - 1/2 = uy 2 n_lat / 2^64 - 1/2
    const unsigned long long zi = __umul64hi(uy, 2ULL * nl);      // in [0, nl]
    const unsigned long long zf = uy * (2ULL * nl);
    const int j = (int)zi - (zf < (1ULL << 63) ? 1 : 0);           // in [-1, nl - 1]
    const unsigned long long yf = zf ^ (1ULL << 63);
    R Lx[NP], Ly[NP];
    weights<R, ORD>(q64_unit(xf, R()), Lx);
    weights<R, ORD>(q64_unit(yf, R()), Ly);
    const size_t plane = (size_t)nl * n;
    if (j >= H && j - H + ORD < nl && i >= H && i - H + ORD < n) {
        // the common case: the stencil lies inside the grid (no pole, no seam),
        // one address for all its rows
        const R *base = samples + (size_t)(j - H) * n + (i - H);
        for (int f = 0; f < a.F; ++f) {
            const R *s = base + (size_t)f * plane;
            R acc = 0;
#pragma unroll
            for (int r = 0; r < NP; ++r) {
                R t = 0;
#pragma unroll
                for (int b = 0; b < NP; ++b) t = fma(Lx[b], __ldg(s + r * n + b), t);
                acc = fma(Ly[r], t, acc);
            }
            const bool vec = (a.vec_mask >> f) & 1u;
            values[(size_t)f * a.n_points + p] = !ok ? (R)NAN : ((neg && vec) ? -acc : acc);
        }
        return;
    }
    // row offsets and the first column of each stencil row (mod n)
    int roff[NP], cfirst[NP];
    bool beyond[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) {
        const int rr = j - H + r;                                  // in [-1 - H, nl - 1 + ORD - H]
        beyond[r] = rr < 0 || rr >= nl;
        const int rm = rr < 0 ? -1 - rr : (rr >= nl ? 2 * nl - 1 - rr : rr);
        roff[r] = rm * n;
        int c = i - H + (beyond[r] ? n / 2 : 0);
        if (c < 0) c += n;
        else if (c >= n) c -= n;
        cfirst[r] = c;
    }
    for (int f = 0; f < a.F; ++f) {
        const R *s = samples + (size_t)f * plane;
        const bool vec = (a.vec_mask >> f) & 1u;
        R acc = 0;
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            const R *row = s + roff[r];
            const int c0 = cfirst[r];
            R t = 0;
            if (c0 <= n - NP) {
#pragma unroll
                for (int b = 0; b < NP; ++b) t = fma(Lx[b], __ldg(row + c0 + b), t);
            } else {
#pragma unroll
                for (int b = 0; b < NP; ++b) {
                    const int c = c0 + b < n ? c0 + b : c0 + b - n;
                    t = fma(Lx[b], __ldg(row + c), t);
                }
            }
            acc = fma((beyond[r] && vec) ? -Ly[r] : Ly[r], t, acc);
        }
        values[(size_t)f * a.n_points + p] = !ok ? (R)NAN : ((neg && vec) ? -acc : acc);
    }
}

template <typename R>
cudaError_t launch(const LagArgs &a, int order, const double *lon, const double *colat,
                   const void *samples, void *values, cudaStream_t st) {
    const unsigned blocks = (unsigned)((a.n_points + 255) / 256);
    if (order == 3)
        k_lagrange<R, 3><<<blocks, 256, 0, st>>>(a, lon, colat, (const R *)samples, (R *)values);
    else
        k_lagrange<R, 5><<<blocks, 256, 0, st>>>(a, lon, colat, (const R *)samples, (R *)values);
    return cudaGetLastError();
}

}  // namespace

extern "C" int dfsnufft_lagrange_interp(int n_lon, int n_lat, int n_fields, const int *parity,
                                        int order, int dtype, int64_t n_points,
                                        const double *lon, const double *colat,
                                        const void *samples, void *values, void *stream) {
    if (order != 3 && order != 5) return DFSNUFFT_ERR_INVALID_ARG;
    if (n_lon < order + 1 || (n_lon & 1) || n_lat < (order + 1) / 2 || n_fields < 1 ||
        n_fields > 32 || !parity || n_points < 1 || n_points > 0x7fffffffLL || !lon ||
        !colat || !samples || !values)
        return DFSNUFFT_ERR_INVALID_ARG;
    if ((long long)n_lon * n_lat > 0x7fffffffLL) return DFSNUFFT_ERR_INVALID_ARG;
    if (dtype != DFSNUFFT_F64 && dtype != DFSNUFFT_F32) return DFSNUFFT_ERR_INVALID_ARG;
    LagArgs a;
    a.n_lon = n_lon;
    a.n_lat = n_lat;
    a.F = n_fields;
    a.n_points = n_points;
    a.vec_mask = 0;
    for (int f = 0; f < n_fields; ++f) {
        if (parity[f] != 1 && parity[f] != -1) return DFSNUFFT_ERR_INVALID_ARG;
        if (parity[f] < 0) a.vec_mask |= 1u << f;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t e = dtype == DFSNUFFT_F64
                              ? launch<double>(a, order, lon, colat, samples, values, st)
                              : launch<float>(a, order, lon, colat, samples, values, st);
    return e == cudaSuccess ? DFSNUFFT_OK : DFSNUFFT_ERR_CUDA;
}

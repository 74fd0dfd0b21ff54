// Departure points of the semi-Lagrangian step and the rotation of vectors from
// the departure to the arrival frame (Sec. 2).
//
//  k_departure  Eq. 2.4 by fixed-point iteration, one thread per arrival point
//               of Grid [0]: D_0 = A; V_k = Q(A, D_k) W(D_k) - W_A(A);
//               D_{k+1} = the point reached from A along the great circle
//               leaving A in the direction -V_k, after the angle |V_k| dt / a.
//               W(D) is tensor-product quintic Lagrange interpolation of the
//               grid samples (the degree the paper uses for this bracket), rows
//               beyond a pole taken from the doubled sphere with the wind
//               components' sign change, f(phi + pi, -theta) = -f(phi, theta).
//  k_rotate     (u, v) at the departure points carried to the arrival frame by
//               Q = [[p, q], [-q, p]] (Sec. 2).
//
// The departure point is kept as a displacement from its arrival point, in the
// arrival point's frame turned by phi_A about the axis: with s = |V| dt / a,
//   X = sin th_A cos s - sin s t_n cos th_A,  Y = sin s t_e,
//   Z = cos th_A cos s + sin s t_n sin th_A        (t = -V / |V|, east/north),
// so that phi_D - phi_A = atan2(Y, X) and theta_D - theta_A follow without
// cancellation (below); positions are written in FP64 as phi_A + dphi,
// theta_A + dtheta.  In the same frame cos theta_D = Z, sin theta_D = rho =
// |(X, Y)|, cos(phi_D - phi_A) = X / rho, sin(...) = Y / rho and cos eta = cos s,
// which gives p and q without further trigonometry.
#include "common.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

template <typename R> struct DepArgs {
    int n_lon, n_lat, members, iterations;
    int P;                    // n_lat * n_lon
    double h_phi, h_th;       // 2 pi / n_lon, pi / n_lat
    R dta;                    // dt / a
    R to_x, to_y;             // n_lon / (2 pi), n_lat / pi: radians to grid cells
    R h_th_r;                 // pi / n_lat
};

template <typename R> struct Geo {
    R X, Y, Z, rho, inv_rho;  // the departure point in A's turned frame; rho = |(X, Y)|
    R dphi, dth;              // phi_D - phi_A, theta_D - theta_A
    R cs;                     // cos s = cos eta
};

__device__ __forceinline__ void sc(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sc(double x, double *s, double *c) { sincos(x, s, c); }

// sin and cos of a colatitude theta in [0, pi] (given in FP64) in precision R
// to a few units of R's rounding relative to each: in the southern half the
// angle is first reflected to pi - theta, whose rounding to R is relative to a
// small angle (theta itself rounded near pi would move sin theta by an absolute
// unit of R).
template <typename R>
__device__ __forceinline__ void colat_sc(double theta, R *s, R *c) {
    const bool south = theta > 0.5 * kPi;
    sc((R)(south ? kPi - theta : theta), s, c);
    if (south) *c = -*c;
}

// Elementary functions of the step's geometry.  FP64 takes the library's; FP32,
// whose angles per time step are small, takes the Taylor series of sin s,
// cos s - 1 and atan z for |s|, |z| <= 1/16 (the first dropped term is below
// 1e-10 of the result) and approximate reciprocals, and the library functions
// beyond.
__device__ __forceinline__ void sc_step(double s, double *ss, double *c1, double *cs) {
    sincos(s, ss, cs);
    *c1 = s < 0.5 ? -*ss * *ss / (1.0 + *cs) : *cs - 1.0;
}
__device__ __forceinline__ void sc_step(float s, float *ss, float *c1, float *cs) {
    if (s <= 0.0625f) {
        const float s2 = s * s;
        *ss = s * (1.f - s2 * (1.f / 6.f) * (1.f - s2 * (1.f / 20.f) * (1.f - s2 * (1.f / 42.f))));
        *c1 = -0.5f * s2 * (1.f - s2 * (1.f / 12.f) * (1.f - s2 * (1.f / 30.f)));
        *cs = 1.f + *c1;
    } else {
        sincosf(s, ss, cs);
        *c1 = s < 0.5f ? -*ss * *ss / (1.f + *cs) : *cs - 1.f;
    }
}
__device__ __forceinline__ double atan2_step(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float atan2_step(float y, float x) {
    if (x > 0.f && fabsf(y) <= 0.0625f * x) {
        const float z = __fdividef(y, x), z2 = z * z;
        return z * (1.f - z2 * (1.f / 3.f - z2 * (1.f / 5.f - z2 * (1.f / 7.f - z2 * (1.f / 9.f)))));
    }
    return atan2f(y, x);
}
__device__ __forceinline__ double rsqrt_step(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsqrt_step(float x) { return rsqrtf(x); }
__device__ __forceinline__ double div_step(double a, double b) { return a / b; }
__device__ __forceinline__ float div_step(float a, float b) { return __fdividef(a, b); }

// The point reached from A (sin/cos of its colatitude) by the angle |(se, sn)|
// along the great circle leaving A in the direction -(se, sn).
template <typename R>
__device__ __forceinline__ Geo<R> move_back(R sA, R cA, R se, R sn) {
    Geo<R> g;
    const R s2 = se * se + sn * sn;
    if (s2 == (R)0) {
        g.X = sA; g.Y = 0; g.Z = cA; g.rho = sA; g.dphi = 0; g.dth = 0; g.cs = 1;
        g.inv_rho = sA > (R)0 ? (R)1 / sA : (R)0;
        return g;
    }
    const R inv_s = rsqrt_step(s2);
    R ss, c1, cs;
    sc_step(s2 * inv_s, &ss, &c1, &cs);
    const R te = -se * inv_s, tn = -sn * inv_s;
    g.X = sA + (c1 * sA - ss * tn * cA);
    g.Y = ss * te;
    g.Z = cA + (c1 * cA + ss * tn * sA);
    const R rho2 = g.X * g.X + g.Y * g.Y;
    g.inv_rho = rho2 > (R)0 ? rsqrt_step(rho2) : (R)0;
    g.rho = rho2 * g.inv_rho;
    g.dphi = atan2_step(g.Y, g.X);
    if (g.X > (R)0) {
        // rho cos th_A - Z sin th_A = -sin s t_n + (rho - X) cos th_A and
        // rho sin th_A + Z cos th_A = cos s + (rho - X) sin th_A, rho - X small
        const R drho = div_step(g.Y * g.Y, g.rho + g.X);
        g.dth = atan2_step(-ss * tn + drho * cA, cs + drho * sA);
    } else {                  // across the polar axis: no small difference to keep
        g.dth = atan2_step(g.rho * cA - g.Z * sA, g.rho * sA + g.Z * cA);
    }
    g.cs = cs;
    return g;
}

// Q = [[p, q], [-q, p]] of A and the departure point g in A's turned frame:
// cos(phi_D - phi_A) = X / rho, sin(...) = Y / rho, cos th_D = Z, sin th_D = rho.
template <typename R>
__device__ __forceinline__ void rotation_pq(R sA, R cA, const Geo<R> &g, R *p, R *q) {
    R cx = 1, sx = 0;
    if (g.rho > (R)0) {
        cx = g.X * g.inv_rho;
        sx = g.Y * g.inv_rho;
    }
    const R inv_den = div_step((R)1, (R)1 + g.cs);      // 1 / (1 + cos eta)
    *p = (sA * g.rho + ((R)1 + cA * g.Z) * cx) * inv_den;
    *q = -(cA + g.Z) * sx * inv_den;
}

// Quintic Lagrange weights on the nodes -2..3 at t in [0, 1).
template <typename R>
__device__ __forceinline__ void lagrange5(R t, R *L) {
    const R a0 = t + 2, a1 = t + 1, a2 = t, a3 = t - 1, a4 = t - 2, a5 = t - 3;
    const R p01 = a0 * a1, p45 = a4 * a5;
    const R p012 = p01 * a2, p345 = a3 * p45;
    L[0] = -(a1 * a2 * p345) * (R)(1.0 / 120.0);
    L[1] = (a0 * a2 * p345) * (R)(1.0 / 24.0);
    L[2] = -(p01 * p345) * (R)(1.0 / 12.0);
    L[3] = (p012 * p45) * (R)(1.0 / 12.0);
    L[4] = -(p012 * a3 * a5) * (R)(1.0 / 24.0);
    L[5] = (p012 * a3 * a4) * (R)(1.0 / 120.0);
}

// One row of the quintic stencil: sum_b L[b] f(row, c0 + b) for both components,
// columns taken modulo n (c0 in [0, n)); the common case reads six consecutive
// columns.
template <typename R>
__device__ __forceinline__ void stencil_row(const R *__restrict__ ru, const R *__restrict__ rv,
                                            int c0, int n, const R *L, R &tu, R &tv) {
    tu = 0;
    tv = 0;
    if (c0 <= n - 6) {
#pragma unroll
        for (int b = 0; b < 6; ++b) {
            tu = fma(L[b], __ldg(ru + c0 + b), tu);
            tv = fma(L[b], __ldg(rv + c0 + b), tv);
        }
    } else {
#pragma unroll
        for (int b = 0; b < 6; ++b) {
            const int c = c0 + b < n ? c0 + b : c0 + b - n;
            tu = fma(L[b], __ldg(ru + c), tu);
            tv = fma(L[b], __ldg(rv + c), tv);
        }
    }
}

// grid ceil(members * P / 256); block 256.  w, wa: members x 2 x n_lat x n_lon
// (east, north); wa may be null; pq (optional): members x 2 x P, p then q of
// the final departure point.
template <typename R>
__global__ void __launch_bounds__(256) k_departure(DepArgs<R> a, const R *__restrict__ w,
                                                   const R *__restrict__ wa,
                                                   double *__restrict__ lon_d,
                                                   double *__restrict__ colat_d,
                                                   R *__restrict__ pq) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)a.members * a.P) return;
    const int m = (int)(gid / a.P);
    const int pi = (int)(gid - (long long)m * a.P);
    const int j = pi / a.n_lon, k = pi - j * a.n_lon;
    const int n = a.n_lon, nl = a.n_lat;
    const R *wu = w + (size_t)m * 2 * a.P;
    const R *wv = wu + a.P;
    R ae = 0, an = 0;
    if (wa) {
        ae = wa[(size_t)m * 2 * a.P + pi];
        an = wa[(size_t)m * 2 * a.P + a.P + pi];
    }
    // sin and cos of theta_A in R, from the row reflected into the northern
    // half so that the angle carries a relative rounding only
    const bool south = 2 * j > nl - 1;
    R sA, cA;
    sc(((R)(south ? nl - 1 - j : j) + (R)0.5) * a.h_th_r, &sA, &cA);
    if (south) cA = -cA;
    const R dta = a.dta, to_x = a.to_x, to_y = a.to_y;
    // D_0 = A: the bracket is the grid value and Q is the identity
    Geo<R> g = move_back(sA, cA, dta * (wu[pi] - ae), dta * (wv[pi] - an));
    for (int it = 1; it < a.iterations; ++it) {
        // position of D in grid-index units relative to A (clamped only to keep
        // the stencil inside the doubled grid; NaN falls to a bound)
        const R dx = fmin(fmax(g.dphi * to_x, (R)-n), (R)n);
        const R dy = fmin(fmax(g.dth * to_y, (R)(-nl - 2)), (R)(nl + 2));
        const R fx = floor(dx), fy = floor(dy);
        R Lx[6], Ly[6];
        lagrange5(dx - fx, Lx);
        lagrange5(dy - fy, Ly);
        int i0 = k + (int)fx;                          // in [-n, 2n)
        if (i0 < 0) i0 += n;
        else if (i0 >= n) i0 -= n;
        int r0 = j + (int)fy;
        r0 = r0 < -1 ? -1 : (r0 > nl - 1 ? nl - 1 : r0);
        R su = 0, sv = 0;
        const int ci = i0 >= 2 ? i0 - 2 : i0 - 2 + n;     // first stencil column
        if (r0 >= 2 && r0 + 3 < nl && ci <= n - 6) {
            // the common case: six rows of six consecutive columns, no pole, no seam
            const R *bu = wu + (size_t)(r0 - 2) * n + ci;
            const R *bv = wv + (size_t)(r0 - 2) * n + ci;
#pragma unroll
            for (int ra = 0; ra < 6; ++ra) {
                R tu = 0, tv = 0;
#pragma unroll
                for (int b = 0; b < 6; ++b) {
                    tu = fma(Lx[b], __ldg(bu + ra * n + b), tu);
                    tv = fma(Lx[b], __ldg(bv + ra * n + b), tv);
                }
                su = fma(Ly[ra], tu, su);
                sv = fma(Ly[ra], tv, sv);
            }
        } else {
#pragma unroll
            for (int ra = 0; ra < 6; ++ra) {
                const int r = r0 - 2 + ra;                 // in [-3, nl + 2]
                const bool beyond = r < 0 || r >= nl;
                const int rr = r < 0 ? -1 - r : (r >= nl ? 2 * nl - 1 - r : r);
                int c0 = i0 - 2 + (beyond ? n / 2 : 0);    // in [-2, 3n/2 - 2)
                if (c0 < 0) c0 += n;
                else if (c0 >= n) c0 -= n;
                R tu, tv;
                stencil_row(wu + (size_t)rr * n, wv + (size_t)rr * n, c0, n, Lx, tu, tv);
                const R wy = beyond ? -Ly[ra] : Ly[ra];
                su = fma(wy, tu, su);
                sv = fma(wy, tv, sv);
            }
        }
        R p, q;
        rotation_pq(sA, cA, g, &p, &q);
        const R ve = p * su + q * sv - ae;
        const R vn = -q * su + p * sv - an;
        g = move_back(sA, cA, dta * ve, dta * vn);
    }
    if (pq) {
        R p, q;
        rotation_pq(sA, cA, g, &p, &q);
        pq[(size_t)m * 2 * a.P + pi] = p;
        pq[(size_t)m * 2 * a.P + a.P + pi] = q;
    }
    double lon = (double)k * a.h_phi + (double)g.dphi;
    if (lon < 0.0) lon += 2.0 * kPi;
    else if (lon >= 2.0 * kPi) lon -= 2.0 * kPi;
    lon_d[gid] = lon;
    colat_d[gid] = ((double)j + 0.5) * a.h_th + (double)g.dth;
}

struct RotArgs {
    int n_lon, n_lat, members, P;
    long long stride;
    double h_phi, h_th;
};

// grid ceil(members * P / 256); block 256.  u_d, v_d may alias u_a, v_a.  With
// pq (members x 2 x P, from k_departure) Q is read; otherwise it is computed
// from the departure points.
template <typename R>
__global__ void __launch_bounds__(256) k_rotate(RotArgs a, const double *__restrict__ lon_d,
                                                const double *__restrict__ colat_d,
                                                const R *__restrict__ pq, const R *u_d,
                                                const R *v_d, R *u_a, R *v_a) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)a.members * a.P) return;
    const int m = (int)(gid / a.P);
    const int pi = (int)(gid - (long long)m * a.P);
    const size_t o = (size_t)m * a.stride + pi;
    if (pq) {
        const R p = pq[(size_t)m * 2 * a.P + pi], q = pq[(size_t)m * 2 * a.P + a.P + pi];
        const R u = u_d[o], v = v_d[o];
        u_a[o] = p * u + q * v;
        v_a[o] = -q * u + p * v;
        return;
    }
    const int j = pi / a.n_lon, k = pi - j * a.n_lon;
    double dl = (double)k * a.h_phi - lon_d[gid];            // phi_A - phi_D
    dl -= 2.0 * kPi * rint(dl * (0.5 / kPi));
    const double thA = ((double)j + 0.5) * a.h_th;
    R sA, cA, sD, cD, sl, cl;
    colat_sc(thA, &sA, &cA);
    colat_sc(colat_d[gid], &sD, &cD);
    sc((R)dl, &sl, &cl);
    const R den = (R)1 + sA * sD * cl + cA * cD;               // 1 + cos eta
    const R p = (sA * sD + ((R)1 + cA * cD) * cl) / den;
    const R q = (cA + cD) * sl / den;
    const R u = u_d[o], v = v_d[o];
    u_a[o] = p * u + q * v;
    v_a[o] = -q * u + p * v;
}

bool grid_ok(int n_lon, int n_lat, int members) {
    if (n_lon < 6 || (n_lon & 1) || n_lat < 3 || members < 1) return false;
    return (long long)n_lon * n_lat * members <= 0x7fffffffLL;
}


template <typename R>
cudaError_t launch_departure(int n_lon, int n_lat, int n_members, int iterations,
                             double dt_over_a, const void *w, const void *w_arrival,
                             double *lon_d, double *colat_d, void *pq, cudaStream_t st) {
    DepArgs<R> a;
    a.n_lon = n_lon;
    a.n_lat = n_lat;
    a.members = n_members;
    a.iterations = iterations;
    a.P = n_lon * n_lat;
    a.h_phi = 2.0 * kPi / n_lon;
    a.h_th = kPi / n_lat;
    a.dta = (R)dt_over_a;
    a.to_x = (R)(n_lon / (2.0 * kPi));
    a.to_y = (R)(n_lat / kPi);
    a.h_th_r = (R)(kPi / n_lat);
    const long long total = (long long)n_members * a.P;
    k_departure<R><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        a, (const R *)w, (const R *)w_arrival, lon_d, colat_d, (R *)pq);
    return cudaGetLastError();
}

}  // namespace

extern "C" int dfsnufft_departure_points(int n_lon, int n_lat, int n_members, int dtype,
                                         int iterations, double dt_over_a, const void *w,
                                         const void *w_arrival, double *lon_d, double *colat_d,
                                         void *pq, void *stream) {
    if (!grid_ok(n_lon, n_lat, n_members) || iterations < 1 || iterations > 64 || !w ||
        !lon_d || !colat_d || !(dt_over_a == dt_over_a) || dt_over_a > 1e300 ||
        dt_over_a < -1e300)
        return DFSNUFFT_ERR_INVALID_ARG;
    if (dtype != DFSNUFFT_F64 && dtype != DFSNUFFT_F32) return DFSNUFFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t e =
        dtype == DFSNUFFT_F64
            ? launch_departure<double>(n_lon, n_lat, n_members, iterations, dt_over_a, w,
                                       w_arrival, lon_d, colat_d, pq, st)
            : launch_departure<float>(n_lon, n_lat, n_members, iterations, dt_over_a, w,
                                      w_arrival, lon_d, colat_d, pq, st);
    return e == cudaSuccess ? DFSNUFFT_OK : DFSNUFFT_ERR_CUDA;
}

extern "C" int dfsnufft_rotate_to_arrival(int n_lon, int n_lat, int n_members, int dtype,
                                          const double *lon_d, const double *colat_d,
                                          const void *pq, const void *u_d, const void *v_d,
                                          int64_t stride, void *u_a, void *v_a, void *stream) {
    if (!grid_ok(n_lon, n_lat, n_members) || (!pq && (!lon_d || !colat_d)) || !u_d || !v_d ||
        !u_a || !v_a || stride < (int64_t)n_lon * n_lat)
        return DFSNUFFT_ERR_INVALID_ARG;
    if (dtype != DFSNUFFT_F64 && dtype != DFSNUFFT_F32) return DFSNUFFT_ERR_INVALID_ARG;
    RotArgs a;
    a.n_lon = n_lon;
    a.n_lat = n_lat;
    a.members = n_members;
    a.P = n_lon * n_lat;
    a.stride = stride;
    a.h_phi = 2.0 * kPi / n_lon;
    a.h_th = kPi / n_lat;
    const long long total = (long long)n_members * a.P;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == DFSNUFFT_F64)
        k_rotate<double><<<blocks, 256, 0, st>>>(a, lon_d, colat_d, (const double *)pq,
                                                 (const double *)u_d, (const double *)v_d,
                                                 (double *)u_a, (double *)v_a);
    else
        k_rotate<float><<<blocks, 256, 0, st>>>(a, lon_d, colat_d, (const float *)pq,
                                                (const float *)u_d, (const float *)v_d,
                                                (float *)u_a, (float *)v_a);
    return cudaGetLastError() == cudaSuccess ? DFSNUFFT_OK : DFSNUFFT_ERR_CUDA;
}

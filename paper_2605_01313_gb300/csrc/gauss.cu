// Fields sampled on a Gauss-Legendre latitude grid (DFSNUFFT_GAUSS_GRID): the
// coefficients of Eq. 5.3 from samples at the colatitudes theta_j = arccos(z_j)
// of the n_lat Gauss-Legendre nodes (Sec. 3) and phi_k = 2 pi k / n_lon, by the
// FFT in longitude and the inversion of the DFT matrix on the doubled column
// in latitude (Sec. 5, interpolation for the spherical-harmonic model).
//
// On the doubled column of mode m (rows theta_j and -theta_j) the data of a
// field of parity s satisfy g(-theta_j) = s (-1)^m g(theta_j), and the solve of
// the 2N x 2N system V c = g (V_{j,n} = e^{i n theta_j}, n = -N..N-1, N = n_lat)
// splits into two real N x N systems:
//   class 0, s (-1)^m = +1:  sum_{n<N} a_n cos(n theta_j) = g_j;
//            c_0 = a_0, c_{+-n} = a_n / 2, c_{-N} = 0;
//   class 1, s (-1)^m = -1:  sum_{n=1..N-1} b_n sin(n theta_j) + beta sin(N theta_j) = g_j;
//            c_{+-n} = -+ i b_n / 2, c_{-N} = i beta, and the Nyquist term's
//            even part a = -i beta w (w = C^{-1} cos(N theta)): c_0 += a_0,
//            c_{+-n} += a_n / 2.
// The inverse matrices C^{-1} (cos) and S^{-1} (sin) are formed once in FP64 on
// the host (Gauss-Jordan), scaled by 1 / n_lon (the FFT's normalisation) and
// applied to all modes of all fields as two real GEMMs: FP32 plans on the
// tensor cores by the library's own tcgen05 kernel (gl_gemm.cu, TF32 with a
// three-term split for FP32 accuracy), FP64 plans by cuBLAS DGEMM.  The
// column of mode -m is the solve of the conjugate data, (a, b, beta) ->
// conjugates.  For a real-field plan's staging only the Hermitian part
// matters (Re v): in the columns 0 < m < N1/2 the beta w terms cancel and are
// left out (of m < 0 only the Nyquist row is written); the columns m = 0 and
// N1/2 keep their values.
//
// Kernels: the longitude pass k_fwd_phi (GL form, forward.cu) writes the row
// spectra into the two classes; k_gl_coeffs maps the GEMM results to the
// centred coefficient layout of dfsnufft_execute.
#include <cublas_v2.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"

cudaError_t dfs_launch_fwd_phi_gl(dfsnufft_plan p, const void *samples, const int *d_parity,
                                  void *g0, void *g1, int K, long long pitch);

namespace {

constexpr double kPi = 3.14159265358979323846;

// Colatitudes of the N Gauss-Legendre nodes, increasing: Newton's method on
// P_N(cos theta) in theta itself (dP/dtheta = N (x P_N - P_{N-1}) / sin theta),
// from theta = pi (j + 3/4) / (N + 1/2), so that nodes near a pole keep their
// relative accuracy.
void gauss_legendre_colat(int N, double *theta) {
    for (int j = 0; j < N; ++j) {
        double th = kPi * (j + 0.75) / (N + 0.5);
        for (int it = 0; it < 20; ++it) {
            const double x = cos(th), s = sin(th);
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= N; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pN = N == 1 ? x : p1, pNm1 = N == 1 ? 1.0 : p0;
            const double d = N * (x * pN - pNm1) / s;
            const double step = pN / d;
            th -= step;
            if (fabs(step) <= 1e-16 * (1.0 + th)) break;
        }
        theta[j] = th;
    }
}

// Inverse of the n x n row-major matrix a (overwritten) by Gauss-Jordan
// elimination with partial pivoting on [a | I].  False if a pivot vanishes or
// memory runs out.
bool invert(double *a, int n) {
    const size_t w = 2 * (size_t)n;
    double *m = (double *)malloc(sizeof(double) * w * n);
    if (!m) return false;
    for (int r = 0; r < n; ++r) {
        memcpy(m + r * w, a + (size_t)r * n, sizeof(double) * n);
        memset(m + r * w + n, 0, sizeof(double) * n);
        m[r * w + n + r] = 1.0;
    }
    bool ok = true;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(m[r * w + c]) > fabs(m[piv * w + c])) piv = r;
        if (m[piv * w + c] == 0.0) {
            ok = false;
            break;
        }
        if (piv != c)
            for (size_t k = c; k < w; ++k) {
                const double t = m[c * w + k];
                m[c * w + k] = m[piv * w + k];
                m[piv * w + k] = t;
            }
        double *rc = m + c * w;
        const double inv = 1.0 / rc[c];
        for (size_t k = c; k < w; ++k) rc[k] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double *rr = m + r * w;
            const double f = rr[c];
            if (f == 0.0) continue;
            for (size_t k = c; k < w; ++k) rr[k] -= f * rc[k];
        }
    }
    if (ok)
        for (int r = 0; r < n; ++r) memcpy(a + (size_t)r * n, m + r * w + n, sizeof(double) * n);
    free(m);
    return ok;
}

template <typename R> void convert(const double *src, R *dst, size_t n, double scale) {
    for (size_t i = 0; i < n; ++i) dst[i] = (R)(src[i] * scale);
}

}  // namespace

namespace {

struct GlArgs {
    int N, N1, F, K;          // N = n_lat; K complex slots per line and class
    long long pitch;          // complex per row of a class matrix (lines K)
    int full;                 // 0: real-field staging (Hermitian part, see above)
};

// Coefficients c_{n,m} and c_{n,-m} of one centred row n (an = |n|) and one
// mode m of a line, from the class results: v0 = out0[an] (class 0, an < N),
// v1 = out1[an - 1] (class 1, an >= 1) and beta = out1[N - 1] of the line's
// slot of m; wn the Nyquist weight of row an.
template <typename C, typename R>
__device__ __forceinline__ void gl_coef(const GlArgs &a, bool cls0, int n, int m, C v0, C v1,
                                        C beta, R wn, C &cm, C &cneg) {
    const int N = a.N;
    const int an = n < 0 ? -n : n;
    if (cls0) {
        // c_0 = a_0, c_{+-n} = a_n / 2, c_{-N} = 0; mode -m: conjugate data
        C v = cmake((R)0, (R)0);
        if (an < N) v = an ? cmake(v0.x * (R)0.5, v0.y * (R)0.5) : v0;
        cm = v;
        cneg = cmake(v.x, -v.y);
    } else if (an == N) {                             // c_{-N} = i beta
        cm = cmake(-beta.y, beta.x);
        cneg = cmake(beta.y, beta.x);                 // i conj(beta)
    } else {
        // -+ i b_n / 2 (zero at n = 0), then - i beta w_n (/ 2 off n = 0)
        C bi = cmake((R)0, (R)0);
        cneg = cmake((R)0, (R)0);
        if (an) {
            const R sg = n > 0 ? (R)0.5 : (R)-0.5;
            bi = cmake(v1.y * sg, -v1.x * sg);        // -i b sg
            cneg = cmake(-v1.y * sg, -v1.x * sg);     // -i conj(b) sg
        }
        cm = bi;
        // literal values for full output and in the columns m = 0 and N1/2,
        // which a real-field plan evaluates as they are (its own mirror, the
        // Nyquist column)
        if (a.full || m == 0 || m == a.N1 / 2) {
            cm = cmake(cm.x + beta.y * wn, cm.y - beta.x * wn);          // - i beta wn
            cneg = cmake(cneg.x - beta.y * wn, cneg.y - beta.x * wn);    // - i conj(beta) wn
        }
    }
}

template <typename C> __device__ __forceinline__ void store_pair(C *p, C x, C y, bool vec) {
    if constexpr (sizeof(C) == 8) {
        if (vec) {
            *reinterpret_cast<float4 *>(p) = make_float4(x.x, x.y, y.x, y.y);
            return;
        }
    }
    p[0] = x;
    p[1] = y;
}

// grid (ceil((N1/4 + 1) / 128), N + 1, lines); block 128 threads over the
// mode pairs q (modes m = 2q, 2q + 1 <= N1/2, one slot of both classes), blockIdx.y
// the row pair an (rows n = +an <= N - 1 and n = -an >= -N).  Each class value
// is read once for both rows; the two modes of a row go out as one 16-byte
// store when vec (FP32, 16-byte aligned coefficients).  out0/out1: the GEMM
// results of the two classes, N x pitch complex; w: N reals.
template <typename R>
__global__ void __launch_bounds__(128) k_gl_coeffs(GlArgs a, const typename CxT<R>::type *out0,
                                                   const typename CxT<R>::type *out1,
                                                   const R *__restrict__ w,
                                                   const int *__restrict__ parity,
                                                   typename CxT<R>::type *__restrict__ coef,
                                                   int vec) {
    dfs_grid_wait();
    typedef typename CxT<R>::type C;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int h1 = a.N1 / 2;
    if (2 * q > h1) return;
    const int an = blockIdx.y;
    const int l = blockIdx.z;
    const int N = a.N;
    const int pneg = parity[l % a.F] < 0;
    const size_t slot = (size_t)l * a.K + q;
    const C zero = cmake((R)0, (R)0);
    const C v0 = an < N ? out0[(size_t)an * a.pitch + slot] : zero;
    const C v1 = an >= 1 && an <= N ? out1[(size_t)(an - 1) * a.pitch + slot] : zero;
    const C beta = out1[(size_t)(N - 1) * a.pitch + slot];
    const R wn = an < N ? (an ? (R)0.5 * w[an] : w[0]) : (R)0;
    const int m0 = 2 * q;
    const bool two = m0 + 1 <= h1;                    // mode 2q + 1 exists
    for (int sgn = 0; sgn < 2; ++sgn) {
        const int n = sgn ? -an : an;
        if (sgn && an == 0) break;                    // n = 0 once
        if (!sgn && an == N) continue;                // n = +N is not a row
        C *col = coef + (size_t)l * 2 * N * a.N1 + (size_t)(n + N) * a.N1;
        C cm[2], cn[2];
        for (int k = 0; k < 2; ++k) {
            const int m = m0 + k;
            if (k == 1 && !two) break;
            gl_coef<C, R>(a, pneg == (m & 1), n, m, v0, v1, beta, wn, cm[k], cn[k]);
        }
        if (two && m0 + 1 < h1) {
            // modes m0, m0 + 1 < N1/2: centred columns m + N1/2, adjacent
            store_pair(col + m0 + h1, cm[0], cm[1], vec != 0);
        } else {
            col[m0 < h1 ? m0 + h1 : 0] = cm[0];
            if (two) col[m0 + 1 < h1 ? m0 + 1 + h1 : 0] = cm[1];
        }
        if (a.full || an == N) {                      // the mirrors of 0 < m < N1/2
            for (int k = 0; k < 2; ++k) {
                const int m = m0 + k;
                if (k == 1 && !two) break;
                if (m > 0 && m < h1) col[h1 - m] = cn[k];
            }
        }
    }
}

}  // namespace

// Host set-up of a Gauss-Legendre plan: nodes, inverse matrices (scaled by
// 1 / n_lon), w, the BLAS handle.  Called by plan creation.
int dfs_gl_setup(dfsnufft_plan p) {
    const dfsnufft_params &q = p->prm;
    const int N = q.n_lat;
    const bool f64 = q.dtype == DFSNUFFT_F64;
    const size_t rs = f64 ? sizeof(double) : sizeof(float);
    double *th = (double *)malloc(sizeof(double) * N);
    double *cm = (double *)malloc(sizeof(double) * (size_t)N * N);
    double *sm = (double *)malloc(sizeof(double) * (size_t)N * N);
    double *wv = (double *)malloc(sizeof(double) * N);
    void *hbuf = malloc(rs * ((size_t)2 * N * N + N));
    int rc = DFSNUFFT_OK;
    if (!th || !cm || !sm || !wv || !hbuf) rc = DFSNUFFT_ERR_OOM;
    if (rc == DFSNUFFT_OK) {
        gauss_legendre_colat(N, th);
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                cm[(size_t)j * N + k] = cos(k * th[j]);
                sm[(size_t)j * N + k] = sin((k + 1) * th[j]);
            }
        if (!invert(cm, N) || !invert(sm, N)) rc = DFSNUFFT_ERR_UNSUPPORTED;
    }
    if (rc == DFSNUFFT_OK) {
        for (int k = 0; k < N; ++k) {
            double acc = 0.0;
            for (int j = 0; j < N; ++j) acc += cm[(size_t)k * N + j] * cos(N * th[j]);
            wv[k] = acc;
        }
        const double sc = 1.0 / q.N1;
        const size_t nn = (size_t)N * N;
        if (!f64) {
            // the tensor-core solve's split matrices, from the scaled FP64 inverses
            for (size_t i = 0; i < nn; ++i) {
                cm[i] *= sc;
                sm[i] *= sc;
            }
            rc = dfs_gl_tc_setup(p, cm, sm, N);
            for (size_t i = 0; i < nn; ++i) {
                cm[i] /= sc;
                sm[i] /= sc;
            }
        }
        if (f64) {
            convert(cm, (double *)hbuf, nn, sc);
            convert(sm, (double *)hbuf + nn, nn, sc);
            convert(wv, (double *)hbuf + 2 * nn, N, 1.0);
        } else {
            convert(cm, (float *)hbuf, nn, sc);
            convert(sm, (float *)hbuf + nn, nn, sc);
            convert(wv, (float *)hbuf + 2 * nn, N, 1.0);
        }
        if (cudaMalloc(&p->d_gl_mat, rs * (2 * nn + N)) != cudaSuccess) {
            p->d_gl_mat = nullptr;
            rc = DFSNUFFT_ERR_OOM;
        }
        if (rc == DFSNUFFT_OK) {
            const cudaError_t e =
                cudaMemcpy(p->d_gl_mat, hbuf, rs * (2 * nn + N), cudaMemcpyHostToDevice);
            if (e) rc = DFSNUFFT_ERR_CUDA;
        }
    }
    if (rc == DFSNUFFT_OK) {
        p->h_gl_colat = th;
        th = nullptr;
        if (f64) {
            cublasHandle_t h = nullptr;
            if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) rc = DFSNUFFT_ERR_CUDA;
            else p->blas = h;
        }
    }
    free(th);
    free(cm);
    free(sm);
    free(wv);
    free(hbuf);
    return rc;
}

void dfs_gl_release(dfsnufft_plan p) {
    if (p->blas) cublasDestroy((cublasHandle_t)p->blas);
    p->blas = nullptr;
    free(p->h_gl_colat);
    p->h_gl_colat = nullptr;
    if (p->d_gl_mat) cudaFree(p->d_gl_mat);
    p->d_gl_mat = nullptr;
    if (p->d_gl_tc) cudaFree(p->d_gl_tc);
    p->d_gl_tc = nullptr;
}

// Samples on the Gauss-Legendre grid to coefficients (the layout of
// dfsnufft_execute); full = false writes the real-field staging described above.
int dfs_launch_forward_gl(dfsnufft_plan p, const void *samples, const int *d_parity,
                          void *coeffs, bool full) {
    const dfsnufft_params &q = p->prm;
    const int N = q.n_lat, lines = p->n_members * p->n_fields;
    const int K = q.N1 / 4 + 1;
    // complex per class row, rounded up so that every GEMM column starts on 32
    // bytes (the tensor-core GEMMs need 16-byte aligned leading dimensions)
    const long long pitch = ((long long)lines * K + 3) / 4 * 4;
    const long long cols = 2 * pitch;                        // reals
    const bool f64 = q.dtype == DFSNUFFT_F64;
    const size_t rs = f64 ? sizeof(double) : sizeof(float);
    // four N x cols blocks in the theta-pass buffer: class inputs, class results
    char *base = (char *)p->d_T;
    void *g0 = base, *g1 = base + rs * N * cols;
    void *o0 = base + 2 * rs * N * cols;
    cudaError_t e = dfs_launch_fwd_phi_gl(p, samples, d_parity, g0, g1, K, pitch);
    if (!e && pitch > (long long)lines * K) {            // zero the padding columns
        const size_t cs = 2 * rs, used = cs * lines * K;
        e = cudaMemset2DAsync((char *)g0 + used, cs * pitch, 0, cs * pitch - used, 2 * N,
                              p->stream);
    }
    if (e) return DFSNUFFT_ERR_CUDA;
    if (f64) {
        cublasHandle_t h = (cublasHandle_t)p->blas;
        if (cublasSetStream(h, p->stream) != CUBLAS_STATUS_SUCCESS) return DFSNUFFT_ERR_CUDA;
        // out_c (col-major cols x N) = g_c (cols x N) * M_c^T, M_c row-major N x N
        const long long sA = (long long)N * cols, sB = (long long)N * N, sC = sA;
        const double one = 1.0, zero = 0.0;
        if (cublasDgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)cols, N, N, &one,
                                      (const double *)g0, (int)cols, sA,
                                      (const double *)p->d_gl_mat, N, sB, &zero, (double *)o0,
                                      (int)cols, sC, 2) != CUBLAS_STATUS_SUCCESS)
            return DFSNUFFT_ERR_CUDA;
    } else if (dfs_gl_tc_gemm(p, (const float *)g0, (float *)o0, N, (int)cols)) {
        return DFSNUFFT_ERR_CUDA;
    }
    GlArgs a;
    a.N = N;
    a.N1 = q.N1;
    a.F = p->n_fields;
    a.K = K;
    a.pitch = pitch;
    a.full = full ? 1 : 0;
    const dim3 grid((q.N1 / 4 + 1 + 127) / 128, N + 1, lines);
    // 16-byte stores of mode pairs: rows of N1 complex from a 16-byte aligned
    // base, pairs starting at the even centred column m + N1/2
    const int vec = ((uintptr_t)coeffs & 15) == 0 && (q.N1 / 2) % 2 == 0;
    if (f64) {
        typedef double2 C;
        const C *r0 = (const C *)o0;
        e = dfs_launch_dependent(k_gl_coeffs<double>, grid, dim3(128), 0, p->stream, a, r0,
                                 r0 + (size_t)N * pitch,
                                 (const double *)p->d_gl_mat + 2 * (size_t)N * N,
                                 (const int *)d_parity, (C *)coeffs, vec);
    } else {
        typedef float2 C;
        const C *r0 = (const C *)o0;
        e = dfs_launch_dependent(k_gl_coeffs<float>, grid, dim3(128), 0, p->stream, a, r0,
                                 r0 + (size_t)N * pitch,
                                 (const float *)p->d_gl_mat + 2 * (size_t)N * N,
                                 (const int *)d_parity, (C *)coeffs, vec);
    }
    return e ? DFSNUFFT_ERR_CUDA : DFSNUFFT_OK;
}

// Bytes of the theta-pass buffer the Gauss-Legendre form needs.
size_t dfs_gl_scratch_bytes(const dfsnufft_params &q, int lines) {
    const size_t rs = q.dtype == DFSNUFFT_F64 ? sizeof(double) : sizeof(float);
    const size_t pitch = ((size_t)lines * (q.N1 / 4 + 1) + 3) / 4 * 4;
    return 4 * rs * (size_t)q.n_lat * 2 * pitch;
}

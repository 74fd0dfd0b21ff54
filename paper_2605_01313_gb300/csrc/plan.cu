// Host runtime and C ABI of dfsnufft: plan parameters, deconvolution factors,
// device memory, and the entry points declared in include/dfsnufft.h.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "common.cuh"
#include "fft_core.cuh"

#define DFS_VERSION "dfsnufft 0.1 (sm_103a)"

static const double kPi = 3.14159265358979323846264338327950288;

// ------------------------------------------------------------------ helpers

static int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

static void set_msg(dfsnufft_plan p, const char *what, cudaError_t e) {
    snprintf(p->msg, sizeof(p->msg), "%s: %s (%s)", what, cudaGetErrorName(e),
             cudaGetErrorString(e));
}

// Record a CUDA failure on the plan (sticky) and return the ABI status.
static int fail_cuda(dfsnufft_plan p, const char *what, cudaError_t e) {
    p->status = DFSNUFFT_ERR_CUDA;
    set_msg(p, what, e);
    return DFSNUFFT_ERR_CUDA;
}

#define DFS_CK(p, call)                                                   \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return fail_cuda((p), #call, e_);          \
    } while (0)

static int dfs_alloc(dfsnufft_plan p, void **ptr, size_t bytes, const char *what) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        snprintf(p->msg, sizeof(p->msg), "out of device memory allocating %s (%zu bytes)", what,
                 bytes);
        *ptr = nullptr;
        return DFSNUFFT_ERR_OOM;
    }
    if (e != cudaSuccess) return fail_cuda(p, what, e);
    return DFSNUFFT_OK;
}

static void dfs_free(void **ptr) {
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
}

// ------------------------------------------------------------------ stage timing

static cudaEvent_t *stage_event(dfsnufft_plan p, int stage, int slot, int which) {
    return &p->ev[((size_t)stage * DFS_TIMING_SLOTS + slot) * 2 + which];
}

static cudaError_t timing_drain(dfsnufft_plan p) {
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e) return e;
    for (int s = 0; s < DFSNUFFT_N_STAGES; ++s) {
        for (int i = 0; i < p->pending[s]; ++i) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, *stage_event(p, s, i, 0), *stage_event(p, s, i, 1));
            if (e) return e;
            p->ms_total[s] += ms;
            p->calls[s] += 1;
        }
        p->pending[s] = 0;
    }
    return cudaSuccess;
}

static cudaError_t timing_begin(dfsnufft_plan p, int stage) {
    if (!p->timing) return cudaSuccess;
    if (p->pending[stage] == DFS_TIMING_SLOTS) {
        cudaError_t e = timing_drain(p);
        if (e) return e;
    }
    return cudaEventRecord(*stage_event(p, stage, p->pending[stage], 0), p->stream);
}

static cudaError_t timing_end(dfsnufft_plan p, int stage) {
    if (!p->timing) return cudaSuccess;
    cudaError_t e = cudaEventRecord(*stage_event(p, stage, p->pending[stage], 1), p->stream);
    p->pending[stage] += 1;
    return e;
}

// ------------------------------------------------------------------ kernel math (host)

extern "C" double dfsnufft_es_kernel(double z, int w, double beta) {
    double u = 2.0 * z / (double)w;
    if (!(fabs(u) < 1.0)) return 0.0;
    return exp(beta * (sqrt((1.0 - u) * (1.0 + u)) - 1.0));
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_q, using the
// three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and
// P_q'(x) = q (x P_q - P_{q-1}) / (x^2 - 1).  legendre_pair gives P_q, P_{q-1}.
static void legendre_pair(int q, double z, double *pq, double *pq1) {
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < q; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pq = p1;
    *pq1 = p0;
}

static void gauss_legendre(int q, double *x, double *wt) {
    for (int i = 0; i < q; ++i) {
        double z = cos(kPi * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pq, pq1;
            legendre_pair(q, z, &pq, &pq1);
            double dz = pq / (q * (z * pq - pq1) / (z * z - 1.0));
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double pq, pq1;
        legendre_pair(q, z, &pq, &pq1);
        double dp = q * (z * pq - pq1) / (z * z - 1.0);
        x[i] = z;
        wt[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

extern "C" int dfsnufft_kernel_ft(int w, double beta, int n_fine, int n_modes, double *out) {
    if (w < 2 || w > 16 || !(beta > 0) || n_fine < 2 || n_modes < 1 || !out)
        return DFSNUFFT_ERR_INVALID_ARG;
    // phihat(xi) = int_{-w/2}^{w/2} phi(z) cos(xi z) dz
    //            = w int_0^1 e^{beta (sqrt(1-u^2) - 1)} cos(xi w u / 2) du
    //            = w int_0^{pi/2} e^{beta (cos s - 1)} cos(xi (w/2) sin s) cos s ds   (u = sin s)
    // The substitution removes the square-root endpoint singularity, so the
    // Gauss-Legendre rule converges exponentially.
    // (no allocation: the allocation-free entry point calls this too)
    const int q = 2 * w + 60;                          // <= 92 nodes
    double x[92], wt[92], fz[92], zz[92];
    gauss_legendre(q, x, wt);
    for (int i = 0; i < q; ++i) {
        double sv = 0.25 * kPi * (x[i] + 1.0);  // node mapped to [0, pi/2]
        zz[i] = 0.5 * w * sin(sv);              // z in fine cells
        fz[i] = 0.25 * kPi * wt[i] * exp(beta * (cos(sv) - 1.0)) * cos(sv);
    }
    for (int qi = 0; qi < n_modes; ++qi) {
        double k = (double)(qi - n_modes / 2);
        double xi = 2.0 * kPi * k / (double)n_fine;
        double acc = 0.0;
        for (int i = 0; i < q; ++i) acc += fz[i] * cos(xi * zz[i]);
        out[qi] = w * acc;
    }
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_es_horner(int w, double beta, double *out) {
    if (w < 2 || w > 16 || !(beta > 0) || !out) return DFSNUFFT_ERR_INVALID_ARG;
    const int D = w;                                   // degree
    const int c0 = (w % 2 == 0) ? w / 2 - 1 : (w - 1) / 2;
    const double mid = (w % 2 == 0) ? 0.5 : 0.0;
    double f[17], cheb[17], mono[17], tk[17], tk1[17], tk2[17];
    for (int a = 0; a < w; ++a) {
        // Chebyshev interpolation in x = 2 s on [-1, 1]
        for (int j = 0; j <= D; ++j) {
            const double x = cos(kPi * (j + 0.5) / (D + 1));
            f[j] = dfsnufft_es_kernel((double)(a - c0) - (mid + 0.5 * x), w, beta);
        }
        for (int k = 0; k <= D; ++k) {
            double acc = 0.0;
            for (int j = 0; j <= D; ++j) acc += f[j] * cos(kPi * k * (j + 0.5) / (D + 1));
            cheb[k] = acc * 2.0 / (D + 1);
        }
        cheb[0] *= 0.5;
        // monomials in x via T_{k+1} = 2 x T_k - T_{k-1}
        for (int k = 0; k <= D; ++k) mono[k] = tk[k] = tk1[k] = tk2[k] = 0.0;
        tk2[0] = 1.0;                                  // T_0
        tk1[1] = 1.0;                                  // T_1
        mono[0] += cheb[0];
        if (D >= 1) mono[1] += cheb[1];
        for (int k = 2; k <= D; ++k) {
            for (int i = 0; i <= D; ++i) tk[i] = (i > 0 ? 2.0 * tk1[i - 1] : 0.0) - tk2[i];
            for (int i = 0; i <= D; ++i) {
                mono[i] += cheb[k] * tk[i];
                tk2[i] = tk1[i];
                tk1[i] = tk[i];
            }
        }
        // x = 2 s: coefficient of s^k is 2^k times that of x^k
        double sc = 1.0;
        for (int k = 0; k <= D; ++k) {
            out[a * (D + 1) + k] = mono[k] * sc;
            sc *= 2.0;
        }
    }
    return DFSNUFFT_OK;
}

// Kernel width rule for sigma = 4.  Modelled worst error of the 1-D kernel
// interpolation of e^{i omega x} over |omega| <= pi / sigma (the band the
// deconvolution inverts), with beta as the plan uses it, for w = 0..16:
// entry w of kErr2 (sigma 2, beta = 2.30 w) and of kErr4 (sigma 4,
// beta = 0.97 pi (1 - 1/8) w).  A sigma-4 plan takes the narrowest w whose
// modelled error is at most that of the sigma-2 width for the same tol.  The
// values come from direct evaluation of the model (kernel samples against
// phihat by adaptive quadrature) on 801 offsets at 4 frequencies.
static const double kErr2[17] = {1, 1, 1.55e-01, 2.66e-02, 3.73e-03, 3.76e-04, 3.11e-05,
                                 2.49e-06, 3.89e-07, 4.51e-08, 7.29e-09, 8.40e-10, 7.82e-11,
                                 6.94e-12, 5.87e-13, 1.05e-13, 2.97e-14};
static const double kErr4[17] = {1, 1, 7.69e-02, 6.65e-03, 4.51e-04, 1.98e-05, 1.29e-06,
                                 1.36e-07, 1.33e-08, 7.95e-10, 3.32e-11, 3.55e-12, 2.97e-13,
                                 2.56e-14, 4.56e-15, 4.79e-15, 4.71e-15};

static bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

extern "C" int dfsnufft_choose_params_opts(int n_lon, int n_lat, double tol, int dtype,
                                           const dfsnufft_options *opts, dfsnufft_params *out) {
    if (!out) return DFSNUFFT_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    dfsnufft_options o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (n_lon < 4 || (n_lon & 1) || n_lat < 2) return DFSNUFFT_ERR_INVALID_ARG;
    if (dtype != DFSNUFFT_F64 && dtype != DFSNUFFT_F32) return DFSNUFFT_ERR_INVALID_ARG;
    if (!(tol > 0.0) || !(tol < 1.0)) return DFSNUFFT_ERR_INVALID_ARG;
    if ((o.flags & ~(DFSNUFFT_REAL_FIELDS | DFSNUFFT_KEEP_ORDER | DFSNUFFT_GAUSS_GRID)) != 0)
        return DFSNUFFT_ERR_INVALID_ARG;
    const int sigma = o.sigma == 0 ? 2 : o.sigma;
    if (sigma != 2 && sigma != 4) return DFSNUFFT_ERR_INVALID_ARG;
    if (o.w != 0 && (o.w < 2 || o.w > 16)) return DFSNUFFT_ERR_INVALID_ARG;
    if ((o.tile_x != 0 && !pow2_in(o.tile_x, 8, 128)) ||
        (o.tile_y != 0 && !pow2_in(o.tile_y, 8, 128)))
        return DFSNUFFT_ERR_INVALID_ARG;
    if (dtype == DFSNUFFT_F64 && tol < 1e-14) return DFSNUFFT_ERR_TOL_UNATTAINABLE;
    if (dtype == DFSNUFFT_F32 && tol < 1e-7) return DFSNUFFT_ERR_TOL_UNATTAINABLE;
    // sigma 2, beta = 2.30 w: the narrowest w whose modelled 1-D error kErr2[w]
    // is at most 2.5 tol (FP64) or 5 tol (FP32).  A lone mode at the corner of
    // the band carries the 1-D band-edge error in both dimensions, about
    // 2 kErr2[w], which this keeps at half of the accepted relative error
    // (10 tol in FP64, 20 tol in FP32).  w = 14 at tol 1e-12 (13 would leave
    // such a mode at about 1.4e-11), 7 at tol 1e-6.
    const double wfac = dtype == DFSNUFFT_F64 ? 2.5 : 5.0;
    int w = 2;
    while (w < 16 && kErr2[w] > wfac * tol) ++w;
    double beta = 2.30 * w;
    if (sigma == 4) {
        int w4 = 2;
        while (w4 < 16 && kErr4[w4] > kErr2[w]) ++w4;
        w = w4;
    }
    if (o.w != 0) w = o.w;
    if (sigma == 4) beta = 0.97 * 3.14159265358979323846 * (1.0 - 1.0 / (2.0 * sigma)) * w;
    else beta = 2.30 * w;
    out->n_lon = n_lon;
    out->n_lat = n_lat;
    out->N1 = n_lon;
    out->N2 = 2 * n_lat;
    const int a1 = sigma * out->N1 > 2 * w ? sigma * out->N1 : 2 * w;
    const int a2 = sigma * out->N2 > 2 * w ? sigma * out->N2 : 2 * w;
    out->n1 = next_pow2(a1 > 16 ? a1 : 16);
    out->n2 = next_pow2(a2 > 16 ? a2 : 16);
    if (out->n1 > (1 << DFS_FFT_MAX_LOG) || out->n2 > (1 << DFS_FFT_MAX_LOG))
        return DFSNUFFT_ERR_UNSUPPORTED;
    out->w = w;
    out->beta = beta;
    out->tol = tol;
    out->dtype = dtype;
    out->sigma = sigma;
    out->flags = o.flags;
    // default bins: the autotuner's choice on the 2048 x 1024 workload in
    // each precision (FP64: wide bins amortise the larger halo of w = 13)
    out->tile_x = o.tile_x ? o.tile_x : (dtype == DFSNUFFT_F32 ? 32 : 128);
    out->tile_y = o.tile_y ? o.tile_y : 16;
    if (out->tile_x > out->n1) out->tile_x = out->n1;
    if (out->tile_y > out->n2) out->tile_y = out->n2;
    // at most DFS_MAX_ROW_BLOCKS bin rows
    while (out->n2 / out->tile_y > DFS_MAX_ROW_BLOCKS) out->tile_y *= 2;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_choose_params(int n_lon, int n_lat, double tol, int dtype,
                                      dfsnufft_params *out) {
    return dfsnufft_choose_params_opts(n_lon, n_lat, tol, dtype, nullptr, out);
}

extern "C" const char *dfsnufft_strerror(int status) {
    switch (status) {
        case DFSNUFFT_OK: return "ok";
        case DFSNUFFT_ERR_INVALID_ARG: return "invalid argument";
        case DFSNUFFT_ERR_TOL_UNATTAINABLE: return "tolerance unattainable in this precision";
        case DFSNUFFT_ERR_NO_POINTS: return "execute called before set_points";
        case DFSNUFFT_ERR_OOM: return "out of device memory";
        case DFSNUFFT_ERR_CUDA: return "CUDA error";
        case DFSNUFFT_ERR_UNSUPPORTED: return "size outside the supported range";
        case DFSNUFFT_ERR_TIMEOUT: return "a kernel timed out waiting on an asynchronous copy";
        default: return "unknown status";
    }
}

extern "C" const char *dfsnufft_version(void) { return DFS_VERSION; }

// ------------------------------------------------------------------ plan lifetime

static void release(dfsnufft_plan p) {
    dfs_gl_release(p);
    void **bufs[] = {&p->d_inv1, &p->d_inv2, &p->d_tw1, &p->d_tw2, &p->d_stw_theta, &p->d_stw_phi,
                     &p->d_T, &p->d_G, (void **)&p->d_bin_count, (void **)&p->d_bin_start,
                     (void **)&p->d_task_bin, (void **)&p->d_n_tasks,
                     (void **)&p->d_status, (void **)&p->d_parity, (void **)&p->d_rowrange,
                     (void **)&p->d_pofs, (void **)&p->d_work,
                     &p->d_urec, (void **)&p->d_base, &p->d_frac, (void **)&p->d_idx,
                     (void **)&p->d_pts_stage, &p->d_coef_stage, &p->d_val_stage,
                     &p->d_df_tw1, &p->d_df_tw2, &p->d_df_inv1, &p->d_df_inv2,
                     &p->d_df_stw_phi, &p->d_df_stw_theta, &p->d_df_stw_half,
                     (void **)&p->d_emax};
    for (size_t i = 0; i < sizeof(bufs) / sizeof(bufs[0]); ++i) dfs_free(bufs[i]);
    free(p->h_pofs);
    p->h_pofs = nullptr;
    if (p->ev) {
        for (int i = 0; i < 2 * DFS_TIMING_SLOTS * DFSNUFFT_N_STAGES; ++i)
            if (p->ev[i]) cudaEventDestroy(p->ev[i]);
        free(p->ev);
        p->ev = nullptr;
    }
    if (p->copy_stream) {
        cudaStreamSynchronize(p->copy_stream);
        cudaStreamDestroy(p->copy_stream);
        p->copy_stream = nullptr;
    }
    if (p->back_stream) {
        cudaStreamSynchronize(p->back_stream);
        cudaStreamDestroy(p->back_stream);
        p->back_stream = nullptr;
    }
    if (p->stage_free) cudaEventDestroy(p->stage_free);
    if (p->coef_ready) cudaEventDestroy(p->coef_ready);
    p->stage_free = p->coef_ready = nullptr;
    for (int i = 0; i < p->n_line_ev; ++i)
        if (p->line_ev[i]) cudaEventDestroy(p->line_ev[i]);
    free(p->line_ev);
    p->line_ev = nullptr;
    p->n_line_ev = 0;
    if (p->pts_copied) cudaEventDestroy(p->pts_copied);
    if (p->vals_copied) cudaEventDestroy(p->vals_copied);
    p->pts_copied = p->vals_copied = nullptr;
}

template <typename C, typename R>
static void fill_twiddles(C *h, int n) {
    for (int k = 0; k < n; ++k) {
        double a = 2.0 * kPi * (double)k / (double)n;
        h[k].x = (R)cos(a);
        h[k].y = (R)sin(a);
    }
}

// Stage-ordered twiddles of a length-2^logn transform with e elements per
// thread (layout of dfs_fft::line_fft_ct): per stage after the first, entry
// (r - 1) Ns + jm = e^{+2 pi i r jm / (Ns R)}.
template <typename C, typename R>
static void fill_stage_twiddles(C *h, int logn, int e) {
    const int le = e == 16 ? 4 : e == 8 ? 3 : 2;
    int l = 0, off = 0;
    while (l < logn) {
        const int lr = logn - l < le ? logn - l : le;
        if (l > 0) {
            const int ns = 1 << l, radix = 1 << lr;
            for (int r = 1; r < radix; ++r)
                for (int jm = 0; jm < ns; ++jm) {
                    const double a = 2.0 * kPi * (double)(r * jm) / (double)(ns * radix);
                    h[off + (r - 1) * ns + jm].x = (R)cos(a);
                    h[off + (r - 1) * ns + jm].y = (R)sin(a);
                }
            off += (radix - 1) << l;
        }
        l += lr;
    }
}

static int stage_table_len(int n) {
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    const int sz = dfs_fft::stage_table_size(logn, DFS_FFT_E);
    return sz > 0 ? sz : 1;
}

static int upload_stage_tables(dfsnufft_plan p) {
    const dfsnufft_params &q = p->prm;
    const size_t cs = q.dtype == DFSNUFFT_F64 ? sizeof(double2) : sizeof(float2);
    const int lens[2] = {q.n2 / 2, q.n1 / 2};
    void *dst[2] = {p->d_stw_theta, p->d_stw_phi};
    for (int k = 0; k < 2; ++k) {
        int logn = 0;
        while ((1 << logn) < lens[k]) ++logn;
        const int sz = stage_table_len(lens[k]);
        void *h = calloc((size_t)sz, cs);
        if (!h) return DFSNUFFT_ERR_OOM;
        if (q.dtype == DFSNUFFT_F64) fill_stage_twiddles<double2, double>((double2 *)h, logn, DFS_FFT_E);
        else fill_stage_twiddles<float2, float>((float2 *)h, logn, DFS_FFT_E);
        cudaError_t e = cudaMemcpy(dst[k], h, cs * sz, cudaMemcpyHostToDevice);
        free(h);
        if (e) return fail_cuda(p, "upload stage twiddles", e);
    }
    return DFSNUFFT_OK;
}

// Double-single copies of an FP64 table: each value v as (hi, lo) FP32 with
// hi = v rounded, lo = v - hi rounded (48 significant bits).
static void split_table(const double *src, float *dst, size_t n) {
    for (size_t i = 0; i < n; ++i) {
        const float hi = (float)src[i];
        dst[2 * i] = hi;
        dst[2 * i + 1] = (float)(src[i] - (double)hi);
    }
}

// Tables of the double-single passes of an FP64 plan (p->gdf): twiddles of
// lengths n1 and n2 and the deconvolution factors, in the layout of the
// df32 / dfc types.
static int upload_df_tables(dfsnufft_plan p) {
    const dfsnufft_params &q = p->prm;
    const size_t nmax = (size_t)(q.n1 > q.n2 ? q.n1 : q.n2);
    double *d = (double *)malloc(sizeof(double) * 2 * nmax);
    float *f = (float *)malloc(sizeof(float) * 4 * nmax);
    int rc = (d && f) ? DFSNUFFT_OK : DFSNUFFT_ERR_OOM;
    struct { void **ptr; int n; bool tw; } tabs[] = {
        {&p->d_df_tw1, q.n1, true}, {&p->d_df_tw2, q.n2, true},
        {&p->d_df_inv1, q.N1, false}, {&p->d_df_inv2, q.N2, false}};
    for (int k = 0; rc == DFSNUFFT_OK && k < 4; ++k) {
        const int n = tabs[k].n;
        size_t vals;
        if (tabs[k].tw) {
            fill_twiddles<double2, double>((double2 *)d, n);
            vals = 2 * (size_t)n;
        } else {
            dfsnufft_kernel_ft(q.w, q.beta, k == 2 ? q.n1 : q.n2, n, d);
            for (int i = 0; i < n; ++i) d[i] = 1.0 / d[i];
            vals = (size_t)n;
        }
        split_table(d, f, vals);
        rc = dfs_alloc(p, tabs[k].ptr, sizeof(float) * 2 * vals, "double-single tables");
        if (rc == DFSNUFFT_OK) {
            const cudaError_t e =
                cudaMemcpy(*tabs[k].ptr, f, sizeof(float) * 2 * vals, cudaMemcpyHostToDevice);
            if (e) rc = fail_cuda(p, "upload double-single tables", e);
        }
    }
    free(d);
    free(f);
    // the stage-ordered twiddles of the phi pass's length-n1/2 transform and of
    // the theta pass's length-n2 one
    struct { void **ptr; int n; } stabs[] = {{&p->d_df_stw_phi, q.n1 / 2},
                                             {&p->d_df_stw_theta, q.n2},
                                             {&p->d_df_stw_half, q.n2 / 2}};
    for (int k = 0; rc == DFSNUFFT_OK && k < 3; ++k) {
        int logn = 0;
        while ((1 << logn) < stabs[k].n) ++logn;
        const size_t sz = (size_t)stage_table_len(stabs[k].n);
        double2 *h = (double2 *)calloc(sz, sizeof(double2));
        float *hf = (float *)malloc(sizeof(float) * 4 * sz);
        rc = (h && hf) ? DFSNUFFT_OK : DFSNUFFT_ERR_OOM;
        if (rc == DFSNUFFT_OK) {
            fill_stage_twiddles<double2, double>(h, logn, DFS_FFT_E);
            split_table(reinterpret_cast<const double *>(h), hf, 2 * sz);
            rc = dfs_alloc(p, stabs[k].ptr, sizeof(float) * 4 * sz, "double-single tables");
        }
        if (rc == DFSNUFFT_OK) {
            const cudaError_t e = cudaMemcpy(*stabs[k].ptr, hf, sizeof(float) * 4 * sz,
                                             cudaMemcpyHostToDevice);
            if (e) rc = fail_cuda(p, "upload double-single tables", e);
        }
        free(h);
        free(hf);
    }
    return rc;
}

static int upload_tables(dfsnufft_plan p) {
    const dfsnufft_params &q = p->prm;
    int rc;
    double *ft1 = (double *)malloc(sizeof(double) * q.N1);
    double *ft2 = (double *)malloc(sizeof(double) * q.N2);
    if (!ft1 || !ft2) {
        free(ft1); free(ft2);
        return DFSNUFFT_ERR_INVALID_ARG;
    }
    dfsnufft_kernel_ft(q.w, q.beta, q.n1, q.N1, ft1);
    dfsnufft_kernel_ft(q.w, q.beta, q.n2, q.N2, ft2);
    for (int i = 0; i < q.N1; ++i) ft1[i] = 1.0 / ft1[i];
    for (int i = 0; i < q.N2; ++i) ft2[i] = 1.0 / ft2[i];
    // factors in plan precision: FP64 values rounded once for FP32 plans
    size_t fs = sizeof(double);
    if (q.dtype == DFSNUFFT_F32) {
        float *f1 = (float *)ft1, *f2 = (float *)ft2;
        for (int i = 0; i < q.N1; ++i) f1[i] = (float)ft1[i];
        for (int i = 0; i < q.N2; ++i) f2[i] = (float)ft2[i];
        fs = sizeof(float);
    }
    cudaError_t e1 = cudaMemcpy(p->d_inv1, ft1, fs * q.N1, cudaMemcpyHostToDevice);
    cudaError_t e2 = cudaMemcpy(p->d_inv2, ft2, fs * q.N2, cudaMemcpyHostToDevice);
    free(ft1);
    free(ft2);
    if (e1 != cudaSuccess) return fail_cuda(p, "upload deconvolution factors", e1);
    if (e2 != cudaSuccess) return fail_cuda(p, "upload deconvolution factors", e2);

    size_t cs = q.dtype == DFSNUFFT_F64 ? sizeof(double2) : sizeof(float2);
    void *h1 = malloc(cs * q.n1), *h2 = malloc(cs * q.n2);
    if (!h1 || !h2) {
        free(h1); free(h2);
        return DFSNUFFT_ERR_INVALID_ARG;
    }
    if (q.dtype == DFSNUFFT_F64) {
        fill_twiddles<double2, double>((double2 *)h1, q.n1);
        fill_twiddles<double2, double>((double2 *)h2, q.n2);
    } else {
        fill_twiddles<float2, float>((float2 *)h1, q.n1);
        fill_twiddles<float2, float>((float2 *)h2, q.n2);
    }
    e1 = cudaMemcpy(p->d_tw1, h1, cs * q.n1, cudaMemcpyHostToDevice);
    e2 = cudaMemcpy(p->d_tw2, h2, cs * q.n2, cudaMemcpyHostToDevice);
    free(h1);
    free(h2);
    if (e1 != cudaSuccess) return fail_cuda(p, "upload twiddles", e1);
    if (e2 != cudaSuccess) return fail_cuda(p, "upload twiddles", e2);
    rc = DFSNUFFT_OK;
    return rc;
}

static int plan_create_impl(int n_members, int n_lon, int n_lat, double tol, int dtype,
                            int n_fields, const dfsnufft_options *opts, void *stream,
                            dfsnufft_plan *out) {
    if (!out) return DFSNUFFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_fields < 1 || n_fields > 64 || n_members < 1 || n_members > 4096 ||
        n_members * n_fields > 65535)
        return DFSNUFFT_ERR_INVALID_ARG;
    dfsnufft_params prm;
    int rc = dfsnufft_choose_params_opts(n_lon, n_lat, tol, dtype, opts, &prm);
    if (rc != DFSNUFFT_OK) return rc;

    dfsnufft_plan p = new (std::nothrow) dfsnufft_plan_s;
    if (!p) return DFSNUFFT_ERR_OOM;
    memset(p, 0, sizeof(*p));
    p->prm = prm;
    p->n_members = n_members;
    p->n_fields = n_fields;
    p->stream = (cudaStream_t)stream;
    p->herm = (prm.flags & DFSNUFFT_REAL_FIELDS) ? 1 : 0;
    p->keep_order = (prm.flags & DFSNUFFT_KEEP_ORDER) ? 1 : 0;
    // FP64 with sorted points: fine grid as double-single pairs, interpolation
    // on the FP32 units in double-single arithmetic
    p->gdf = (dtype == DFSNUFFT_F64 && !p->keep_order) ? 1 : 0;
    p->c0 = (prm.w % 2 == 0) ? prm.w / 2 - 1 : (prm.w - 1) / 2;
    p->nbx = prm.n1 / prm.tile_x;    // base cells lie in [0, n): no wrap bin
    p->nby = prm.n2 / prm.tile_y;
    p->nbins = p->nbx * p->nby;
    p->bstride = (p->nbins + 4) & ~3;     // 16-byte aligned member slices
    p->cstride = dfs_cstride(p->bstride, p->nbins, prm.tile_y);
    p->nch = (p->nbins + DFS_SCAN_CHUNK - 1) / DFS_SCAN_CHUNK;

    size_t cs = dtype == DFSNUFFT_F64 ? sizeof(double2) : sizeof(float2);
    const size_t nf = (size_t)n_fields * n_members;      // FFT lines
    const size_t nm = (size_t)n_members;
    struct { void **ptr; size_t bytes; const char *what; } allocs[] = {
        {&p->d_inv1, cs / 2 * prm.N1, "deconvolution factors"},
        {&p->d_inv2, cs / 2 * prm.N2, "deconvolution factors"},
        {&p->d_tw1, cs * prm.n1, "twiddles"},
        {&p->d_tw2, cs * prm.n2, "twiddles"},
        {&p->d_stw_theta, cs * stage_table_len(prm.n2 / 2), "stage twiddles"},
        {&p->d_stw_phi, cs * stage_table_len(prm.n1 / 2), "stage twiddles"},
        {&p->d_T, cs * nf * prm.n2 * dfs_tpitch(p->herm, prm.N1), "theta-pass buffer"},
        {&p->d_G, cs / 2 * nf * prm.n2 * prm.n1, "fine grid (real part)"},
        {(void **)&p->d_bin_count, sizeof(int) * p->cstride * nm, "bin counts and scan workspace"},
        {(void **)&p->d_bin_start, sizeof(int) * p->bstride * nm, "bin starts"},
        {(void **)&p->d_task_bin, sizeof(int) * p->bstride * nm, "bin list"},
        {(void **)&p->d_n_tasks, sizeof(int) * nm, "bin list size"},
        {(void **)&p->d_status, sizeof(int), "status word"},
        {(void **)&p->d_parity, sizeof(int) * 64, "field parities"},
        {(void **)&p->d_rowrange, sizeof(int2) * nm, "row ranges"},
        {(void **)&p->d_pofs, sizeof(int) * (nm + 1), "point offsets"},
        {(void **)&p->d_work, sizeof(int) * 2 * nm, "interpolation work counters"},
    };
    p->h_pofs = (int64_t *)calloc(nm + 1, sizeof(int64_t));
    if (!p->h_pofs) {
        delete p;
        return DFSNUFFT_ERR_OOM;
    }
    for (size_t i = 0; i < sizeof(allocs) / sizeof(allocs[0]); ++i) {
        rc = dfs_alloc(p, allocs[i].ptr, allocs[i].bytes, allocs[i].what);
        if (rc != DFSNUFFT_OK) {
            release(p);
            delete p;
            return rc;
        }
    }
    rc = upload_tables(p);
    if (rc == DFSNUFFT_OK) rc = upload_stage_tables(p);
    if (rc == DFSNUFFT_OK && p->gdf) rc = upload_df_tables(p);
    if (rc == DFSNUFFT_OK && p->gdf)
        rc = dfs_alloc(p, (void **)&p->d_emax, sizeof(int) * nf, "line exponents");
    if (rc == DFSNUFFT_OK && (prm.flags & DFSNUFFT_GAUSS_GRID)) {
        // samples on Gauss-Legendre latitudes: the solve matrices, in the theta-pass
        // buffer's room for the class matrices
        p->gl = 1;
        if (!dfs_forward_supported(prm) ||
            dfs_gl_scratch_bytes(prm, n_members * n_fields) >
                (dtype == DFSNUFFT_F64 ? sizeof(double2) : sizeof(float2)) *
                    (size_t)n_members * n_fields * prm.n2 * dfs_tpitch(p->herm, prm.N1))
            rc = DFSNUFFT_ERR_UNSUPPORTED;
        else
            rc = dfs_gl_setup(p);
    }
    if (rc == DFSNUFFT_OK) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (!e) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (!e) e = cudaMemset(p->d_status, 0, sizeof(int));
        if (!e) e = cudaMemset(p->d_work, 0, sizeof(int) * 2 * nm);
        if (e) rc = fail_cuda(p, "device query", e);
    }
    if (rc != DFSNUFFT_OK) {
        release(p);
        delete p;
        return rc;
    }
    *out = p;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_plan_create(int n_lon, int n_lat, double tol, int dtype, int n_fields,
                                    void *stream, dfsnufft_plan *out) {
    return plan_create_impl(1, n_lon, n_lat, tol, dtype, n_fields, nullptr, stream, out);
}

extern "C" int dfsnufft_plan_create_batch(int n_members, int n_lon, int n_lat, double tol,
                                          int dtype, int n_fields, void *stream,
                                          dfsnufft_plan *out) {
    return plan_create_impl(n_members, n_lon, n_lat, tol, dtype, n_fields, nullptr, stream, out);
}

extern "C" int dfsnufft_plan_create_opts(int n_members, int n_lon, int n_lat, double tol,
                                         int dtype, int n_fields, const dfsnufft_options *opts,
                                         void *stream, dfsnufft_plan *out) {
    return plan_create_impl(n_members, n_lon, n_lat, tol, dtype, n_fields, opts, stream, out);
}

extern "C" int dfsnufft_destroy(dfsnufft_plan p) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    cudaStreamSynchronize(p->stream);
    release(p);
    delete p;
    return DFSNUFFT_OK;
}

extern "C" const char *dfsnufft_plan_last_error(dfsnufft_plan p) { return p ? p->msg : ""; }

extern "C" int dfsnufft_plan_check(dfsnufft_plan p) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    DFS_CK(p, cudaStreamSynchronize(p->stream));
    int st = 0;
    DFS_CK(p, cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        p->status = DFSNUFFT_ERR_TIMEOUT;
        snprintf(p->msg, sizeof(p->msg), "a kernel gave up waiting on an asynchronous copy");
    }
    return p->status;
}

extern "C" int dfsnufft_plan_get_params(dfsnufft_plan p, dfsnufft_params *out) {
    if (!p || !out) return DFSNUFFT_ERR_INVALID_ARG;
    *out = p->prm;
    return DFSNUFFT_OK;
}

// ------------------------------------------------------------------ points

static int ensure_point_capacity(dfsnufft_plan p, int64_t n) {
    if (n <= p->cap_points) return DFSNUFFT_OK;
    // the stream may still use the old buffers
    DFS_CK(p, cudaStreamSynchronize(p->stream));
    dfs_free(&p->d_urec);
    dfs_free((void **)&p->d_base);
    dfs_free(&p->d_frac);
    dfs_free((void **)&p->d_idx);
    p->cap_points = 0;
    size_t rs = p->prm.dtype == DFSNUFFT_F64 ? sizeof(double) : sizeof(float);
    int rc;
    if ((rc = dfs_alloc(p, &p->d_urec, (size_t)dfs_fold_rec_bytes(p->prm.dtype) * n,
                        "unsorted point records")) ||
        (rc = dfs_alloc(p, (void **)&p->d_base, sizeof(int2) * n, "point bases")) ||
        (rc = dfs_alloc(p, &p->d_frac, 2 * rs * n, "point offsets")) ||
        (rc = dfs_alloc(p, (void **)&p->d_idx, sizeof(int) * n, "point order")))
        return rc;
    p->cap_points = n;
    return DFSNUFFT_OK;
}

// Record the members' point counts; the device offsets are uploaded only when
// they change (so that repeated calls enqueue no host-to-device copy).
static int update_counts(dfsnufft_plan p, const int64_t *counts) {
    const int M = p->n_members;
    int64_t total = 0, mx = 0;
    bool same = p->has_points;
    for (int k = 0; k < M; ++k) {
        if (counts[k] < 1) return DFSNUFFT_ERR_INVALID_ARG;
        if (p->h_pofs[k + 1] - p->h_pofs[k] != counts[k]) same = false;
        total += counts[k];
        if (counts[k] > mx) mx = counts[k];
    }
    if (total > 0x7fffffffLL) return DFSNUFFT_ERR_INVALID_ARG;
    int rc = ensure_point_capacity(p, total);
    if (rc) return rc;
    if (!same) {
        p->h_pofs[0] = 0;
        for (int k = 0; k < M; ++k) p->h_pofs[k + 1] = p->h_pofs[k] + counts[k];
        int *tmp = (int *)malloc(sizeof(int) * (M + 1));
        if (!tmp) return DFSNUFFT_ERR_OOM;
        for (int k = 0; k <= M; ++k) tmp[k] = (int)p->h_pofs[k];
        cudaError_t e = cudaMemcpyAsync(p->d_pofs, tmp, sizeof(int) * (M + 1),
                                        cudaMemcpyHostToDevice, p->stream);
        free(tmp);
        if (e) return fail_cuda(p, "upload point offsets", e);
    }
    p->n_points = total;
    p->max_member_points = mx;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_set_points_batch(dfsnufft_plan p, const int64_t *n_points,
                                         const double *lon, const double *colat) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (!n_points || !lon || !colat) return DFSNUFFT_ERR_INVALID_ARG;
    int rc = update_counts(p, n_points);
    if (rc) return rc;
    p->has_points = 0;
    DFS_CK(p, timing_begin(p, 0));
    DFS_CK(p, dfs_launch_set_points(p, lon, colat));
    DFS_CK(p, timing_end(p, 0));
    p->has_points = 1;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_set_points(dfsnufft_plan p, int64_t n_points, const double *lon,
                                   const double *colat) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->n_members != 1) return DFSNUFFT_ERR_INVALID_ARG;
    if (n_points < 1 || n_points > 0x7fffffffLL) return DFSNUFFT_ERR_INVALID_ARG;
    return dfsnufft_set_points_batch(p, &n_points, lon, colat);
}

extern "C" int dfsnufft_execute(dfsnufft_plan p, const void *coeffs, void *values) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (!p->has_points) return DFSNUFFT_ERR_NO_POINTS;
    if (!coeffs || !values) return DFSNUFFT_ERR_INVALID_ARG;
    DFS_CK(p, timing_begin(p, 1));
    DFS_CK(p, dfs_launch_theta_pass(p, coeffs));
    DFS_CK(p, timing_end(p, 1));
    DFS_CK(p, timing_begin(p, 2));
    DFS_CK(p, dfs_launch_phi_pass(p));
    DFS_CK(p, timing_end(p, 2));
    DFS_CK(p, timing_begin(p, 3));
    DFS_CK(p, dfs_launch_interp(p, values));
    DFS_CK(p, timing_end(p, 3));
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_execute_pr(dfsnufft_plan p, int M, int N, const void *pr, void *values) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (!p->has_points) return DFSNUFFT_ERR_NO_POINTS;
    if (!pr || !values || !p->herm) return DFSNUFFT_ERR_INVALID_ARG;
    if (M < 0 || M > p->prm.N1 / 2 - 1 || N < 1 || N > p->prm.N2 / 2 - 1)
        return DFSNUFFT_ERR_INVALID_ARG;
    DFS_CK(p, timing_begin(p, 1));
    DFS_CK(p, dfs_launch_theta_pass(p, pr, M, N));
    DFS_CK(p, timing_end(p, 1));
    DFS_CK(p, timing_begin(p, 2));
    DFS_CK(p, dfs_launch_phi_pass(p));
    DFS_CK(p, timing_end(p, 2));
    DFS_CK(p, timing_begin(p, 3));
    DFS_CK(p, dfs_launch_interp(p, values));
    DFS_CK(p, timing_end(p, 3));
    return DFSNUFFT_OK;
}

// ------------------------------------------------------------------ grid values

// Upload the fields' parities when they differ from the last ones uploaded.
static int set_parity(dfsnufft_plan p, const int *parity) {
    const int F = p->n_fields;
    bool same = p->parity_set != 0;
    for (int f = 0; f < F; ++f) {
        if (parity[f] != 1 && parity[f] != -1) return DFSNUFFT_ERR_INVALID_ARG;
        if (p->h_parity[f] != parity[f]) same = false;
    }
    if (same) return DFSNUFFT_OK;
    for (int f = 0; f < F; ++f) p->h_parity[f] = parity[f];
    DFS_CK(p, cudaMemcpyAsync(p->d_parity, p->h_parity, sizeof(int) * F,
                              cudaMemcpyHostToDevice, p->stream));
    // the copy reads h_parity; finish it before the host may change the array
    DFS_CK(p, cudaStreamSynchronize(p->stream));
    p->parity_set = 1;
    return DFSNUFFT_OK;
}

static int grid_to_coeffs(dfsnufft_plan p, const void *samples, const int *parity,
                          void *coeffs, bool full) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (!samples || !parity || !coeffs) return DFSNUFFT_ERR_INVALID_ARG;
    if (!dfs_forward_supported(p->prm)) return DFSNUFFT_ERR_UNSUPPORTED;
    int rc = set_parity(p, parity);
    if (rc) return rc;
    if (p->gl) {
        rc = dfs_launch_forward_gl(p, samples, p->d_parity, coeffs, full);
        if (rc) {
            p->status = rc;
            snprintf(p->msg, sizeof(p->msg), "Gauss-Legendre grid to coefficients failed");
        }
        return rc;
    }
    DFS_CK(p, dfs_launch_forward(p, samples, p->d_parity, coeffs, full));
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_grid_to_coeffs(dfsnufft_plan p, const void *samples, const int *parity,
                                       void *coeffs) {
    return grid_to_coeffs(p, samples, parity, coeffs, true);
}

extern "C" int dfsnufft_interpolate_grid(dfsnufft_plan p, const void *samples, const int *parity,
                                         void *values) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (!p->has_points) return DFSNUFFT_ERR_NO_POINTS;
    if (!samples || !parity || !values) return DFSNUFFT_ERR_INVALID_ARG;
    if (!dfs_forward_supported(p->prm)) return DFSNUFFT_ERR_UNSUPPORTED;
    if (!p->d_coef_stage) {
        const size_t cs = p->prm.dtype == DFSNUFFT_F64 ? sizeof(double2) : sizeof(float2);
        int rc = dfs_alloc(p, &p->d_coef_stage,
                           cs * (size_t)p->n_members * p->n_fields * p->prm.N2 * p->prm.N1,
                           "coefficient staging");
        if (rc) return rc;
    }
    // a real-field plan reads the columns m >= 0 and the Nyquist row only
    int rc = grid_to_coeffs(p, samples, parity, p->d_coef_stage, !p->herm);
    if (rc) return rc;
    rc = dfsnufft_execute(p, p->d_coef_stage, values);
    if (rc) return rc;
    if (p->copy_stream) DFS_CK(p, cudaEventRecord(p->stage_free, p->stream));
    return DFSNUFFT_OK;
}

// ------------------------------------------------------------------ host-buffer variants

// Device staging of the host points, sized to the point capacity.
static int ensure_point_staging(dfsnufft_plan p) {
    if (p->pts_stage_cap >= p->cap_points) return DFSNUFFT_OK;
    DFS_CK(p, cudaStreamSynchronize(p->stream));
    dfs_free((void **)&p->d_pts_stage);
    p->pts_stage_cap = 0;
    const int rc = dfs_alloc(p, (void **)&p->d_pts_stage, 2 * sizeof(double) * p->cap_points,
                             "point staging");
    if (rc) return rc;
    p->pts_stage_cap = p->cap_points;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_set_points_host(dfsnufft_plan p, int64_t n_points, const double *lon,
                                        const double *colat) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (p->n_members != 1 || n_points < 1 || n_points > 0x7fffffffLL || !lon || !colat)
        return DFSNUFFT_ERR_INVALID_ARG;
    int rc = update_counts(p, &n_points);
    if (rc) return rc;
    rc = ensure_point_staging(p);
    if (rc) return rc;
    size_t b = sizeof(double) * (size_t)n_points;
    DFS_CK(p, cudaMemcpyAsync(p->d_pts_stage, lon, b, cudaMemcpyHostToDevice, p->stream));
    DFS_CK(p, cudaMemcpyAsync(p->d_pts_stage + p->pts_stage_cap, colat, b,
                              cudaMemcpyHostToDevice, p->stream));
    // the next execute_host's coefficient copies queue behind these on the link
    if (!p->pts_copied)
        DFS_CK(p, cudaEventCreateWithFlags(&p->pts_copied, cudaEventDisableTiming));
    DFS_CK(p, cudaEventRecord(p->pts_copied, p->stream));
    p->pts_pending = 1;
    p->has_points = 0;
    DFS_CK(p, timing_begin(p, 0));
    DFS_CK(p, dfs_launch_set_points(p, p->d_pts_stage, p->d_pts_stage + p->pts_stage_cap));
    DFS_CK(p, timing_end(p, 0));
    p->has_points = 1;
    return DFSNUFFT_OK;
}

// Host coefficients into the staging buffer.  A real-field plan's theta pass
// reads the columns m >= 0 (array columns N1/2 .. N1-1), the Nyquist column
// m = -N1/2 (array column 0) and the Nyquist row n = -N2/2 (row 0 of each line),
// so only those are copied: in row-major order the columns N1/2 .. N1-1 of one
// row and column 0 of the next are contiguous, one 2-D copy of N1/2 + 1
// elements a row takes both, and the first row of each line is copied from
// column 0 to N1/2.  Other plans copy the whole array.
// Lines l0 .. l0 + nl - 1 of the coefficients (all lines: nl = members x fields).
static cudaError_t stage_coefficients(dfsnufft_plan p, const void *coeffs, size_t cs,
                                      cudaStream_t st, int l0, int nl) {
    const dfsnufft_params &q = p->prm;
    const size_t rows = (size_t)nl * q.N2;
    const size_t row = cs * q.N1, half = cs * (q.N1 / 2);
    const size_t off = (size_t)l0 * q.N2 * row;
    char *d = static_cast<char *>(p->d_coef_stage) + off;
    const char *h = static_cast<const char *>(coeffs) + off;
    if (!p->herm)
        return cudaMemcpyAsync(d, h, rows * row, cudaMemcpyHostToDevice, st);
    cudaError_t e = cudaSuccess;
    if (rows > 1)
        e = cudaMemcpy2DAsync(d + half, row, h + half, row, half + cs, rows - 1,
                              cudaMemcpyHostToDevice, st);
    if (!e)
        e = cudaMemcpyAsync(d + (rows - 1) * row + half, h + (rows - 1) * row + half, half,
                            cudaMemcpyHostToDevice, st);
    if (!e)
        e = cudaMemcpy2DAsync(d, (size_t)q.N2 * row, h, (size_t)q.N2 * row, half + cs,
                              (size_t)nl, cudaMemcpyHostToDevice, st);
    return e;
}

// Bytes stage_coefficients copies.
static size_t staged_coefficient_bytes(dfsnufft_plan p, size_t cs) {
    const dfsnufft_params &q = p->prm;
    const size_t lines = (size_t)p->n_members * p->n_fields;
    const size_t rows = lines * q.N2;
    const size_t half = cs * (q.N1 / 2);
    if (!p->herm) return rows * cs * q.N1;
    return (rows - 1) * (half + cs) + half + lines * (half + cs);
}

// At least 2 n events for the per-field pipeline of execute_host.
static int ensure_line_events(dfsnufft_plan p, int n) {
    if (p->n_line_ev >= 2 * n) return DFSNUFFT_OK;
    cudaEvent_t *ev = (cudaEvent_t *)realloc(p->line_ev, sizeof(cudaEvent_t) * 2 * n);
    if (!ev) return DFSNUFFT_ERR_OOM;
    p->line_ev = ev;
    for (int i = p->n_line_ev; i < 2 * n; ++i) {
        DFS_CK(p, cudaEventCreateWithFlags(&p->line_ev[i], cudaEventDisableTiming));
        p->n_line_ev = i + 1;
    }
    if (!p->vals_copied)
        DFS_CK(p, cudaEventCreateWithFlags(&p->vals_copied, cudaEventDisableTiming));
    return DFSNUFFT_OK;
}

// Device staging of host coefficients and values, the copy stream and its
// events (cs: bytes of one complex coefficient).
static int ensure_host_staging(dfsnufft_plan p, size_t cs) {
    const dfsnufft_params &q = p->prm;
    const size_t rs = cs / 2;
    int rc;
    if (!p->d_coef_stage) {
        rc = dfs_alloc(p, &p->d_coef_stage, cs * (size_t)p->n_members * p->n_fields * q.N2 * q.N1,
                       "coefficient staging");
        if (rc) return rc;
    }
    if (p->val_stage_cap < p->n_points) {
        DFS_CK(p, cudaStreamSynchronize(p->stream));
        dfs_free(&p->d_val_stage);
        rc = dfs_alloc(p, &p->d_val_stage, rs * (size_t)p->n_fields * p->cap_points,
                       "value staging");
        if (rc) return rc;
        p->val_stage_cap = p->cap_points;
    }
    if (!p->copy_stream) {
        DFS_CK(p, cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
        DFS_CK(p, cudaEventCreateWithFlags(&p->stage_free, cudaEventDisableTiming));
        DFS_CK(p, cudaEventCreateWithFlags(&p->coef_ready, cudaEventDisableTiming));
        DFS_CK(p, cudaEventRecord(p->stage_free, p->stream));     // every earlier reader
    }
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_execute_host(dfsnufft_plan p, const void *coeffs, void *values) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (!p->has_points) return DFSNUFFT_ERR_NO_POINTS;
    if (!coeffs || !values) return DFSNUFFT_ERR_INVALID_ARG;
    const dfsnufft_params &q = p->prm;
    size_t cs = q.dtype == DFSNUFFT_F64 ? sizeof(double2) : sizeof(float2);
    size_t rs = cs / 2;
    size_t vb = rs * (size_t)p->n_fields * (size_t)p->n_points;
    int rc = ensure_host_staging(p, cs);
    if (rc) return rc;
    // the copies wait only for the last reader of the staging buffer (and for
    // set_points_host's point copies, which use the same link), not for the
    // set_points kernels queued on the plan's stream
    DFS_CK(p, cudaStreamWaitEvent(p->copy_stream, p->stage_free, 0));
    if (p->pts_pending) {
        DFS_CK(p, cudaStreamWaitEvent(p->copy_stream, p->pts_copied, 0));
        p->pts_pending = 0;
    }
    const int F = p->n_fields;
    if (p->n_members == 1 && F > 1 && q.dtype == DFSNUFFT_F32) {
        // FP32 (bound by the host link): pipelined per field, so that field f's
        // transform and interpolation start once its coefficients have landed,
        // and its values travel back while later fields are still being copied
        // in or computed.  FP64 plans are bound by arithmetic and take one
        // transform of all fields.
        rc = ensure_line_events(p, F);
        if (rc) return rc;
        if (!p->back_stream)
            DFS_CK(p, cudaStreamCreateWithFlags(&p->back_stream, cudaStreamNonBlocking));
        for (int f = 0; f < F; ++f) {
            DFS_CK(p, stage_coefficients(p, coeffs, cs, p->copy_stream, f, 1));
            DFS_CK(p, cudaEventRecord(p->line_ev[2 * f], p->copy_stream));
        }
        const size_t fb = rs * (size_t)p->n_points;
        for (int f = 0; f < F; ++f) {
            DFS_CK(p, cudaStreamWaitEvent(p->stream, p->line_ev[2 * f], 0));
            p->win0 = f;
            p->nwin = 1;
            rc = dfsnufft_execute(p, p->d_coef_stage, p->d_val_stage);
            p->win0 = p->nwin = 0;
            if (rc) return rc;
            DFS_CK(p, cudaEventRecord(p->line_ev[2 * f + 1], p->stream));
            DFS_CK(p, cudaStreamWaitEvent(p->back_stream, p->line_ev[2 * f + 1], 0));
            DFS_CK(p, cudaMemcpyAsync(static_cast<char *>(values) + f * fb,
                                      static_cast<const char *>(p->d_val_stage) + f * fb, fb,
                                      cudaMemcpyDeviceToHost, p->back_stream));
        }
        DFS_CK(p, cudaEventRecord(p->stage_free, p->stream));
        DFS_CK(p, cudaEventRecord(p->vals_copied, p->back_stream));
        DFS_CK(p, cudaStreamWaitEvent(p->stream, p->vals_copied, 0));
        return dfsnufft_plan_check(p);
    }
    DFS_CK(p, stage_coefficients(p, coeffs, cs, p->copy_stream, 0, p->n_members * F));
    DFS_CK(p, cudaEventRecord(p->coef_ready, p->copy_stream));
    DFS_CK(p, cudaStreamWaitEvent(p->stream, p->coef_ready, 0));
    rc = dfsnufft_execute(p, p->d_coef_stage, p->d_val_stage);
    if (rc) return rc;
    DFS_CK(p, cudaEventRecord(p->stage_free, p->stream));
    DFS_CK(p, cudaMemcpyAsync(values, p->d_val_stage, vb, cudaMemcpyDeviceToHost, p->stream));
    return dfsnufft_plan_check(p);
}

namespace {
// Every fine row of every member needed: the theta and phi passes of a field
// transformed before the points are sorted compute all rows.
__global__ void k_rowrange_all(int2 *rowrange, int members, int n2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < members) rowrange[k] = make_int2(0, n2);
}
}  // namespace

// set_points_host then execute_host, scheduled together.  For a one-member FP32
// plan of several fields the host link carries field 0's coefficients first,
// then the points, then the other fields' coefficients; field 0's theta and phi
// passes (over every fine row, the needed range being unknown until the points
// are sorted) run while the points travel, and each field's values go back as
// soon as it is done.  Other plans run the two calls one after the other.
extern "C" int dfsnufft_execute_points_host(dfsnufft_plan p, int64_t n_points, const double *lon,
                                            const double *colat, const void *coeffs,
                                            void *values) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    const dfsnufft_params &q = p->prm;
    const int F = p->n_fields;
    if (p->n_members != 1 || F < 2 || q.dtype != DFSNUFFT_F32) {
        const int rc = dfsnufft_set_points_host(p, n_points, lon, colat);
        return rc ? rc : dfsnufft_execute_host(p, coeffs, values);
    }
    if (n_points < 1 || n_points > 0x7fffffffLL || !lon || !colat || !coeffs || !values)
        return DFSNUFFT_ERR_INVALID_ARG;
    int rc = update_counts(p, &n_points);
    if (rc) return rc;
    const size_t cs = sizeof(float2), rs = sizeof(float);
    if ((rc = ensure_point_staging(p)) || (rc = ensure_host_staging(p, cs)) ||
        (rc = ensure_line_events(p, F)))
        return rc;
    if (!p->back_stream)
        DFS_CK(p, cudaStreamCreateWithFlags(&p->back_stream, cudaStreamNonBlocking));
    if (!p->pts_copied)
        DFS_CK(p, cudaEventCreateWithFlags(&p->pts_copied, cudaEventDisableTiming));
    // the copies wait for everything queued before the call (the last readers
    // of the point and coefficient staging among it)
    DFS_CK(p, cudaEventRecord(p->stage_free, p->stream));
    DFS_CK(p, cudaStreamWaitEvent(p->copy_stream, p->stage_free, 0));
    p->pts_pending = 0;
    p->has_points = 0;
    DFS_CK(p, stage_coefficients(p, coeffs, cs, p->copy_stream, 0, 1));
    DFS_CK(p, cudaEventRecord(p->line_ev[0], p->copy_stream));
    const size_t b = sizeof(double) * (size_t)n_points;
    DFS_CK(p, cudaMemcpyAsync(p->d_pts_stage, lon, b, cudaMemcpyHostToDevice, p->copy_stream));
    DFS_CK(p, cudaMemcpyAsync(p->d_pts_stage + p->pts_stage_cap, colat, b,
                              cudaMemcpyHostToDevice, p->copy_stream));
    DFS_CK(p, cudaEventRecord(p->pts_copied, p->copy_stream));
    for (int f = 1; f < F; ++f) {
        DFS_CK(p, stage_coefficients(p, coeffs, cs, p->copy_stream, f, 1));
        DFS_CK(p, cudaEventRecord(p->line_ev[2 * f], p->copy_stream));
    }
    // field 0's transform over every row while the points travel
    DFS_CK(p, cudaStreamWaitEvent(p->stream, p->line_ev[0], 0));
    k_rowrange_all<<<1, 32, 0, p->stream>>>(p->d_rowrange, p->n_members, q.n2);
    DFS_CK(p, cudaGetLastError());
    p->win0 = 0;
    p->nwin = 1;
    DFS_CK(p, timing_begin(p, 1));
    DFS_CK(p, dfs_launch_theta_pass(p, p->d_coef_stage));
    DFS_CK(p, timing_end(p, 1));
    DFS_CK(p, timing_begin(p, 2));
    DFS_CK(p, dfs_launch_phi_pass(p));
    DFS_CK(p, timing_end(p, 2));
    p->win0 = p->nwin = 0;
    // the points sorted (this also sets the needed row range of the later fields)
    DFS_CK(p, cudaStreamWaitEvent(p->stream, p->pts_copied, 0));
    DFS_CK(p, timing_begin(p, 0));
    DFS_CK(p, dfs_launch_set_points(p, p->d_pts_stage, p->d_pts_stage + p->pts_stage_cap));
    DFS_CK(p, timing_end(p, 0));
    p->has_points = 1;
    const size_t fb = rs * (size_t)n_points;
    for (int f = 0; f < F; ++f) {
        p->win0 = f;
        p->nwin = 1;
        if (f > 0) {
            DFS_CK(p, cudaStreamWaitEvent(p->stream, p->line_ev[2 * f], 0));
            DFS_CK(p, timing_begin(p, 1));
            DFS_CK(p, dfs_launch_theta_pass(p, p->d_coef_stage));
            DFS_CK(p, timing_end(p, 1));
            DFS_CK(p, timing_begin(p, 2));
            DFS_CK(p, dfs_launch_phi_pass(p));
            DFS_CK(p, timing_end(p, 2));
        }
        DFS_CK(p, timing_begin(p, 3));
        DFS_CK(p, dfs_launch_interp(p, p->d_val_stage));
        DFS_CK(p, timing_end(p, 3));
        p->win0 = p->nwin = 0;
        DFS_CK(p, cudaEventRecord(p->line_ev[2 * f + 1], p->stream));
        DFS_CK(p, cudaStreamWaitEvent(p->back_stream, p->line_ev[2 * f + 1], 0));
        DFS_CK(p, cudaMemcpyAsync(static_cast<char *>(values) + f * fb,
                                  static_cast<const char *>(p->d_val_stage) + f * fb, fb,
                                  cudaMemcpyDeviceToHost, p->back_stream));
    }
    DFS_CK(p, cudaEventRecord(p->stage_free, p->stream));
    DFS_CK(p, cudaEventRecord(p->vals_copied, p->back_stream));
    DFS_CK(p, cudaStreamWaitEvent(p->stream, p->vals_copied, 0));
    return dfsnufft_plan_check(p);
}

// ------------------------------------------------------------------ measurement aids

extern "C" int dfsnufft_plan_host_copy_bytes(dfsnufft_plan p, int64_t *points_h2d,
                                             int64_t *coeffs_h2d, int64_t *values_d2h) {
    if (!p || !points_h2d || !coeffs_h2d || !values_d2h) return DFSNUFFT_ERR_INVALID_ARG;
    const size_t cs = p->prm.dtype == DFSNUFFT_F64 ? sizeof(double2) : sizeof(float2);
    *points_h2d = (int64_t)(2 * sizeof(double) * (size_t)p->n_points);
    *coeffs_h2d = (int64_t)staged_coefficient_bytes(p, cs);
    *values_d2h = (int64_t)(cs / 2 * (size_t)p->n_fields * (size_t)p->n_points);
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_plan_enable_timing(dfsnufft_plan p, int enable) {
    if (!p) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (enable && !p->ev) {
        const int n = 2 * DFS_TIMING_SLOTS * DFSNUFFT_N_STAGES;
        p->ev = (cudaEvent_t *)calloc(n, sizeof(cudaEvent_t));
        if (!p->ev) return DFSNUFFT_ERR_OOM;
        for (int i = 0; i < n; ++i) DFS_CK(p, cudaEventCreate(&p->ev[i]));
    }
    if (p->timing) DFS_CK(p, timing_drain(p));
    for (int s = 0; s < DFSNUFFT_N_STAGES; ++s) {
        p->pending[s] = 0;
        p->ms_total[s] = 0.0;
        p->calls[s] = 0;
    }
    p->timing = enable ? 1 : 0;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_plan_read_timing(dfsnufft_plan p, double *ms_total, int64_t *calls) {
    if (!p || !ms_total || !calls) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (p->timing) DFS_CK(p, timing_drain(p));
    for (int s = 0; s < DFSNUFFT_N_STAGES; ++s) {
        ms_total[s] = p->ms_total[s];
        calls[s] = p->calls[s];
    }
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_plan_point_stats(dfsnufft_plan p, int64_t *rows_needed,
                                         int64_t *nonempty_bins) {
    if (!p || !rows_needed || !nonempty_bins) return DFSNUFFT_ERR_INVALID_ARG;
    if (p->status) return p->status;
    if (!p->has_points) return DFSNUFFT_ERR_NO_POINTS;
    DFS_CK(p, cudaStreamSynchronize(p->stream));
    const int M = p->n_members;
    int2 *range = (int2 *)malloc(sizeof(int2) * M);
    int *ntask = (int *)malloc(sizeof(int) * M);
    if (!range || !ntask) {
        free(range);
        free(ntask);
        return DFSNUFFT_ERR_OOM;
    }
    cudaError_t e1 = cudaMemcpy(range, p->d_rowrange, sizeof(int2) * M, cudaMemcpyDeviceToHost);
    cudaError_t e2 = cudaMemcpy(ntask, p->d_n_tasks, sizeof(int) * M, cudaMemcpyDeviceToHost);
    int64_t rows = 0, bins = 0;
    for (int k = 0; k < M; ++k) {
        rows += range[k].y;
        bins += ntask[k];
    }
    free(range);
    free(ntask);
    if (e1) return fail_cuda(p, "read row ranges", e1);
    if (e2) return fail_cuda(p, "read bin counts", e2);
    // per field: the members' average
    const int64_t blocks = (rows / M) / DFS_ROW_BLOCK;
    *rows_needed = blocks * DFS_ROW_BLOCK;
    *nonempty_bins = bins;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_plan_latitudes(dfsnufft_plan p, double *colat) {
    if (!p || !colat) return DFSNUFFT_ERR_INVALID_ARG;
    const int N = p->prm.n_lat;
    for (int j = 0; j < N; ++j)
        colat[j] = p->gl ? p->h_gl_colat[j] : (j + 0.5) * (3.14159265358979323846 / N);
    return DFSNUFFT_OK;
}

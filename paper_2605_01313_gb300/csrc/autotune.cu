// Autotuner: chooses a plan's interpolation bin size, oversampling factor and
// kernel width for one workload by measurement.  Every candidate is a real plan
// run on the caller's points and coefficients (set_points + execute, timed with
// CUDA events on the caller's stream); its values at a sample of member 0's
// points are compared with an FP64 plan at tol 1e-14 (a general plan, the
// accuracy reference), and a candidate counts only if its relative l-inf error
// stays within the acceptance bound of the requested tolerance.
//
// Search, in two stages: (1) every bin size of the candidate set at the
// width rule's kernel and oversampling 2; (2) with the fastest accepted bin,
// one kernel narrower than the rule at oversampling 2, the unsorted-points
// form (DFSNUFFT_KEEP_ORDER), and oversampling 4 at its own width rule and one
// narrower.  The fastest accepted candidate wins;
// the default configuration is always among the candidates.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

__global__ void k_widen(const float2 *__restrict__ in, double2 *__restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_double2(in[i].x, in[i].y);
}

__global__ void k_gather(const double *__restrict__ src, const int *__restrict__ idx, int n,
                         double *__restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    bool alloc(size_t bytes) { return cudaMalloc(&p, bytes) == cudaSuccess; }
};

// Time one candidate and measure its error on the sample.
int run_candidate(const dfsnufft_tune_args *a, const dfsnufft_options &o,
                  const std::vector<int> &sample, const std::vector<double> &ref, double ref_max,
                  void *values, std::vector<unsigned char> &host_vals, dfsnufft_tune_result *res) {
    memset(res, 0, sizeof(*res));
    res->opts = o;
    res->ms = INFINITY;
    res->err = INFINITY;
    dfsnufft_plan p = nullptr;
    int rc = dfsnufft_plan_create_opts(a->n_members, a->n_lon, a->n_lat, a->tol, a->dtype,
                                       a->n_fields, &o, a->stream, &p);
    if (rc) {
        res->status = rc;
        return DFSNUFFT_OK;
    }
    dfsnufft_plan_get_params(p, &res->prm);
    cudaStream_t s = (cudaStream_t)a->stream;
    const int steps = a->steps > 0 ? a->steps : 5;
    std::vector<float> ms;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) rc = DFSNUFFT_ERR_CUDA;
    for (int it = -1; it < steps && !rc; ++it) {        // it = -1: untimed warm-up
        if (it >= 0 && cudaEventRecord(e0, s)) rc = DFSNUFFT_ERR_CUDA;
        if (!rc) rc = dfsnufft_set_points_batch(p, a->n_points, a->lon, a->colat);
        if (!rc) rc = dfsnufft_execute(p, a->coeffs, values);
        if (!rc && it >= 0) {
            float t = 0;
            if (cudaEventRecord(e1, s) || cudaEventSynchronize(e1) ||
                cudaEventElapsedTime(&t, e0, e1))
                rc = DFSNUFFT_ERR_CUDA;
            ms.push_back(t);
        }
    }
    if (!rc) rc = dfsnufft_plan_check(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfsnufft_destroy(p);
    res->status = rc;
    if (rc) {
        // a candidate the device cannot run (launch limits) is skipped; a
        // failure that leaves the stream broken ends the search
        cudaGetLastError();
        return cudaStreamSynchronize(s) == cudaSuccess ? DFSNUFFT_OK : DFSNUFFT_ERR_CUDA;
    }
    std::sort(ms.begin(), ms.end());
    res->ms = ms[ms.size() / 2];
    // member 0's values: fields x n_points[0]
    const size_t rsz = a->dtype == DFSNUFFT_F64 ? sizeof(double) : sizeof(float);
    const int64_t P0 = a->n_points[0];
    if (cudaMemcpy(host_vals.data(), values, rsz * a->n_fields * P0, cudaMemcpyDeviceToHost))
        return DFSNUFFT_ERR_CUDA;
    double err = 0;
    const int ns = (int)sample.size();
    for (int f = 0; f < a->n_fields; ++f) {
        double e = 0, mx = 0;
        for (int i = 0; i < ns; ++i) {
            const size_t at = (size_t)f * P0 + sample[i];
            const double v = rsz == 8 ? ((const double *)host_vals.data())[at]
                                      : (double)((const float *)host_vals.data())[at];
            const double r = ref[(size_t)f * ns + i];
            e = fmax(e, fabs(v - r));
            mx = fmax(mx, fabs(r));
        }
        err = fmax(err, e / fmax(mx, ref_max * 1e-300));
    }
    res->err = err;
    return DFSNUFFT_OK;
}

}  // namespace

extern "C" int dfsnufft_autotune(const dfsnufft_tune_args *a, dfsnufft_tune_result *results,
                                 int max_results, int *n_results, dfsnufft_options *best) {
    if (!a || !best || !a->n_points || !a->lon || !a->colat || !a->coeffs || a->n_members < 1 ||
        a->n_fields < 1 || (a->flags & ~(DFSNUFFT_REAL_FIELDS | DFSNUFFT_KEEP_ORDER)))
        return DFSNUFFT_ERR_INVALID_ARG;
    if (n_results) *n_results = 0;
    dfsnufft_params dp;
    dfsnufft_options base;
    memset(&base, 0, sizeof(base));
    base.flags = a->flags;
    int rc = dfsnufft_choose_params_opts(a->n_lon, a->n_lat, a->tol, a->dtype, &base, &dp);
    if (rc) return rc;
    int64_t total = 0;
    for (int k = 0; k < a->n_members; ++k) {
        if (a->n_points[k] < 1) return DFSNUFFT_ERR_INVALID_ARG;
        total += a->n_points[k];
    }
    if (total > 0x7fffffffLL) return DFSNUFFT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)a->stream;
    const int F = a->n_fields;
    const int64_t P0 = a->n_points[0];
    const size_t rsz = a->dtype == DFSNUFFT_F64 ? sizeof(double) : sizeof(float);
    const size_t ncoef = (size_t)F * dp.N2 * dp.N1;          // member 0's coefficients

    // ---- the reference: FP64 general plan at tol 1e-14 on a sample of member 0
    const int ns = (int)std::min<int64_t>(P0, 4096);
    std::vector<int> sample(ns);
    for (int i = 0; i < ns; ++i) sample[i] = (int)((P0 * (int64_t)i) / ns);
    DevBuf d_idx, d_pts, d_c64, d_ref, d_vals;
    if (!d_idx.alloc(sizeof(int) * ns) || !d_pts.alloc(2 * sizeof(double) * ns) ||
        !d_ref.alloc(sizeof(double) * F * ns) || !d_vals.alloc(rsz * F * (size_t)total))
        return DFSNUFFT_ERR_OOM;
    const void *c64 = a->coeffs;
    if (a->dtype == DFSNUFFT_F32) {
        if (!d_c64.alloc(sizeof(double2) * ncoef)) return DFSNUFFT_ERR_OOM;
        k_widen<<<1024, 256, 0, s>>>((const float2 *)a->coeffs, (double2 *)d_c64.p, ncoef);
        c64 = d_c64.p;
    }
    double *pts = (double *)d_pts.p;
    if (cudaMemcpyAsync(d_idx.p, sample.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s))
        return DFSNUFFT_ERR_CUDA;
    k_gather<<<(ns + 255) / 256, 256, 0, s>>>(a->lon, (const int *)d_idx.p, ns, pts);
    k_gather<<<(ns + 255) / 256, 256, 0, s>>>(a->colat, (const int *)d_idx.p, ns, pts + ns);
    if (cudaGetLastError()) return DFSNUFFT_ERR_CUDA;
    std::vector<double> ref((size_t)F * ns);
    {
        dfsnufft_plan rp = nullptr;
        rc = dfsnufft_plan_create(a->n_lon, a->n_lat, 1e-14, DFSNUFFT_F64, F, s, &rp);
        if (rc) return rc;
        int64_t nsp = ns;
        rc = dfsnufft_set_points_batch(rp, &nsp, pts, pts + ns);
        if (!rc) rc = dfsnufft_execute(rp, c64, d_ref.p);
        if (!rc) rc = dfsnufft_plan_check(rp);
        dfsnufft_destroy(rp);
        if (rc) return rc;
        if (cudaMemcpy(ref.data(), d_ref.p, sizeof(double) * F * ns, cudaMemcpyDeviceToHost))
            return DFSNUFFT_ERR_CUDA;
    }
    double ref_max = 0;
    for (double v : ref) ref_max = fmax(ref_max, fabs(v));
    const double accept = (a->dtype == DFSNUFFT_F64 ? 10.0 : 20.0) * a->tol;
    std::vector<unsigned char> host_vals(rsz * F * (size_t)P0);

    std::vector<dfsnufft_tune_result> all;
    auto run = [&](const dfsnufft_options &o) -> int {
        for (const auto &r : all)
            if (!memcmp(&r.opts, &o, sizeof(o))) return DFSNUFFT_OK;      // already timed
        dfsnufft_tune_result r;
        const int e = run_candidate(a, o, sample, ref, ref_max, d_vals.p, host_vals, &r);
        if (e) return e;
        all.push_back(r);
        return DFSNUFFT_OK;
    };
    auto fastest = [&](bool accepted_only) -> const dfsnufft_tune_result * {
        const dfsnufft_tune_result *b = nullptr;
        for (const auto &r : all) {
            if (r.status || (accepted_only && !(r.err <= accept))) continue;
            if (!b || r.ms < b->ms) b = &r;
        }
        return b;
    };

    // stage 1: bin sizes at the rule's width and oversampling 2
    static const int kx[] = {16, 32, 64, 128};
    static const int ky[] = {8, 16, 32, 64};
    if ((rc = run(base))) return rc;
    for (int tx : kx)
        for (int ty : ky) {
            if (tx * ty < 128 || tx * ty > 4096) continue;
            if (tx > dp.n1 || ty > dp.n2) continue;
            dfsnufft_options o = base;
            o.tile_x = tx;
            o.tile_y = ty;
            if ((rc = run(o))) return rc;
        }
    // stage 2: narrower kernel, oversampling 4, at the best bin
    const dfsnufft_tune_result *b1 = fastest(true);
    dfsnufft_options t = b1 ? b1->opts : base;
    {
        dfsnufft_options o = t;
        o.w = dp.w - 1;
        if (o.w >= 2 && (rc = run(o))) return rc;
        dfsnufft_options ko = t;                    // unsorted points (same values)
        ko.flags |= DFSNUFFT_KEEP_ORDER;
        if ((rc = run(ko))) return rc;
        dfsnufft_params p4;
        dfsnufft_options o4 = t;
        o4.sigma = 4;
        o4.w = 0;
        if (dfsnufft_choose_params_opts(a->n_lon, a->n_lat, a->tol, a->dtype, &o4, &p4) ==
            DFSNUFFT_OK) {
            if ((rc = run(o4))) return rc;
            o4.w = p4.w - 1;
            if (o4.w >= 2 && (rc = run(o4))) return rc;
        }
    }
    const dfsnufft_tune_result *b = fastest(true);
    if (!b) b = fastest(false);
    if (!b) return DFSNUFFT_ERR_UNSUPPORTED;
    *best = b->opts;
    if (results && n_results) {
        const int n = std::min<int>((int)all.size(), std::max(0, max_results));
        for (int i = 0; i < n; ++i) results[i] = all[i];
        *n_results = n;
    }
    return DFSNUFFT_OK;
}

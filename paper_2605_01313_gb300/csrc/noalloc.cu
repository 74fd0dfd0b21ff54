// dfsnufft_execute_noalloc: the set_points + execute pipeline on a static
// device scratch array, for callers that cannot allocate device memory (a model
// step running inside another framework's memory pool, or a latency-critical
// loop that cannot afford cudaMalloc/cudaFree and the synchronisation they
// imply).  The kernels are the library's own; only where their working memory
// comes from differs.
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace {

// Resident on every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DFSNUFFT_NOALLOC_SCRATCH_BYTES];

const int kMaxDevices = 64;
const int kMaxFine = 2048;                       // fine-grid cells per dimension
const double kPi = 3.14159265358979323846264338327950288;

struct DeviceState {
    unsigned char *base;                         // device address of the scratch
    // configuration whose kernel tables are in the scratch now
    int have_tables, n1, n2, N1, N2, w, dtype;
    double beta;
};
DeviceState g_state[kMaxDevices];
std::mutex g_mutex;                              // set-up and table uploads

// Host staging for the tables (static: nothing is allocated per call).
double2 g_tw_stage[2 * kMaxFine];
double g_ft_stage[kMaxFine];
int g_pofs_stage[2];

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// 1 / phihat(k) at the centred modes, phihat(xi) = w int_0^{pi/2}
// e^{beta (cos s - 1)} cos(xi (w/2) sin s) cos s ds by Gauss-Legendre on
// [0, pi/2] (nodes by Newton's method on the Legendre recurrence).
void inverse_kernel_ft(int w, double beta, int n_fine, int n_modes, double *out) {
    const int q = 2 * w + 60;                    // <= 92
    double node[96], weight[96];
    for (int i = 0; i < q; ++i) {
        double z = cos(kPi * (i + 0.75) / (q + 0.5));
        double p0 = 1.0, p1 = z;
        for (int it = 0; it < 100; ++it) {
            p0 = 1.0;
            p1 = z;
            for (int k = 1; k < q; ++k) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            double dz = p1 / (q * (z * p1 - p0) / (z * z - 1.0));
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        p0 = 1.0;
        p1 = z;
        for (int k = 1; k < q; ++k) {
            double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
            p0 = p1;
            p1 = p2;
        }
        double dp = q * (z * p1 - p0) / (z * z - 1.0);
        node[i] = z;
        weight[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    for (int m = 0; m < n_modes; ++m) {
        double xi = 2.0 * kPi * (double)(m - n_modes / 2) / (double)n_fine;
        double acc = 0.0;
        for (int i = 0; i < q; ++i) {
            double s = 0.25 * kPi * (node[i] + 1.0);
            acc += 0.25 * kPi * weight[i] * exp(beta * (cos(s) - 1.0)) * cos(s) *
                   cos(xi * 0.5 * w * sin(s));
        }
        out[m] = 1.0 / (w * acc);
    }
}

// Deconvolution factors in plan precision (FP64 values rounded once for FP32).
cudaError_t upload_factors(const dfsnufft_params &prm, int dtype, int n_fine, int n_modes,
                           void *dst, cudaStream_t st) {
    inverse_kernel_ft(prm.w, prm.beta, n_fine, n_modes, g_ft_stage);
    size_t bytes = sizeof(double) * n_modes;
    if (dtype == DFSNUFFT_F32) {
        float *f = reinterpret_cast<float *>(g_ft_stage);
        for (int i = 0; i < n_modes; ++i) f[i] = (float)g_ft_stage[i];
        bytes = sizeof(float) * n_modes;
    }
    return cudaMemcpyAsync(dst, g_ft_stage, bytes, cudaMemcpyHostToDevice, st);
}

template <typename C, typename R>
cudaError_t upload_twiddles(int n, void *dst, cudaStream_t st) {
    C *h = reinterpret_cast<C *>(g_tw_stage);
    for (int k = 0; k < n; ++k) {
        double a = 2.0 * kPi * (double)k / (double)n;
        h[k].x = (R)cos(a);
        h[k].y = (R)sin(a);
    }
    // pageable source: the call returns once the staging buffer may be reused
    return cudaMemcpyAsync(dst, h, sizeof(C) * n, cudaMemcpyHostToDevice, st);
}

}  // namespace

extern "C" int dfsnufft_execute_noalloc(int n_lon, int n_lat, double tol, int dtype,
                                        int n_fields, int64_t n_points, const double *lon,
                                        const double *colat, const void *coeffs, void *values,
                                        void *stream) {
    if (n_fields < 1 || n_fields > 64 || n_points < 1 || n_points > 0x7fffffffLL || !lon ||
        !colat || !coeffs || !values)
        return DFSNUFFT_ERR_INVALID_ARG;
    dfsnufft_params prm;
    int rc = dfsnufft_choose_params(n_lon, n_lat, tol, dtype, &prm);
    if (rc != DFSNUFFT_OK) return rc;
    if (prm.n1 > kMaxFine || prm.n2 > kMaxFine) return DFSNUFFT_ERR_UNSUPPORTED;

    // the plan-shaped view of the problem, its buffers carved from the scratch
    dfsnufft_plan_s p;
    memset(&p, 0, sizeof(p));
    p.prm = prm;
    p.n_fields = n_fields;
    p.stream = (cudaStream_t)stream;
    p.c0 = (prm.w % 2 == 0) ? prm.w / 2 - 1 : (prm.w - 1) / 2;
    p.nbx = prm.n1 / prm.tile_x;    // base cells lie in [0, n): no wrap bin
    p.nby = prm.n2 / prm.tile_y;
    p.nbins = p.nbx * p.nby;
    p.bstride = (p.nbins + 4) & ~3;
    p.cstride = dfs_cstride(p.bstride);
    p.nch = (p.nbins + DFS_SCAN_CHUNK - 1) / DFS_SCAN_CHUNK;
    p.n_members = 1;
    p.n_points = n_points;
    p.cap_points = n_points;
    p.max_member_points = n_points;
    p.has_points = 1;
    const size_t cs = dtype == DFSNUFFT_F64 ? sizeof(double2) : sizeof(float2);
    const size_t rs = cs / 2;                    // factor tables are in plan precision
    const size_t nf = (size_t)n_fields, P = (size_t)n_points;
    size_t off[20], total = 0;
    const size_t sizes[] = {rs * prm.N1, rs * prm.N2, cs * prm.n1,
                            cs * prm.n2, cs * nf * prm.n2 * prm.N1, rs * nf * prm.n2 * prm.n1,
                            sizeof(int) * p.cstride, sizeof(int) * p.bstride,
                            sizeof(int) * p.bstride, sizeof(int), 2 * sizeof(int),
                            sizeof(int) * P, sizeof(int2) * P, 2 * rs * P, sizeof(int) * P,
                            sizeof(int2)};
    const int nbuf = (int)(sizeof(sizes) / sizeof(sizes[0]));
    for (int i = 0; i < nbuf; ++i) {
        off[i] = total;
        total += align_up(sizes[i]);
    }
    if (total > (size_t)DFSNUFFT_NOALLOC_SCRATCH_BYTES) return DFSNUFFT_ERR_UNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return DFSNUFFT_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState &ds = g_state[dev];
    if (!ds.base) {
        // once per device, with that device current
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return DFSNUFFT_ERR_CUDA;
        ds.base = (unsigned char *)ptr;
    }
    unsigned char *b = ds.base;
    p.d_inv1 = b + off[0];
    p.d_inv2 = b + off[1];
    p.d_tw1 = b + off[2];
    p.d_tw2 = b + off[3];
    p.d_T = b + off[4];
    p.d_G = b + off[5];
    p.d_bin_count = (int *)(b + off[6]);
    p.d_bin_start = (int *)(b + off[7]);
    p.d_task_bin = (int *)(b + off[8]);
    p.d_n_tasks = (int *)(b + off[9]);
    p.d_rank = (int *)(b + off[11]);
    p.d_base = (int2 *)(b + off[12]);
    p.d_frac = b + off[13];
    p.d_idx = (int *)(b + off[14]);
    p.d_pofs = (int *)(b + off[10]);
    p.d_rowrange = (int2 *)(b + off[15]);

    // kernel tables: uploaded only when the configuration differs from the
    // one whose tables the scratch holds (their offsets depend only on it)
    const bool same = ds.have_tables && ds.n1 == prm.n1 && ds.n2 == prm.n2 &&
                      ds.N1 == prm.N1 && ds.N2 == prm.N2 && ds.w == prm.w &&
                      ds.dtype == dtype && ds.beta == prm.beta;
    if (!same) {
        ds.have_tables = 0;
        const bool ok =
            !upload_factors(prm, dtype, prm.n1, prm.N1, p.d_inv1, p.stream) &&
            !upload_factors(prm, dtype, prm.n2, prm.N2, p.d_inv2, p.stream) &&
            (dtype == DFSNUFFT_F64
                 ? !upload_twiddles<double2, double>(prm.n1, p.d_tw1, p.stream) &&
                       !upload_twiddles<double2, double>(prm.n2, p.d_tw2, p.stream)
                 : !upload_twiddles<float2, float>(prm.n1, p.d_tw1, p.stream) &&
                       !upload_twiddles<float2, float>(prm.n2, p.d_tw2, p.stream));
        if (!ok) return DFSNUFFT_ERR_CUDA;
        ds.have_tables = 1;
        ds.n1 = prm.n1;
        ds.n2 = prm.n2;
        ds.N1 = prm.N1;
        ds.N2 = prm.N2;
        ds.w = prm.w;
        ds.dtype = dtype;
        ds.beta = prm.beta;
    }
    // one member: point offsets {0, P}
    g_pofs_stage[0] = 0;
    g_pofs_stage[1] = (int)n_points;
    if (cudaMemcpyAsync(p.d_pofs, g_pofs_stage, sizeof(g_pofs_stage), cudaMemcpyHostToDevice,
                        p.stream) != cudaSuccess)
        return DFSNUFFT_ERR_CUDA;
    // set_points clears the bin counters before counting
    if (dfs_launch_set_points(&p, lon, colat) != cudaSuccess ||
        dfs_launch_theta_pass(&p, coeffs) != cudaSuccess ||
        dfs_launch_phi_pass(&p) != cudaSuccess || dfs_launch_interp(&p, values) != cudaSuccess)
        return DFSNUFFT_ERR_CUDA;
    return DFSNUFFT_OK;
}

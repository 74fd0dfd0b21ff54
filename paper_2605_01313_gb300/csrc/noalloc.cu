// dfsnufft_execute_noalloc: the set_points + execute pipeline on a static
// device scratch array, for callers that cannot allocate device memory (a model
// step running inside another framework's memory pool, or a latency-critical
// loop that cannot afford cudaMalloc/cudaFree and the synchronisation they
// imply).  The kernels are the library's own; only where their working memory
// comes from differs.
//
// Each call writes everything it needs into the scratch from values carried in
// its own kernel arguments: the point offsets, the deconvolution factors
// (computed on the host by dfsnufft_kernel_ft, the plan path's routine, and
// passed by value) and the twiddles (computed on the device).  No host buffer is
// read after the call returns, and nothing depends on what an earlier call left
// in the scratch.
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace {

// Resident on every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DFSNUFFT_NOALLOC_SCRATCH_BYTES];

const int kMaxDevices = 64;
const int kMaxFine = 2048;                       // fine-grid cells per dimension
const int kMaxModes = kMaxFine / 2;              // modes per dimension at sigma 2

// Device address of the scratch, resolved once per device.
unsigned char *g_base[kMaxDevices];
std::mutex g_mutex;

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Per-call tables, by value (about 16 KB of kernel arguments).
struct NoallocTables {
    int N1, N2, n1, n2;
    int n_points;
    int f64;                                     // plan precision of the tables
    double inv[2 * kMaxModes];                   // 1 / phihat: N1 values, then N2
};

// Writes the deconvolution factors (plan precision), the twiddles
// e^{+2 pi i k / n} of both fine lengths and the point offsets {0, P}.
__global__ void __launch_bounds__(256) k_noalloc_tables(const __grid_constant__ NoallocTables t,
                                                        void *__restrict__ inv1,
                                                        void *__restrict__ inv2,
                                                        void *__restrict__ tw1,
                                                        void *__restrict__ tw2,
                                                        int *__restrict__ pofs) {
    const int total = t.N1 + t.N2 + t.n1 + t.n2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < t.N1 + t.N2) {
            void *dst = i < t.N1 ? inv1 : inv2;
            const int k = i < t.N1 ? i : i - t.N1;
            if (t.f64) static_cast<double *>(dst)[k] = t.inv[i];
            else static_cast<float *>(dst)[k] = (float)t.inv[i];
            continue;
        }
        const int j = i - t.N1 - t.N2;
        const int n = j < t.n1 ? t.n1 : t.n2;
        const int k = j < t.n1 ? j : j - t.n1;
        void *dst = j < t.n1 ? tw1 : tw2;
        double sn, cs;
        sincospi(2.0 * (double)k / (double)n, &sn, &cs);     // n a power of two: exact ratio
        if (t.f64) static_cast<double2 *>(dst)[k] = make_double2(cs, sn);
        else static_cast<float2 *>(dst)[k] = make_float2((float)cs, (float)sn);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        pofs[0] = 0;
        pofs[1] = t.n_points;
    }
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
    if (prm.n1 > kMaxFine || prm.n2 > kMaxFine || prm.N1 > kMaxModes || prm.N2 > kMaxModes)
        return DFSNUFFT_ERR_UNSUPPORTED;

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
    p.cstride = dfs_cstride(p.bstride, p.nbins, prm.tile_y);
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
                            (size_t)dfs_fold_rec_bytes(dtype) * P, sizeof(int2) * P, 2 * rs * P,
                            sizeof(int) * P,
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
    unsigned char *b = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_base[dev]) {
            // once per device, with that device current
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) return DFSNUFFT_ERR_CUDA;
            g_base[dev] = (unsigned char *)ptr;
        }
        b = g_base[dev];
    }
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
    p.d_urec = b + off[11];
    p.d_base = (int2 *)(b + off[12]);
    p.d_frac = b + off[13];
    p.d_idx = (int *)(b + off[14]);
    p.d_pofs = (int *)(b + off[10]);
    p.d_rowrange = (int2 *)(b + off[15]);

    // this call's tables, carried by value into the scratch
    NoallocTables t;
    t.N1 = prm.N1;
    t.N2 = prm.N2;
    t.n1 = prm.n1;
    t.n2 = prm.n2;
    t.n_points = (int)n_points;
    t.f64 = dtype == DFSNUFFT_F64 ? 1 : 0;
    if (dfsnufft_kernel_ft(prm.w, prm.beta, prm.n1, prm.N1, t.inv) != DFSNUFFT_OK ||
        dfsnufft_kernel_ft(prm.w, prm.beta, prm.n2, prm.N2, t.inv + prm.N1) != DFSNUFFT_OK)
        return DFSNUFFT_ERR_INVALID_ARG;
    for (int i = 0; i < prm.N1 + prm.N2; ++i) t.inv[i] = 1.0 / t.inv[i];
    const int items = prm.N1 + prm.N2 + prm.n1 + prm.n2;
    k_noalloc_tables<<<(items + 255) / 256, 256, 0, p.stream>>>(t, p.d_inv1, p.d_inv2, p.d_tw1,
                                                              p.d_tw2, p.d_pofs);
    if (cudaGetLastError() != cudaSuccess) return DFSNUFFT_ERR_CUDA;
    // set_points clears the bin counters before counting
    if (dfs_launch_set_points(&p, lon, colat) != cudaSuccess ||
        dfs_launch_theta_pass(&p, coeffs) != cudaSuccess ||
        dfs_launch_phi_pass(&p) != cudaSuccess || dfs_launch_interp(&p, values) != cudaSuccess)
        return DFSNUFFT_ERR_CUDA;
    return DFSNUFFT_OK;
}

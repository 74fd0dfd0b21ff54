// Internal definitions shared by the dfsnufft translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfsnufft.h"

// ---------------------------------------------------------------- dependent launches
// A kernel of the hot path launched by dfs_launch_dependent may start
// launching while the kernel before it in the stream drains (programmatic
// stream serialization): its CTAs are placed as soon as the previous grid's
// CTAs have all exited, without a fresh launch in between.  Such a kernel's
// first statement is dfs_grid_wait(), which returns once the previous grid
// has completed and its writes are visible, so that nothing it reads or writes
// runs ahead of the work it depends on.
__device__ __forceinline__ void dfs_grid_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t dfs_launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// ---------------------------------------------------------------- complex helpers
template <typename R> struct CxT;
template <> struct CxT<float> { typedef float2 type; };
template <> struct CxT<double> { typedef double2 type; };

__host__ __device__ __forceinline__ float2 cmake(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 cmake(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
template <typename C>
__host__ __device__ __forceinline__ C cmul(C a, C b) {
    return cmake(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------- plan layout
// Elements per thread of the FFT kernels (both passes, both precisions).
#define DFS_FFT_E 8
// Row-block granularity of the "fine rows needed" mask (rows per flag).
#define DFS_ROW_BLOCK 16
#define DFS_MAX_ROW_BLOCKS (8192 / DFS_ROW_BLOCK)
// Bin scan: chunks of DFS_SCAN_CHUNK bins (one CTA each), at most
// DFS_SCAN_MAXCH chunks (bins <= (8192/8) x DFS_MAX_ROW_BLOCKS).
#define DFS_SCAN_CHUNK 4096
#define DFS_SCAN_MAXCH 128
#define DFS_FFT_MIN_LOG 4
#define DFS_FFT_MAX_LOG 13
// Event pairs kept per stage before read_timing must drain them.
#define DFS_TIMING_SLOTS 64

struct dfsnufft_plan_s {
    dfsnufft_params prm;
    int n_members;          // members of the same grid, each with its own points
    int n_fields;           // fields per member (lines of the FFT passes: n_members x n_fields)
    int c0;                 // first tap sits c0 cells left of the point's base cell
    int herm;               // DFSNUFFT_REAL_FIELDS: theta pass on columns m >= 0 only
    int keep_order;         // DFSNUFFT_KEEP_ORDER: points processed unsorted, in caller order
    int gdf;                // FP64 plan run in double-single arithmetic (df32.cuh): theta
                            // and phi passes, fine grid as (hi, lo) pairs, interpolation
    void *d_df_tw1, *d_df_tw2;      // double-single twiddles (n1, n2 complex)
    void *d_df_inv1, *d_df_inv2;    // double-single deconvolution factors (N1, N2)
    void *d_df_stw_phi;             // double-single stage-ordered twiddles (length n1/2)
    void *d_df_stw_theta;           // and (length n2) for the theta pass
    void *d_df_stw_half;            // and (length n2/2) for the forward column pass
    int *d_emax;                    // per line: largest coefficient exponent (df32.cuh scaling)
    int nbx, nby, nbins;    // interpolation bins
    int bstride;            // per-member stride of the bin arrays: >= nbins + 1, multiple of 4
    int cstride;            // per-member stride of d_bin_count: bstride + the scan workspace
    int nch;                // bin-scan chunks, ceil(nbins / DFS_SCAN_CHUNK)
    cudaStream_t stream;

    // device buffers owned by the plan
    void *d_inv1;           // N1: 1 / phihat(m), centred, plan precision
    void *d_inv2;           // N2: 1 / phihat(n), centred, plan precision
    void *d_tw1;            // n1 twiddles e^{+2 pi i k / n1} (plan precision)
    void *d_tw2;            // n2 twiddles
    void *d_stw_theta;      // stage-ordered twiddles of the length-n2/2 theta transforms
    void *d_stw_phi;        // stage-ordered twiddles of the length-n1/2 phi transforms
    void *d_T;              // theta-pass output, (members x fields) x n2 x dfs_tpitch columns
    void *d_G;              // fine grids (real part), (members x fields) x n2 x n1, plan precision
    int *d_bin_count;       // members x cstride: counts, then the scan workspace
    int *d_bin_start;       // members x bstride (nbins + 1 used), member-local positions
    int *d_task_bin;        // members x bstride: lists of non-empty bins
    int *d_n_tasks;         // members
    int2 *d_rowrange;           // per member: circular range of needed fine rows (first, count)
    int *d_pofs;                // members + 1 point offsets (device)
    int64_t *h_pofs;            // members + 1 point offsets of the current points (host)
    int64_t max_member_points;  // largest member's point count
    int *d_status;              // device status word (DFS_STATUS_*), zero when healthy
    int *d_work;                // per member: the interpolation's next sub-task and
                                // finished-CTA counters (zero between launches)
    // Gauss-Legendre latitude grid (DFSNUFFT_GAUSS_GRID, gauss.cu)
    int gl;
    void *d_gl_mat;             // C^{-1}, S^{-1} (n_lat x n_lat each, / n_lon), then w
    double *h_gl_colat;         // the n_lat colatitudes
    void *blas;                 // cublasHandle_t (FP64 plans)
    void *d_gl_tc;              // FP32 plans: M_hi, M_lo (2 classes each) of the tcgen05 solve
    CUtensorMap tmap_gl_hi, tmap_gl_lo;
    int *d_parity;              // fields: +1 scalar / -1 wind component (grid input)
    int h_parity[64];           // the parities last uploaded
    int parity_set;
    int num_sms;                // multiprocessors of the plan's device
    CUtensorMap tmap_G;         // 2-D map of d_G (8-byte elements), box set by the interpolation
    int tmap_G_ok;              // tmap_G is valid (FP32 plans that own their buffers)
    int interp_ctas_per_sm;     // resident CTAs of the TMA interpolation (0: not yet known)
    // lines (members x fields) the next theta, phi and interpolation launches
    // cover: [win0, win0 + nwin), every line when nwin == 0 (the host-buffer
    // path of one-member plans pipelines its fields this way)
    int win0, nwin;

    // point data (capacity grows with set_points)
    int64_t n_points, cap_points;   // all members' points
    void *d_urec;           // unsorted folded records (dfs_fold_rec_bytes each): base
                            // cell, rank inside its bin (input order), offsets
    int2 *d_base;           // sorted: first-tap fine index (i0, j0)
    void *d_frac;           // sorted: offsets (tx, ty) in plan precision
    int *d_idx;             // sorted: original point index
    double *d_pts_stage;    // host-variant staging: 2 x cap_points
    void *d_coef_stage;     // host-variant staging of coefficients
    void *d_val_stage;      // host-variant staging of values
    int64_t val_stage_cap;
    int64_t pts_stage_cap;
    // host-variant coefficient copies run on their own stream, so that they
    // overlap the work queued before them (set_points): stage_free is recorded
    // on the plan's stream after each read of d_coef_stage, coef_ready on
    // copy_stream after the copies
    cudaStream_t copy_stream;
    cudaEvent_t stage_free, coef_ready;
    // the per-field pipeline's value copies back to the host: a stream of their
    // own, so that a field's values leave as soon as it is done instead of
    // queueing behind the later fields' coefficient copies
    cudaStream_t back_stream;
    // one-member host-buffer path, pipelined per field: for line f, coefficients
    // staged (line_ev[2 f]) and values ready (line_ev[2 f + 1]); pts_copied marks
    // the end of set_points_host's point copies (pts_pending: not yet waited for)
    cudaEvent_t *line_ev;
    int n_line_ev;
    cudaEvent_t pts_copied, vals_copied;
    int pts_pending;

    // stage timing (dfsnufft_plan_enable_timing)
    int timing;
    cudaEvent_t *ev;            // 2 * DFS_TIMING_SLOTS * DFSNUFFT_N_STAGES events
    int pending[DFSNUFFT_N_STAGES];
    double ms_total[DFSNUFFT_N_STAGES];
    int64_t calls[DFSNUFFT_N_STAGES];

    int has_points;
    int status;             // sticky CUDA status
    char msg[512];
};

// Columns of the theta-pass output: all N1 phi-modes, or for real fields the
// N1/2 + 1 modes m = 0..N1/2 (the rest follow by conjugate symmetry), stored
// with a row pitch rounded up to 4 elements.
__host__ __device__ __forceinline__ int dfs_tcols(int herm, int N1) { return herm ? N1 / 2 + 1 : N1; }
__host__ __device__ __forceinline__ int dfs_tpitch(int herm, int N1) {
    return herm ? ((N1 / 2 + 1 + 3) & ~3) : N1;
}

// Bytes of one unsorted point record of set_points (points.cu FoldRec): packed
// base cell and rank (two ints) and the two offsets in plan precision.
__host__ __device__ __forceinline__ int dfs_fold_rec_bytes(int dtype) {
    return dtype == DFSNUFFT_F64 ? 24 : 16;
}

// Ints per member of the count array: counts (bstride), completion counter (4),
// bin-row flags (DFS_MAX_ROW_BLOCKS bytes), chunk sums and non-empty counts,
// then from dfs_rowcount_offset the per-row counts of every bin (nbins x
// tile_y, bin-major), which order the points inside a bin by fine row.
__host__ __device__ __forceinline__ int dfs_rowcount_offset(int bstride) {
    return bstride + 4 + DFS_MAX_ROW_BLOCKS / 4 + 2 * DFS_SCAN_MAXCH;
}
__host__ __device__ __forceinline__ int dfs_cstride(int bstride, int nbins, int tile_y) {
    return dfs_rowcount_offset(bstride) + ((nbins * tile_y + 3) & ~3);
}

// The line window of the next launches: first line and count.
__host__ __forceinline__ void dfs_lines(const dfsnufft_plan_s *p, int &line0, int &nlines) {
    line0 = p->nwin ? p->win0 : 0;
    nlines = p->nwin ? p->nwin : p->n_members * p->n_fields;
}

// ---------------------------------------------------------------- launches
// points.cu
cudaError_t dfs_launch_set_points(dfsnufft_plan p, const double *lon, const double *colat);
// fft.cu
// prM >= 0: coeffs holds partial-regularity coefficients truncated at (prM, prN)
cudaError_t dfs_launch_theta_pass(dfsnufft_plan p, const void *coeffs, int prM = -1,
                                  int prN = -1);
cudaError_t dfs_launch_phi_pass(dfsnufft_plan p);
// Largest FP64 exponent of each of lines line0 .. line0 + lines - 1 into
// p->d_emax (the double-single scaling of df32.cuh): every one of the
// line_elems complex values of a line, or (herm) those a real-field theta pass
// reads of a rows x N1 array.
cudaError_t dfs_launch_line_maxexp(dfsnufft_plan p, const void *data, int line_elems, int rows,
                                   int herm, int line0, int lines);
// interp.cu
cudaError_t dfs_launch_interp(dfsnufft_plan p, void *values);
// forward.cu
bool dfs_forward_supported(const dfsnufft_params &q);
// gauss.cu
int dfs_gl_setup(dfsnufft_plan p);
void dfs_gl_release(dfsnufft_plan p);
int dfs_launch_forward_gl(dfsnufft_plan p, const void *samples, const int *d_parity,
                          void *coeffs, bool full);
size_t dfs_gl_scratch_bytes(const dfsnufft_params &q, int lines);
// gl_gemm.cu: the FP32 latitude solve on the tensor cores
int dfs_gl_tc_setup(dfsnufft_plan p, const double *cm, const double *sm, int N);
cudaError_t dfs_gl_tc_gemm(dfsnufft_plan p, const float *g, float *out, int N, int cols);
// full = false: of the columns m < 0 only the Nyquist row n = -N2/2 is written
// (all that a real-field plan's theta pass reads there)
cudaError_t dfs_launch_forward(dfsnufft_plan p, const void *samples, const int *d_parity,
                               void *coeffs, bool full);

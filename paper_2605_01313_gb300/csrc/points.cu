// set_points: fold the departure points onto the fine-grid torus (FP64), sort
// them by interpolation bin with a counting sort, and mark the fine rows their
// stencils touch.
//
// Every point gets, in FP64, its fine-grid coordinates x = phi n1 / 2pi and
// y = theta n2 / 2pi wrapped to [0, n) (the doubled torus is 2pi-periodic in
// both angles, Sec. 4-5), an integer base cell b and an offset t = x - b:
//   even w: b = floor(x),       t in [0, 1)
//   odd  w: b = floor(x + 1/2), t in [-1/2, 1/2)
// The w taps sit at cells b - c0 .. b - c0 + w - 1 (c0 = w/2 - 1 or (w-1)/2),
// at kernel arguments z_a = (a - c0) - t, all inside [-w/2, w/2].  Only the
// small offset t leaves this file in plan precision, so the FP32 form keeps
// its kernel arguments accurate to ~3e-8 cells whatever the grid size.
#include "common.cuh"

namespace {

struct FoldParams {
    double sx, sy;      // n / (2 pi)
    int n1, n2;
    int odd_w;
    int c0, w;
    int tile_x, tile_y, nbx;
    int n_row_blocks;
};

__device__ __forceinline__ double wrap(double v, int n) {
    double dn = (double)n;
    double t = v - dn * floor(v / dn);
    if (t >= dn) t -= dn;
    if (t < 0.0) t += dn;
    return t;
}

// A non-finite coordinate is placed at cell 0 with a NaN offset: its stencil
// stays inside the grid and its value comes out NaN.
__device__ __forceinline__ void fold_point(const FoldParams &f, double lon, double colat,
                                           int &bx, int &by, double &tx, double &ty) {
    double x = wrap(lon * f.sx, f.n1);
    double y = wrap(colat * f.sy, f.n2);
    bool ok = (x >= 0.0 && x < (double)f.n1) && (y >= 0.0 && y < (double)f.n2);
    if (!ok) {
        x = 0.0;
        y = 0.0;
    }
    double fx = f.odd_w ? floor(x + 0.5) : floor(x);
    double fy = f.odd_w ? floor(y + 0.5) : floor(y);
    bx = (int)fx;
    by = (int)fy;
    tx = ok ? x - fx : __longlong_as_double(0x7ff8000000000000LL);
    ty = ok ? y - fy : tx;
}

__device__ __forceinline__ int bin_of(const FoldParams &f, int bx, int by) {
    return (by / f.tile_y) * f.nbx + bx / f.tile_x;
}

__global__ void k_fold_count(int n, const double *__restrict__ lon,
                             const double *__restrict__ colat, FoldParams f,
                             int *__restrict__ bin_count, int *__restrict__ rank,
                             unsigned char *__restrict__ rowmask) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool live = p < n;
    int bin = -1;
    int j0 = 0;
    if (live) {
        int bx, by;
        double tx, ty;
        fold_point(f, lon[p], colat[p], bx, by, tx, ty);
        bin = bin_of(f, bx, by);
        j0 = by - f.c0;
    }
    // warp-aggregated increment: lanes sharing a bin take consecutive ranks
    unsigned live_mask = __ballot_sync(0xffffffffu, live);
    if (!live) return;
    unsigned peers = __match_any_sync(live_mask, bin);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&bin_count[bin], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    rank[p] = base + __popc(peers & ((1u << lane) - 1u));
    // fine rows j0 .. j0 + w - 1 (mod n2) span at most two row blocks (w <= 16)
    int r_lo = j0 & (f.n2 - 1);
    int r_hi = (j0 + f.w - 1) & (f.n2 - 1);
    rowmask[r_lo / DFS_ROW_BLOCK] = 1;
    rowmask[r_hi / DFS_ROW_BLOCK] = 1;
}

// One CTA: exclusive scan of the bin counts and the list of non-empty bins.
__global__ void __launch_bounds__(1024) k_scan_bins(int nbins, const int *__restrict__ count,
                                                    int *__restrict__ start,
                                                    int *__restrict__ task_bin,
                                                    int *__restrict__ n_tasks) {
    __shared__ int s_cnt[32], s_ne[32];
    const int tid = threadIdx.x;
    const int per = (nbins + blockDim.x - 1) / blockDim.x;
    const int lo = tid * per;
    const int hi = min(lo + per, nbins);
    int sum = 0, ne = 0;
    for (int i = lo; i < hi; ++i) {
        int c = count[i];
        sum += c;
        ne += c > 0;
    }
    // block-wide exclusive scan of (sum, ne)
    int lane = tid & 31, wid = tid >> 5;
    int xs = sum, xn = ne;
    for (int o = 1; o < 32; o <<= 1) {
        int ys = __shfl_up_sync(0xffffffffu, xs, o);
        int yn = __shfl_up_sync(0xffffffffu, xn, o);
        if (lane >= o) {
            xs += ys;
            xn += yn;
        }
    }
    if (lane == 31) {
        s_cnt[wid] = xs;
        s_ne[wid] = xn;
    }
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int vs = lane < nw ? s_cnt[lane] : 0;
        int vn = lane < nw ? s_ne[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int ys = __shfl_up_sync(0xffffffffu, vs, o);
            int yn = __shfl_up_sync(0xffffffffu, vn, o);
            if (lane >= o) {
                vs += ys;
                vn += yn;
            }
        }
        if (lane < nw) {
            s_cnt[lane] = vs;
            s_ne[lane] = vn;
        }
    }
    __syncthreads();
    int off_s = xs - sum + (wid > 0 ? s_cnt[wid - 1] : 0);
    int off_n = xn - ne + (wid > 0 ? s_ne[wid - 1] : 0);
    for (int i = lo; i < hi; ++i) {
        int c = count[i];
        start[i] = off_s;
        off_s += c;
        if (c > 0) task_bin[off_n++] = i;
    }
    if (tid == blockDim.x - 1) {
        start[nbins] = off_s;
        *n_tasks = off_n;
    }
}

template <typename R>
__global__ void k_scatter(int n, const double *__restrict__ lon, const double *__restrict__ colat,
                          FoldParams f, const int *__restrict__ start,
                          const int *__restrict__ rank, int2 *__restrict__ base,
                          R *__restrict__ frac, int *__restrict__ idx) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int bx, by;
    double tx, ty;
    fold_point(f, lon[p], colat[p], bx, by, tx, ty);
    int pos = start[bin_of(f, bx, by)] + rank[p];
    base[pos] = make_int2(bx - f.c0, by - f.c0);
    frac[2 * pos] = (R)tx;
    frac[2 * pos + 1] = (R)ty;
    idx[pos] = p;
}

}  // namespace

cudaError_t dfs_launch_set_points(dfsnufft_plan p, const double *lon, const double *colat) {
    const dfsnufft_params &q = p->prm;
    const double two_pi = 6.283185307179586476925286766559;
    FoldParams f;
    f.sx = (double)q.n1 / two_pi;
    f.sy = (double)q.n2 / two_pi;
    f.n1 = q.n1;
    f.n2 = q.n2;
    f.odd_w = q.w & 1;
    f.c0 = p->c0;
    f.w = q.w;
    f.tile_x = q.tile_x;
    f.tile_y = q.tile_y;
    f.nbx = p->nbx;
    f.n_row_blocks = p->n_row_blocks;
    int n = (int)p->n_points;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->d_bin_count, 0, sizeof(int) * p->nbins, p->stream))) return e;
    if ((e = cudaMemsetAsync(p->d_rowmask, 0, p->n_row_blocks, p->stream))) return e;
    const int tpb = 256;
    int blocks = (n + tpb - 1) / tpb;
    k_fold_count<<<blocks, tpb, 0, p->stream>>>(n, lon, colat, f, p->d_bin_count, p->d_rank,
                                               p->d_rowmask);
    k_scan_bins<<<1, 1024, 0, p->stream>>>(p->nbins, p->d_bin_count, p->d_bin_start,
                                          p->d_task_bin, p->d_n_tasks);
    if (q.dtype == DFSNUFFT_F64)
        k_scatter<double><<<blocks, tpb, 0, p->stream>>>(n, lon, colat, f, p->d_bin_start,
                                                        p->d_rank, p->d_base,
                                                        (double *)p->d_frac, p->d_idx);
    else
        k_scatter<float><<<blocks, tpb, 0, p->stream>>>(n, lon, colat, f, p->d_bin_start,
                                                       p->d_rank, p->d_base, (float *)p->d_frac,
                                                       p->d_idx);
    return cudaGetLastError();
}

// set_points: fold the departure points onto the fine-grid torus, sort them by
// interpolation bin with a counting sort, and find the range of fine rows their
// stencils touch.
//
// The doubled torus is 2 pi periodic in both angles (Sec. 4-5), so a coordinate
// only matters as a fraction of a turn.  That fraction is computed exactly in
// integer arithmetic from the FP64 bit pattern: Y = floor(v / (2 pi) 2^64)
// mod 2^64 (Q0.64 turns), from the 53-bit significand times 1/(2 pi) held to
// 128 bits.  GB300 runs FP64 at a small fraction of its integer rate, and the
// fixed-point result is also more accurate (one unit in 2^-64 turns) than an
// FP64 product would be.  For a fine grid of n = 2^L cells the point sits at
// x = Y / 2^(64-L) cells; it gets an integer base cell b and an offset t = x - b:
//   even w: b = floor(x),       t in [0, 1)
//   odd  w: b = floor(x + 1/2), t in [-1/2, 1/2)
// The w taps sit at cells b - c0 .. b - c0 + w - 1 (c0 = w/2 - 1 or (w-1)/2),
// at kernel arguments z_a = (a - c0) - t, all inside [-w/2, w/2].  Only the
// offset t leaves this file in plan precision (FP32 or FP64), so the FP32 form
// keeps its kernel arguments accurate to ~1e-9 cells at any grid size.
#include "common.cuh"
#include "turns.cuh"

namespace {

struct FoldParams {
    int L1, L2;         // log2 of the fine sizes
    int odd_w;
    int c0, w;
    int ltx, lty, nbx;  // log2 of the bin size (powers of two), bins per bin row
};

// Base cell and offset of one coordinate on a fine grid of 2^L cells.  tq is the
// offset t in units of 2^-64 cells (signed for odd w).
__device__ __forceinline__ void split_cell(unsigned long long Y, int L, int odd_w, int &b,
                                           long long &tq) {
    if (odd_w) {
        const unsigned long long yr = Y + (1ULL << (63 - L));
        b = (int)(yr >> (64 - L));
        tq = (long long)((yr << L) ^ (1ULL << 63));
    } else {
        b = (int)(Y >> (64 - L));
        tq = (long long)(Y << L);           // unsigned fraction, read back as such
    }
}

template <typename R> __device__ __forceinline__ R offset_value(long long tq, int odd_w);
template <> __device__ __forceinline__ float offset_value<float>(long long tq, int odd_w) {
    return odd_w ? (float)(int)(tq >> 32) * 0x1p-32f
                 : (float)(unsigned)((unsigned long long)tq >> 32) * 0x1p-32f;
}
template <> __device__ __forceinline__ double offset_value<double>(long long tq, int odd_w) {
    return odd_w ? (double)(tq >> 11) * 0x1p-53
                 : (double)(long long)((unsigned long long)tq >> 11) * 0x1p-53;
}

// A coordinate that cannot be folded (non-finite, or beyond 2^53 rad) is placed
// at cell 0; its offset becomes NaN so that its value comes out NaN.
__device__ __forceinline__ bool fold_point(const FoldParams &f, double lon, double colat,
                                           int &bx, int &by, long long &tx, long long &ty) {
    unsigned long long yx = 0, yy = 0;
    const bool ok = turns_q64(lon, yx) & turns_q64(colat, yy);
    split_cell(ok ? yx : 0ULL, f.L1, f.odd_w, bx, tx);
    split_cell(ok ? yy : 0ULL, f.L2, f.odd_w, by, ty);
    return ok;
}

__device__ __forceinline__ int bin_of(const FoldParams &f, int bx, int by) {
    return (by >> f.lty) * f.nbx + (bx >> f.ltx);
}

// Unsorted record of a folded point, written by k_fold_count and moved to its
// sorted place by k_scatter: base cell (bx | by << 16, both below 2^13), the
// point's rank inside its bin (input order) and its offsets in plan precision.
// 16 bytes in FP32 (one vector store and load), 24 in FP64.
template <typename R> struct FoldRec;
template <> struct __align__(16) FoldRec<float> {
    int base, rank;
    float tx, ty;
};
template <> struct __align__(8) FoldRec<double> {
    int base, rank;
    double tx, ty;
};
static_assert(sizeof(FoldRec<float>) == 16 && sizeof(FoldRec<double>) == 24,
              "record sizes of dfs_fold_rec_bytes");

// Sort key of a point: its bin, then its base cell's row inside the bin (the
// rank within a bin follows fine rows, so that the points of one warp share
// stencil rows and read consecutive shared-memory words).
__device__ __forceinline__ int rowkey_of(const FoldParams &f, int bx, int by) {
    return (bin_of(f, bx, by) << f.lty) | (by & ((1 << f.lty) - 1));
}

// grid (ceil(max member points / 256), members): member k = blockIdx.y.  Folds
// every point once (kept in its unsorted record) and counts the points of each
// row of each bin (the row counts at rowoff in the member's count slice); the
// rank of a point is its position among its row's points, in input order.
template <typename R>
__global__ void __launch_bounds__(256) k_fold_count(const double *__restrict__ lon,
                                                    const double *__restrict__ colat,
                                                    FoldParams f, const int *__restrict__ pofs,
                                                    int cstride, int rowoff,
                                                    int *__restrict__ bin_count,
                                                    FoldRec<R> *__restrict__ urec) {
    const int k = blockIdx.y;
    const int p0 = pofs[k];
    const int pl = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = pl < pofs[k + 1] - p0;
    int bin = -1;                               // the row key
    FoldRec<R> rec;
    if (live) {
        int bx, by;
        long long tx, ty;
        const bool ok = fold_point(f, lon[p0 + pl], colat[p0 + pl], bx, by, tx, ty);
        bin = rowkey_of(f, bx, by);
        rec.base = bx | (by << 16);
        rec.tx = offset_value<R>(tx, f.odd_w);
        rec.ty = offset_value<R>(ty, f.odd_w);
        if (!ok) rec.tx = rec.ty = (R)__int_as_float(0x7fc00000);
    }
    // warp aggregation over runs of equal bins (points arrive nearly sorted):
    // the first lane of each run takes the run's ranks with one atomicAdd
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, bin, 1);
    const bool head = live && (lane == 0 || prev != bin);
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned live_mask = __ballot_sync(0xffffffffu, live);
    // this lane's run: from its head to the lane before the next head (or the
    // last live lane)
    const int my_head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    const unsigned later = heads & ~(0xffffffffu >> (31 - lane));   // heads after this lane
    const int run_end = later ? __ffs(later) - 1 : 32 - __clz(live_mask);
    int base = 0;
    if (head) base = atomicAdd(&bin_count[(size_t)k * cstride + rowoff + bin], run_end - lane);
    base = __shfl_sync(0xffffffffu, base, my_head);
    if (live) {
        rec.rank = base + lane - my_head;
        urec[p0 + pl] = rec;
    }
}

// grid (ceil(nbins / 256), members): for each bin, the exclusive prefix of its
// row counts (in place: the offset of each row inside the bin) and the bin's
// total, which the bin scan takes.
__global__ void __launch_bounds__(256) k_row_prefix(int nbins, int tile_y, int cstride,
                                                    int rowoff, int *__restrict__ count_all) {
    dfs_grid_wait();
    const int bin = blockIdx.x * blockDim.x + threadIdx.x;
    if (bin >= nbins) return;
    int *slice = count_all + (size_t)blockIdx.y * cstride;
    int *rc = slice + rowoff + (size_t)bin * tile_y;
    int sum = 0;
    if ((tile_y & 3) == 0 && tile_y <= 32 && (reinterpret_cast<uintptr_t>(rc) & 15) == 0) {
        // all of the bin's row counts in flight at once (16-byte loads), then
        // the offsets stored over them
        const int nq = tile_y >> 2;
        int4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < nq) v[q] = reinterpret_cast<const int4 *>(rc)[q];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < nq) {
                int4 o;
                o.x = sum;
                o.y = o.x + v[q].x;
                o.z = o.y + v[q].y;
                o.w = o.z + v[q].z;
                sum = o.w + v[q].w;
                reinterpret_cast<int4 *>(rc)[q] = o;
            }
        slice[bin] = sum;
        return;
    }
    for (int r = 0; r < tile_y; ++r) {
        const int c = rc[r];
        rc[r] = sum;
        sum += c;
    }
    slice[bin] = sum;
}

// Smallest index i in [from, from + nb) (circular over nb bits) whose bit in
// `bits` equals `value`; from + nb if there is none.
__device__ int next_bit(const unsigned *bits, int nb, int from, int value) {
    int i = from;
    const int end = from + nb;
    while (i < end) {
        const int k = i < nb ? i : i - nb;
        unsigned w = bits[k >> 5];
        if (!value) w = ~w;
        w >>= (k & 31);
        // bits past nb in the last word do not count
        const int avail = min(32 - (k & 31), nb - k);
        if (avail < 32) w &= (1u << avail) - 1u;
        if (w) {
            const int hit = i + __ffs(w) - 1;
            return hit < end ? hit : end;
        }
        i += avail;
    }
    return end;
}

struct ScanParams {
    int nbins, nbx, nbr;      // bins, bins per bin row, bin rows in use (n2 / tile_y)
    int bstride;              // per-member stride of the start and task arrays (multiple of 4)
    int cstride;              // per-member stride of the count slice (counts + scan workspace)
    int nch;                  // chunks of DFS_SCAN_CHUNK bins
    int tile_y, c0, w, n2;
};

// Layout of a member's count slice (cstride ints, zeroed before each
// set_points): counts [0, bstride), then the scan workspace: a completion
// counter, the bin-row flags (bytes) and the chunk sums and non-empty counts.
__device__ __forceinline__ int *ws_done(int *slice, const ScanParams &sp) { return slice + sp.bstride; }
__device__ __forceinline__ unsigned char *ws_rows(int *slice, const ScanParams &sp) {
    return reinterpret_cast<unsigned char *>(slice + sp.bstride + 4);
}
__device__ __forceinline__ int *ws_sum(int *slice, const ScanParams &sp) {
    return slice + sp.bstride + 4 + DFS_MAX_ROW_BLOCKS / 4;
}
__device__ __forceinline__ int *ws_ne(int *slice, const ScanParams &sp) {
    return ws_sum(slice, sp) + DFS_SCAN_MAXCH;
}

// Counts of bins [i0, i0 + 16) (zero past nbins); all loads issued first.
__device__ __forceinline__ void load16(const int *count, int i0, int nbins, int *c) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + 4 * u;
        if (i + 3 < nbins) {
            const int4 v = *reinterpret_cast<const int4 *>(count + i);
            c[4 * u] = v.x;
            c[4 * u + 1] = v.y;
            c[4 * u + 2] = v.z;
            c[4 * u + 3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) c[4 * u + q] = i + q < nbins ? count[i + q] : 0;
        }
    }
}

// Exclusive block-wide scan of (a, b) over the CTA's threads; returns the
// thread's prefixes and the totals.  blockDim.x <= 1024.
__device__ __forceinline__ void block_scan2(int a, int b, int &pa, int &pb, int &ta, int &tb) {
    __shared__ int s_a[32], s_b[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int xa = a, xb = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ya = __shfl_up_sync(0xffffffffu, xa, o);
        const int yb = __shfl_up_sync(0xffffffffu, xb, o);
        if (lane >= o) {
            xa += ya;
            xb += yb;
        }
    }
    if (lane == 31) {
        s_a[wid] = xa;
        s_b[wid] = xb;
    }
    __syncthreads();
    if (wid == 0) {
        int va = lane < nw ? s_a[lane] : 0;
        int vb = lane < nw ? s_b[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ya = __shfl_up_sync(0xffffffffu, va, o);
            const int yb = __shfl_up_sync(0xffffffffu, vb, o);
            if (lane >= o) {
                va += ya;
                vb += yb;
            }
        }
        if (lane < nw) {
            s_a[lane] = va;
            s_b[lane] = vb;
        }
    }
    __syncthreads();
    pa = xa - a + (wid > 0 ? s_a[wid - 1] : 0);
    pb = xb - b + (wid > 0 ? s_b[wid - 1] : 0);
    ta = s_a[nw - 1];
    tb = s_b[nw - 1];
    __syncthreads();
}

// Run by every thread of the last CTA of a member once all its bin-row flags
// are published: the circular range of fine rows the stencils touch.  The
// points of bin row by use rows by*tile_y - c0 .. (by+1)*tile_y - c0 + w - 2,
// so the range is the complement of the longest circular run of empty bin
// rows, widened by the stencil and rounded out to whole row blocks.
__device__ void finish_rowrange(const ScanParams &sp, const unsigned char *rows,
                                unsigned *s_bits, int2 *range_out) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int k = wid; k * 32 < sp.nbr; k += nw) {
        const int i = k * 32 + lane;
        const unsigned b = __ballot_sync(0xffffffffu, i < sp.nbr && __ldcg(rows + i) != 0);
        if (lane == 0) s_bits[k] = b;
    }
    __syncthreads();
    if (tid == 0) {
        const int nb = sp.nbr;
        const int s0 = next_bit(s_bits, nb, 0, 1);
        int2 range = make_int2(0, 0);
        if (s0 < nb) {
            int best = 0, best_at = 0;
            int pos = s0;
            while (pos < s0 + nb) {
                const int z0 = next_bit(s_bits, nb, pos >= nb ? pos - nb : pos, 0) +
                               (pos >= nb ? nb : 0);
                if (z0 >= s0 + nb) break;
                const int z1 = next_bit(s_bits, nb, z0 >= nb ? z0 - nb : z0, 1) +
                               (z0 >= nb ? nb : 0);
                const int end = z1 < s0 + nb ? z1 : s0 + nb;
                if (end - z0 > best) {
                    best = end - z0;
                    best_at = z0;
                }
                pos = end;
            }
            // needed rows: after the gap, through the last non-empty bin row's stencil
            int first = ((best_at + best) % nb) * sp.tile_y - sp.c0;
            int cnt = (nb - best) * sp.tile_y + sp.w - 1;
            first &= sp.n2 - 1;
            const int fb = first & ~(DFS_ROW_BLOCK - 1);
            cnt = ((cnt + (first - fb) + DFS_ROW_BLOCK - 1) / DFS_ROW_BLOCK) * DFS_ROW_BLOCK;
            range = make_int2(fb, cnt < sp.n2 ? cnt : sp.n2);
        }
        *range_out = range;
    }
}

// Pass 1 of the bin scan.  grid (nch, members), DFS_SCAN_CHUNK / 16 threads:
// sum and number of non-empty bins of each chunk of DFS_SCAN_CHUNK bins.
__global__ void __launch_bounds__(DFS_SCAN_CHUNK / 16) k_scan_sums(ScanParams sp,
                                                                   int *__restrict__ count_all) {
    dfs_grid_wait();
    int *slice = count_all + (size_t)blockIdx.y * sp.cstride;
    int c[16];
    load16(slice, blockIdx.x * DFS_SCAN_CHUNK + 16 * threadIdx.x, sp.nbins, c);
    int sum = 0, ne = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        sum += c[q];
        ne += c[q] > 0;
    }
    int pa, pb, ta, tb;
    block_scan2(sum, ne, pa, pb, ta, tb);
    if (threadIdx.x == 0) {
        ws_sum(slice, sp)[blockIdx.x] = ta;
        ws_ne(slice, sp)[blockIdx.x] = tb;
    }
}

// Pass 2.  grid (nch, members): the chunk's offset from the sums of the chunks
// before it, then each thread's sixteen bins: exclusive start offsets, the
// list of non-empty bins (in bin order) and the bin-row flags.  The last CTA
// of a member to finish (completion counter; the CTAs publish their flags with
// a fence before counting) finds the circular range of fine rows the stencils
// touch: the points of bin row by use rows by*tile_y - c0 .. (by+1)*tile_y -
// c0 + w - 2, so the range is the complement of the longest circular run of
// empty bin rows, widened by the stencil and rounded out to whole row blocks.
__global__ void __launch_bounds__(DFS_SCAN_CHUNK / 16) k_scan_write(ScanParams sp,
                                                                    int *__restrict__ count_all,
                                                                    int *__restrict__ start_all,
                                                                    int *__restrict__ task_all,
                                                                    int *__restrict__ n_tasks,
                                                                    int2 *__restrict__ rowrange) {
    dfs_grid_wait();
    const int member = blockIdx.y, chunk = blockIdx.x;
    int *slice = count_all + (size_t)member * sp.cstride;
    int *start = start_all + (size_t)member * sp.bstride;
    int *task_bin = task_all + (size_t)member * sp.bstride;
    unsigned char *rows = ws_rows(slice, sp);
    __shared__ unsigned char s_row[DFS_SCAN_CHUNK];
    __shared__ unsigned s_bits[(DFS_MAX_ROW_BLOCKS + 31) / 32];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int nbins = sp.nbins;
    const int first_bin = chunk * DFS_SCAN_CHUNK;
    const int row_lo = first_bin / sp.nbx;                 // bin rows this chunk can touch
    const int nrow = min(DFS_SCAN_CHUNK, (min(first_bin + DFS_SCAN_CHUNK, nbins) - 1) / sp.nbx -
                                             row_lo + 1);
    for (int i = tid; i < nrow; i += blockDim.x) s_row[i] = 0;
    int c[16];
    const int i0 = first_bin + 16 * tid;
    load16(slice, i0, nbins, c);
    // offsets of this chunk: the sums of the chunks before it
    int cs = 0, cn = 0;
    if (tid < chunk) {
        cs = ws_sum(slice, sp)[tid];
        cn = ws_ne(slice, sp)[tid];
    }
    int sum = 0, ne = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        sum += c[q];
        ne += c[q] > 0;
    }
    int pa, pb, base_s, base_n;
    block_scan2(cs, cn, pa, pb, base_s, base_n);
    int ps, pn, ts, tn;
    block_scan2(sum, ne, ps, pn, ts, tn);
    int off_s = base_s + ps, off_n = base_n + pn;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + 4 * u;
        int st[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            st[q] = off_s;
            off_s += c[4 * u + q];
            if (c[4 * u + q] > 0 && i + q < nbins) {
                task_bin[off_n++] = i + q;
                s_row[(i + q) / sp.nbx - row_lo] = 1;
            }
        }
        if (i + 3 < nbins) {
            *reinterpret_cast<int4 *>(start + i) = make_int4(st[0], st[1], st[2], st[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i + q < nbins) start[i + q] = st[q];
        }
    }
    if (chunk == sp.nch - 1 && tid == 0) {
        start[nbins] = base_s + ts;
        n_tasks[member] = base_n + tn;
    }
    __syncthreads();
    for (int i = tid; i < nrow; i += blockDim.x)
        if (s_row[i]) rows[row_lo + i] = 1;
    // publish the flags, then count this CTA done
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(ws_done(slice, sp), 1) == sp.nch - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last CTA of the member: bin-row flags -> needed row range
    finish_rowrange(sp, rows, s_bits, rowrange + member);
}

// Points kept in the caller's order (DFSNUFFT_KEEP_ORDER): fold every point to
// its record at its own index, flag the bin rows it touches, and let the last
// CTA of the member find the needed row range.  grid (ceil(max member points /
// 256), members).
template <typename R>
__global__ void __launch_bounds__(256) k_fold_direct(const double *__restrict__ lon,
                                                     const double *__restrict__ colat,
                                                     FoldParams f, ScanParams sp,
                                                     const int *__restrict__ pofs,
                                                     int *__restrict__ count_all,
                                                     int2 *__restrict__ base,
                                                     R *__restrict__ frac,
                                                     int2 *__restrict__ rowrange) {
    __shared__ unsigned char s_row[DFS_MAX_ROW_BLOCKS];
    __shared__ unsigned s_bits[(DFS_MAX_ROW_BLOCKS + 31) / 32];
    __shared__ int s_last;
    const int k = blockIdx.y;
    const int p0 = pofs[k];
    const int pl = blockIdx.x * blockDim.x + threadIdx.x;
    int *slice = count_all + (size_t)k * sp.cstride;
    unsigned char *rows = ws_rows(slice, sp);
    for (int i = threadIdx.x; i < sp.nbr; i += blockDim.x) s_row[i] = 0;
    __syncthreads();
    if (pl < pofs[k + 1] - p0) {
        int bx, by;
        long long tx, ty;
        const bool ok = fold_point(f, lon[p0 + pl], colat[p0 + pl], bx, by, tx, ty);
        base[p0 + pl] = make_int2(bx - f.c0, by - f.c0);
        R ox = offset_value<R>(tx, f.odd_w), oy = offset_value<R>(ty, f.odd_w);
        if (!ok) ox = oy = (R)__int_as_float(0x7fc00000);
        frac[2 * (size_t)(p0 + pl)] = ox;
        frac[2 * (size_t)(p0 + pl) + 1] = oy;
        s_row[by >> f.lty] = 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < sp.nbr; i += blockDim.x)
        if (s_row[i]) rows[i] = 1;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ws_done(slice, sp), 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    finish_rowrange(sp, rows, s_bits, rowrange + k);
}

// grid (ceil(max member points / 256), members): member k = blockIdx.y.  Each
// point's unsorted record goes to its sorted place in the member's slice
// [pofs[k], pofs[k+1]): bin start plus rank.  idx holds member-local point
// indices.
template <typename R>
__global__ void __launch_bounds__(256) k_scatter(const FoldRec<R> *__restrict__ urec,
                                                 FoldParams f, const int *__restrict__ pofs,
                                                 int bstride, const int *__restrict__ start_all,
                                                 int cstride, int rowoff,
                                                 const int *__restrict__ count_all,
                                                 int2 *__restrict__ base,
                                                 typename CxT<R>::type *__restrict__ frac,
                                                 int *__restrict__ idx) {
    dfs_grid_wait();
    const int k = blockIdx.y;
    const int p0 = pofs[k];
    const int pl = blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= pofs[k + 1] - p0) return;
    const FoldRec<R> rec = urec[p0 + pl];
    const int bx = rec.base & 0xffff, by = rec.base >> 16;
    const int pos = p0 + start_all[(size_t)k * bstride + bin_of(f, bx, by)] +
                    count_all[(size_t)k * cstride + rowoff + rowkey_of(f, bx, by)] + rec.rank;
    base[pos] = make_int2(bx - f.c0, by - f.c0);
    frac[pos] = cmake(rec.tx, rec.ty);
    idx[pos] = pl;
}

int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace

cudaError_t dfs_launch_set_points(dfsnufft_plan p, const double *lon, const double *colat) {
    const dfsnufft_params &q = p->prm;
    FoldParams f;
    f.L1 = ilog2(q.n1);
    f.L2 = ilog2(q.n2);
    f.odd_w = q.w & 1;
    f.c0 = p->c0;
    f.w = q.w;
    f.ltx = ilog2(q.tile_x);
    f.lty = ilog2(q.tile_y);
    f.nbx = p->nbx;
    const int M = p->n_members;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->d_bin_count, 0, sizeof(int) * (size_t)M * p->cstride, p->stream)))
        return e;
    const int tpb = 256;
    const dim3 grid((unsigned)((p->max_member_points + tpb - 1) / tpb), M);
    ScanParams sp;
    sp.nbins = p->nbins;
    sp.bstride = p->bstride;
    sp.cstride = p->cstride;
    sp.nch = p->nch;
    sp.nbx = p->nbx;
    sp.nbr = q.n2 / q.tile_y;
    sp.tile_y = q.tile_y;
    sp.c0 = p->c0;
    sp.w = q.w;
    sp.n2 = q.n2;
    if (p->keep_order) {
        if (q.dtype == DFSNUFFT_F64)
            k_fold_direct<double><<<grid, tpb, 0, p->stream>>>(lon, colat, f, sp, p->d_pofs,
                                                              p->d_bin_count, p->d_base,
                                                              (double *)p->d_frac, p->d_rowrange);
        else
            k_fold_direct<float><<<grid, tpb, 0, p->stream>>>(lon, colat, f, sp, p->d_pofs,
                                                             p->d_bin_count, p->d_base,
                                                             (float *)p->d_frac, p->d_rowrange);
        return cudaGetLastError();
    }
    const int rowoff = dfs_rowcount_offset(p->bstride);
    if (q.dtype == DFSNUFFT_F64)
        k_fold_count<double><<<grid, tpb, 0, p->stream>>>(lon, colat, f, p->d_pofs, p->cstride,
                                                          rowoff, p->d_bin_count,
                                                          (FoldRec<double> *)p->d_urec);
    else
        k_fold_count<float><<<grid, tpb, 0, p->stream>>>(lon, colat, f, p->d_pofs, p->cstride,
                                                         rowoff, p->d_bin_count,
                                                         (FoldRec<float> *)p->d_urec);
    // the kernels after the fold start launching while their predecessor drains
    if ((e = dfs_launch_dependent(k_row_prefix, dim3((p->nbins + 255) / 256, M), dim3(256), 0,
                                  p->stream, p->nbins, q.tile_y, p->cstride, rowoff,
                                  p->d_bin_count)))
        return e;
    const dim3 sgrid(p->nch, M);
    if ((e = dfs_launch_dependent(k_scan_sums, sgrid, dim3(DFS_SCAN_CHUNK / 16), 0, p->stream, sp,
                                  p->d_bin_count)))
        return e;
    if ((e = dfs_launch_dependent(k_scan_write, sgrid, dim3(DFS_SCAN_CHUNK / 16), 0, p->stream, sp,
                                  p->d_bin_count, p->d_bin_start, p->d_task_bin, p->d_n_tasks,
                                  p->d_rowrange)))
        return e;
    if (q.dtype == DFSNUFFT_F64)
        return dfs_launch_dependent(k_scatter<double>, grid, dim3(tpb), 0, p->stream,
                                    (const FoldRec<double> *)p->d_urec, f, p->d_pofs, p->bstride,
                                    (const int *)p->d_bin_start, p->cstride, rowoff,
                                    (const int *)p->d_bin_count, p->d_base, (double2 *)p->d_frac,
                                    p->d_idx);
    return dfs_launch_dependent(k_scatter<float>, grid, dim3(tpb), 0, p->stream,
                                (const FoldRec<float> *)p->d_urec, f, p->d_pofs, p->bstride,
                                (const int *)p->d_bin_start, p->cstride, rowoff,
                                (const int *)p->d_bin_count, p->d_base, (float2 *)p->d_frac,
                                p->d_idx);
}

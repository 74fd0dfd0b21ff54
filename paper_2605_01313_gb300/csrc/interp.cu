// Interpolation from the fine grid to the departure points: the last stage of
// the type-2 NUFFT evaluating Eq. 5.3 (Sec. 5).  For each point
//
//   Re v_p = sum_{b<w} sum_{a<w} phi(z_b^y) phi(z_a^x) Re G[j0 + b][i0 + a]   (indices mod n)
//
// with phi the exponential-of-semicircle kernel
// phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)) and z_a = (a - c0) - t the
// offsets produced by set_points; the weights come from a per-tap polynomial
// fit of phi in t (see Horner below).
//
// The weights are real, so only the real part of the fine grid is read (the
// phi pass stores nothing else).  Points arrive sorted by bin (tile_x x tile_y
// fine cells); one CTA takes a bin, stages the bin's tile plus its halo of
// every field into shared memory with coalesced loads, and each thread then
// evaluates one point at a time from shared memory, computing its 2w kernel
// values once for all fields.
#include "common.cuh"
#include "tma.cuh"

namespace {

struct InterpArgs {
    int n1, n2;
    int tile_x, tile_y, nbx;
    int c0;
    int F, FG;            // fields per member, fields staged per pass
    int bstride;          // per-member stride of the bin arrays
};

// Kernel weights by Horner's rule: for tap a the weight phi((a - c0) - t) is a
// degree-W polynomial in s = t - mid (mid = 0 for odd W, 1/2 for even W),
// fitted on the host (dfsnufft_es_horner) to about e^-beta, the size of the
// kernel's own jump at the edge of its support.  The coefficients ride in the
// kernel's parameter block, so every Horner step is one FMA with a constant
// operand; a NaN offset gives NaN weights.
template <typename R, int W>
struct Horner {
    R c[W][W + 1];
};

template <typename R, int W>
__device__ __forceinline__ void es_weights(R t, const Horner<R, W> &h, R *wv) {
    const R s = t - (W % 2 == 0 ? (R)0.5 : (R)0);
#pragma unroll
    for (int a = 0; a < W; ++a) {
        R acc = h.c[a][W];
#pragma unroll
        for (int k = W - 1; k >= 0; --k) acc = fma(acc, s, h.c[a][k]);
        wv[a] = acc;
    }
}

template <typename R, int W>
__global__ void __launch_bounds__(256) k_interp(InterpArgs a, const __grid_constant__ Horner<R, W> hw,
                                                const R *__restrict__ grid,
                                                const int2 *__restrict__ base,
                                                const R *__restrict__ frac,
                                                const int *__restrict__ idx,
                                                const int *__restrict__ bin_start_all,
                                                const int *__restrict__ task_all,
                                                const int *__restrict__ n_tasks,
                                                const int *__restrict__ pofs,
                                                R *__restrict__ out_all) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *tile = reinterpret_cast<R *>(smem_raw);
    const int TH = a.tile_y + W - 1;
    const int TW = a.tile_x + W - 1;
    const int tsz = TH * TW;
    // member k = blockIdx.y: its bins, sorted records [p0, p0 + Pk), F fine grids
    // and F x Pk outputs
    const int k = blockIdx.y;
    const int p0 = pofs[k];
    const int Pk = pofs[k + 1] - p0;
    const int ntask = n_tasks[k];
    const int *task_bin = task_all + (size_t)k * a.bstride;
    const int *bin_start = bin_start_all + (size_t)k * a.bstride;
    for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
        const int bin = task_bin[task];
        const int by = bin / a.nbx;
        const int bx = bin - by * a.nbx;
        const int col0 = bx * a.tile_x - a.c0;
        const int row0 = by * a.tile_y - a.c0;
        const int s = p0 + bin_start[bin];
        const int e = p0 + bin_start[bin + 1];
        for (int f0 = 0; f0 < a.F; f0 += a.FG) {
            const int fg = min(a.FG, a.F - f0);
            __syncthreads();
            // one warp per tile row: coalesced reads of TW consecutive cells
            for (int rr = threadIdx.x >> 5; rr < fg * TH; rr += blockDim.x >> 5) {
                const int ff = rr / TH;
                const int r = rr - ff * TH;
                const int gr = (row0 + r) & (a.n2 - 1);
                const R *src = grid + ((size_t)(k * a.F + f0 + ff) * a.n2 + gr) * a.n1;
                R *dst = tile + ff * tsz + r * TW;
                for (int cc = threadIdx.x & 31; cc < TW; cc += 32)
                    dst[cc] = src[(col0 + cc) & (a.n1 - 1)];
            }
            __syncthreads();
            for (int pi = s + threadIdx.x; pi < e; pi += blockDim.x) {
                const int2 b = base[pi];
                R wx[W], wy[W];
                es_weights<R, W>(frac[2 * pi], hw, wx);
                es_weights<R, W>(frac[2 * pi + 1], hw, wy);
                const int ox = b.x - col0;
                const int oy = b.y - row0;
                const int dst = idx[pi];
                for (int ff = 0; ff < fg; ++ff) {
                    const R *tp = tile + ff * tsz + oy * TW + ox;
                    R acc = 0;
#pragma unroll
                    for (int bb = 0; bb < W; ++bb) {
                        R rr = 0;
#pragma unroll
                        for (int aa = 0; aa < W; ++aa) rr += wx[aa] * tp[bb * TW + aa];
                        acc += wy[bb] * rr;
                    }
                    out_all[(size_t)a.F * p0 + (size_t)(f0 + ff) * Pk + dst] = acc;
                }
            }
        }
    }
}

// FP32 form: the tile starts at an even column and each stencil row is read as
// WP/2 aligned pairs of cells (8-byte shared loads).  Neighbouring points of
// the departure grid sit about two cells apart, so a warp's loads fall on
// consecutive 8-byte words and do not conflict in the shared-memory banks.
// The point's parity within its pair shifts its w weights into a zero-padded
// vector of WP weights.
template <int W>
__global__ void __launch_bounds__(128) k_interp_f32(InterpArgs a,
                                                    const __grid_constant__ Horner<float, W> hw,
                                                    const float *__restrict__ grid,
                                                    const int2 *__restrict__ base,
                                                    const float *__restrict__ frac,
                                                    const int *__restrict__ idx,
                                                    const int *__restrict__ bin_start_all,
                                                    const int *__restrict__ task_all,
                                                    const int *__restrict__ n_tasks,
                                                    const int *__restrict__ pofs,
                                                    float *__restrict__ out_all) {
    constexpr int WP = (W + 2) & ~1;          // taps read per row, even
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);
    const int TH = a.tile_y + W - 1;
    const int TW = a.tile_x + WP;             // even: rows stay 8-byte aligned
    const int Q = TW / 2;                     // pairs per tile row
    const int tsz = TH * TW;
    // member k = blockIdx.y: its bins, sorted records [p0, p0 + Pk), F fine grids
    // and F x Pk outputs
    const int k = blockIdx.y;
    const int p0 = pofs[k];
    const int Pk = pofs[k + 1] - p0;
    const int ntask = n_tasks[k];
    const int *task_bin = task_all + (size_t)k * a.bstride;
    const int *bin_start = bin_start_all + (size_t)k * a.bstride;
    for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
        const int bin = task_bin[task];
        const int by = bin / a.nbx;
        const int bx = bin - by * a.nbx;
        const int col0 = (bx * a.tile_x - a.c0) & ~1;
        const int row0 = by * a.tile_y - a.c0;
        const int s = p0 + bin_start[bin];
        const int e = p0 + bin_start[bin + 1];
        for (int f0 = 0; f0 < a.F; f0 += a.FG) {
            const int fg = min(a.FG, a.F - f0);
            __syncthreads();
            // one warp per tile row, a lane per pair of cells (Q <= 32); each warp
            // issues the loads of 4 rows before storing any, to keep them in flight
            {
                const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
                const int nrows = fg * TH;
                const int gc = (col0 + 2 * lane) & (a.n1 - 1);
                for (int r0 = threadIdx.x >> 5; r0 < nrows; r0 += 4 * nwarp) {
                    float2 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int rr = r0 + u * nwarp;
                        if (rr < nrows && lane < Q) {
                            const int ff = rr / TH;
                            const int gr = (row0 + rr - ff * TH) & (a.n2 - 1);
                            v[u] = *reinterpret_cast<const float2 *>(
                                grid + ((size_t)(k * a.F + f0 + ff) * a.n2 + gr) * a.n1 + gc);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int rr = r0 + u * nwarp;
                        if (rr < nrows && lane < Q) {
                            const int ff = rr / TH;
                            *reinterpret_cast<float2 *>(tile + ff * tsz + (rr - ff * TH) * TW +
                                                        2 * lane) = v[u];
                        }
                    }
                }
            }
            __syncthreads();
            for (int pi = s + threadIdx.x; pi < e; pi += blockDim.x) {
                const int2 b = base[pi];
                float wx[W], wy[W], w8[WP];
                es_weights<float, W>(frac[2 * pi], hw, wx);
                es_weights<float, W>(frac[2 * pi + 1], hw, wy);
                const int ox = b.x - col0;
                const int odd = ox & 1;
#pragma unroll
                for (int k = 0; k < WP; ++k) {
                    const float lo = k < W ? wx[k] : 0.f;
                    const float hi = (k >= 1 && k - 1 < W) ? wx[k - 1] : 0.f;
                    w8[k] = odd ? hi : lo;
                }
                const int oy = b.y - row0;
                const int dst = idx[pi];
                for (int ff = 0; ff < fg; ++ff) {
                    const float2 *tp = reinterpret_cast<const float2 *>(
                        tile + ff * tsz + oy * TW + (ox - odd));
                    float acc = 0.f;
#pragma unroll
                    for (int bb = 0; bb < W; ++bb) {
                        float rr = 0.f;
#pragma unroll
                        for (int k = 0; k < WP / 2; ++k) {
                            const float2 g = tp[bb * Q + k];
                            rr += w8[2 * k] * g.x + w8[2 * k + 1] * g.y;
                        }
                        acc += wy[bb] * rr;
                    }
                    out_all[(size_t)a.F * p0 + (size_t)(f0 + ff) * Pk + dst] = acc;
                }
            }
        }
    }
}

template <typename R, int W>
cudaError_t launch_w(dfsnufft_plan p, void *values) {
    typedef typename CxT<R>::type C;
    const dfsnufft_params &q = p->prm;
    InterpArgs a;
    a.n1 = q.n1;
    a.n2 = q.n2;
    a.tile_x = q.tile_x;
    a.tile_y = q.tile_y;
    a.nbx = p->nbx;
    a.c0 = p->c0;
    a.F = p->n_fields;
    a.bstride = p->bstride;
    Horner<R, W> hw;
    {
        double hc[W * (W + 1)];
        dfsnufft_es_horner(W, q.beta, hc);
        for (int i = 0; i < W; ++i)
            for (int k = 0; k <= W; ++k) hw.c[i][k] = (R)hc[i * (W + 1) + k];
    }
    // FP32: paired loads, tile rows of at most 32 pairs
    const bool pair = sizeof(R) == 4 && W <= 8 && (q.tile_x + ((W + 2) & ~1)) / 2 <= 32;
    const int tw = pair ? q.tile_x + ((W + 2) & ~1) : q.tile_x + W - 1;
    const size_t per_field = sizeof(R) * (size_t)(q.tile_y + W - 1) * tw;
    int fg = (int)((96 * 1024) / per_field);
    if (fg < 1) fg = 1;
    if (fg > a.F) fg = a.F;
    a.FG = fg;
    const size_t smem = per_field * fg;
    // blocks per member: enough to fill the GPU across all members
    int per = (152 * 16 + p->n_members - 1) / p->n_members;
    if (per > p->nbins) per = p->nbins;
    if (per < 1) per = 1;
    const dim3 blocks(per, p->n_members);
    if (pair) {
        cudaError_t e = dfs_allow_smem((const void *)k_interp_f32<W>, smem);
        if (e) return e;
        Horner<float, W> hf;
        for (int i = 0; i < W; ++i)
            for (int k = 0; k <= W; ++k) hf.c[i][k] = (float)hw.c[i][k];
        k_interp_f32<W><<<blocks, 128, smem, p->stream>>>(
            a, hf, (const float *)p->d_G, p->d_base, (const float *)p->d_frac, p->d_idx,
            p->d_bin_start, p->d_task_bin, p->d_n_tasks, p->d_pofs, (float *)values);
    } else {
        cudaError_t e = dfs_allow_smem((const void *)k_interp<R, W>, smem);
        if (e) return e;
        const int threads = sizeof(R) == 4 ? 128 : 256;
        k_interp<R, W><<<blocks, threads, smem, p->stream>>>(
            a, hw, (const R *)p->d_G, p->d_base, (const R *)p->d_frac, p->d_idx, p->d_bin_start,
            p->d_task_bin, p->d_n_tasks, p->d_pofs, (R *)values);
    }
    return cudaGetLastError();
}

template <typename R, int W>
cudaError_t dispatch(dfsnufft_plan p, void *values, int w) {
    if constexpr (W > 16) {
        return cudaErrorInvalidValue;
    } else {
        if (w == W) return launch_w<R, W>(p, values);
        return dispatch<R, W + 1>(p, values, w);
    }
}

}  // namespace

cudaError_t dfs_launch_interp(dfsnufft_plan p, void *values) {
    if (p->prm.dtype == DFSNUFFT_F64) return dispatch<double, 2>(p, values, p->prm.w);
    return dispatch<float, 2>(p, values, p->prm.w);
}

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
// fine cells); a CTA takes a bin, has the bin's tile plus its halo of every
// field in shared memory, and each thread then evaluates one point at a time
// from shared memory, computing its 2w kernel values once for all fields.
//
// FP32 plans run k_interp_tma: persistent CTAs walk their bins with the next
// bin's tiles arriving by TMA (one 2-D box per field) while the current bin is
// evaluated; the few bins whose tile wraps around the torus seam are staged
// with plain loads instead.  Inside a bin the points come sorted by fine row
// (set_points), so a warp's lanes mostly read consecutive words of one row;
// each stencil row is read with loads as wide as its alignment allows (see
// "Stencil reads" below).  k_interp_f32 (plain loads, paired reads) serves
// plans without a tensor map, and k_interp the FP64 form and wide kernels.
#include <limits.h>

#include "common.cuh"
#include "df32.cuh"
#include "tma.cuh"

namespace {

struct InterpArgs {
    int n1, n2;
    int tile_x, tile_y, nbx;
    int c0;
    int F, FG;            // fields per member, fields staged per pass
    int NG;               // field groups per bin, ceil(F / FG)
    int BW, box_f;        // TMA box width (cells, multiple of 4), floats per staged box
    int bstride;          // per-member stride of the bin arrays
    int fa, fn;           // fields evaluated: fa .. fa + fn - 1 of each member
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

// The i-th of n claims of the TMA kernel's counter, as a position in the bin
// list: from both ends inward (n - 1 - i/2 for even i, i/2 for odd i, a
// permutation of [0, n)).  The densest bins are those of the first and last
// bin rows, where departure points near the poles crowd, so they start first
// rather than one of them holding up the end of the launch.  (The kernels
// that walk the list with a fixed stride keep the plain order: on the
// wave-scheduled FP64 grid this order measured 1179 against 1140 us.)
__device__ __forceinline__ int ends_inward(int i, int n) {
    return (i & 1) ? i >> 1 : n - 1 - (i >> 1);
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
    dfs_grid_wait();
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
        for (int f0 = a.fa; f0 < a.fa + a.fn; f0 += a.FG) {
            const int fg = min(a.FG, a.fa + a.fn - f0);
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

// ---- FP64 plans in double-single arithmetic (df32.cuh)
//
// The fine grid holds (hi, lo) FP32 pairs (written so by the phi pass), the
// Horner coefficients are split the same way, the weights are evaluated by
// double-single Horner steps and every stencil sum is a compensated dot
// product (Dot2): about 10 FP32 operations a tap instead of one FP64 FMA, on
// units that run 64 times faster, with an error of about (w u)^2 sum |w g|
// (u = 2^-24, a few 1e-13 of the value for smooth fields).
#define DFS_DF_FG 4            // fields a CTA of k_interp_df stages at once, at most

template <int W> struct HornerDF {
    float hi[W][W + 1], lo[W][W + 1];
};

// The kernel is even, so tap W-1-a at s is tap a at -s: with tap a's
// polynomial split into even and odd parts in u = s^2, P_a(+-s) = E(u) +- s O(u)
// gives both weights of the mirror pair from two Horner chains of half length.
template <int W>
__device__ __forceinline__ void df_pair(const HornerDF<W> &h, int a, df32 s, df32 u, df32 &lo,
                                        df32 &hi) {
    constexpr int KE = W - (W & 1);           // highest even power
    constexpr int KO = W - 1 + (W & 1);       // highest odd power
    df32 e = {h.hi[a][KE], h.lo[a][KE]};
#pragma unroll
    for (int k = KE - 2; k >= 0; k -= 2) e = df_mul_add(e, u, df32{h.hi[a][k], h.lo[a][k]});
    df32 o = {h.hi[a][KO], h.lo[a][KO]};
#pragma unroll
    for (int k = KO - 2; k >= 1; k -= 2) o = df_mul_add(o, u, df32{h.hi[a][k], h.lo[a][k]});
    const df32 so = s * o;
    lo = e + so;                               // tap a
    hi = e - so;                               // tap W-1-a
}

template <int W>
__device__ __forceinline__ df32 df_offset(double t) {
    return split_double(t - (W % 2 == 0 ? 0.5 : 0.0));
}

template <int W>
__device__ __forceinline__ void df_weights(double t, const HornerDF<W> &h, df32 *wv) {
    const df32 s = df_offset<W>(t);
    const df32 u = s * s;
#pragma unroll
    for (int a = 0; a < (W + 1) / 2; ++a) {
        df32 lo, hi;
        df_pair<W>(h, a, s, u, lo, hi);
        wv[a] = lo;
        if (W - 1 - a != a) wv[W - 1 - a] = hi;
    }
}

// As k_interp, with the tile of (hi, lo) pairs.
template <int W>
__global__ void __launch_bounds__(256) k_interp_df(InterpArgs a,
                                                   const __grid_constant__ HornerDF<W> hw,
                                                   const float2 *__restrict__ grid,
                                                   const int2 *__restrict__ base,
                                                   const double *__restrict__ frac,
                                                   const int *__restrict__ idx,
                                                   const int *__restrict__ bin_start_all,
                                                   const int *__restrict__ task_all,
                                                   const int *__restrict__ n_tasks,
                                                   const int *__restrict__ pofs,
                                                   double *__restrict__ out_all,
                                                   const int *__restrict__ emax) {
    dfs_grid_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);
    const int TH = a.tile_y + W - 1;
    const int TW = a.tile_x + W - 1;
    const int tsz = TH * TW;
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
        for (int f0 = a.fa; f0 < a.fa + a.fn; f0 += a.FG) {
            const int fg = min(a.FG, a.fa + a.fn - f0);
            __syncthreads();
            for (int rr = threadIdx.x >> 5; rr < fg * TH; rr += blockDim.x >> 5) {
                const int ff = rr / TH;
                const int r = rr - ff * TH;
                const int gr = (row0 + r) & (a.n2 - 1);
                const float2 *src = grid + ((size_t)(k * a.F + f0 + ff) * a.n2 + gr) * a.n1;
                float2 *dst = tile + ff * tsz + r * TW;
                for (int cc = threadIdx.x & 31; cc < TW; cc += 32)
                    dst[cc] = src[(col0 + cc) & (a.n1 - 1)];
            }
            __syncthreads();
            for (int pi = s + threadIdx.x; pi < e; pi += blockDim.x) {
                const int2 b = base[pi];
                df32 wx[W];
                df_weights<W>(frac[2 * pi], hw, wx);
                const df32 sy = df_offset<W>(frac[2 * pi + 1]);
                const df32 uy = sy * sy;
                const int ox = b.x - col0;
                const int oy = b.y - row0;
                const int dst = idx[pi];
                // stencil rows by mirror pairs (bb, W-1-bb), whose y weights come
                // from one pair of Horner chains; all fields of the group per
                // row: few live registers
                float r2[DFS_DF_FG], c2[DFS_DF_FG];
#pragma unroll
                for (int ff = 0; ff < DFS_DF_FG; ++ff) r2[ff] = c2[ff] = 0.f;
                auto row = [&](int bb, df32 wyb) {
#pragma unroll
                    for (int ff = 0; ff < DFS_DF_FG; ++ff) {
                        if (ff >= fg) break;
                        const float2 *tp = tile + ff * tsz + (oy + bb) * TW + ox;
                        float r = 0.f, c = 0.f;
#pragma unroll
                        for (int aa = 0; aa < W; ++aa) {
                            const float2 g = tp[aa];
                            dot2_step(r, c, wx[aa], df32{g.x, g.y});
                        }
                        dot2_step(r2[ff], c2[ff], wyb, quick_two_sum(r, c));
                    }
                };
#pragma unroll 1
                for (int bb = 0; bb < (W + 1) / 2; ++bb) {
                    df32 wlo, whi;
                    df_pair<W>(hw, bb, sy, uy, wlo, whi);
                    row(bb, wlo);
                    if (W - 1 - bb != bb) row(W - 1 - bb, whi);
                }
                // back to the caller's scale: the line was carried as c 2^-s
#pragma unroll
                for (int ff = 0; ff < DFS_DF_FG; ++ff)
                    if (ff < fg)
                        out_all[(size_t)a.F * p0 + (size_t)(f0 + ff) * Pk + dst] =
                            ((double)r2[ff] + (double)c2[ff]) *
                            df_pow2(df_line_shift(emax[k * a.F + f0 + ff]));
            }
        }
    }
}

// FP32 weights by mirror pairs.  The kernel is even and the fit is made on
// nodes symmetric about the centre, so tap W-1-a at s is tap a at -s: with tap
// a's polynomial split into even and odd parts in u = s^2, P_a(+-s) = E(u) +-
// s O(u) gives both weights of the pair from two Horner chains of half length
// (about 36 FMAs instead of 49 for w = 7).
template <int W>
__device__ __forceinline__ void es_weights_mirror(float t, const Horner<float, W> &h, float *wv) {
    constexpr int KE = W - (W & 1);           // highest even power
    constexpr int KO = W - 1 + (W & 1);       // highest odd power
    const float s = t - (W % 2 == 0 ? 0.5f : 0.f);
    const float u = s * s;
#pragma unroll
    for (int a = 0; a < (W + 1) / 2; ++a) {
        float e = h.c[a][KE];
#pragma unroll
        for (int k = KE - 2; k >= 0; k -= 2) e = fmaf(e, u, h.c[a][k]);
        float o = h.c[a][KO];
#pragma unroll
        for (int k = KO - 2; k >= 1; k -= 2) o = fmaf(o, u, h.c[a][k]);
        wv[a] = fmaf(s, o, e);
        if (W - 1 - a != a) wv[W - 1 - a] = fmaf(-s, o, e);
    }
}

// Weights of one FP32 point for the paired reads: wy[W] and the x weights
// shifted by the parity of the first tap into a zero-padded vector w8[WP].
template <int W>
__device__ __forceinline__ void paired_weights(float tx, float ty, int odd,
                                               const Horner<float, W> &hw, float *w8,
                                               float *wy) {
    constexpr int WP = (W + 2) & ~1;
    float wx[W];
    es_weights_mirror<W>(tx, hw, wx);
    es_weights_mirror<W>(ty, hw, wy);
#pragma unroll
    for (int k = 0; k < WP; ++k) {
        const float lo = k < W ? wx[k] : 0.f;
        const float hi = (k >= 1 && k - 1 < W) ? wx[k - 1] : 0.f;
        w8[k] = odd ? hi : lo;
    }
}

// Stencil reads of the FP32 TMA kernel.  A tile row holds BW cells (a multiple
// of 4) and starts on a 16-byte boundary; the point's W taps start at column
// ox of its row.  Three read patterns, chosen by W:
//
// Exact-width reads, W = 4q + 3 (w = 7 on 32-cell bins, whose row stride is a
// compile-time constant): the row's W cells are one 8-byte pair, one single
// cell and q aligned 16-byte quads, in an order fixed by m = ox mod 4.
// Offsets from the first tap:
//   m = 0: quads at 0,  pair at 4q,     single at 4q + 2
//   m = 1: single at 0, pair at 1,      quads at 3
//   m = 2: pair at 0,   quads at 2,     single at 4q + 2
//   m = 3: single at 0, quads at 1,     pair at 4q + 1
// Every access is aligned to its width and no cell outside the stencil is
// read: 2 + q loads a row instead of (W + 1) / 2 pairs, and fewer bank
// conflicts, since a quarter-warp's 16-byte loads of neighbouring points of
// one row fall on distinct banks.  For 2.1M points and three fields on a
// 2048 x 1024 grid (w = 7) this took the kernel from 86 to 77 us.
//
// Split reads, other odd W (and w = 7 on other bin widths): (W - 1) / 2
// aligned pairs and one single cell (first when ox is odd, last when it is
// even); 80 us on the same case.  Launches of one field (the host-buffer
// pipeline) would run faster in this form (fewer registers, and the per-point
// set-up of the exact-width weights is not shared by several fields), but the
// two forms add a row's products in different orders, and every launch of a
// plan keeps one form so that all its entry points give the same bits.
//
// Paired reads, even W: WP / 2 aligned pairs from the even column at or
// below ox, the point's weights shifted by the parity of ox (paired_weights).
template <int W> struct ExactRow {
    static constexpr int Q4 = W / 4;          // 16-byte quads a row
    int o4, o2, o1;                           // offsets of the quads, the pair, the single cell
    float w4[Q4 > 0 ? 4 * Q4 : 1], w2[2], w1; // the x weights in that order
};

template <int W>
__device__ __forceinline__ void exact_weights(float tx, float ty, int m,
                                              const Horner<float, W> &hw, ExactRow<W> &er,
                                              float *wy) {
    static_assert(W % 4 == 3, "exact-width reads need W = 4q + 3");
    constexpr int Q4 = ExactRow<W>::Q4;
    float wx[W];
    es_weights_mirror<W>(tx, hw, wx);
    es_weights_mirror<W>(ty, hw, wy);
    er.o4 = (4 - m) & 3;
    er.o2 = m == 0 ? 4 * Q4 : m == 1 ? 1 : m == 2 ? 0 : 4 * Q4 + 1;
    er.o1 = (m & 1) ? 0 : W - 1;
#pragma unroll
    for (int i = 0; i < 4 * Q4; ++i)
        er.w4[i] = m == 0 ? wx[i] : m == 1 ? wx[3 + i] : m == 2 ? wx[2 + i] : wx[1 + i];
#pragma unroll
    for (int i = 0; i < 2; ++i)
        er.w2[i] = m == 0 ? wx[4 * Q4 + i] : m == 1 ? wx[1 + i] : m == 2 ? wx[i]
                                                                        : wx[4 * Q4 + 1 + i];
    er.w1 = (m & 1) ? wx[0] : wx[W - 1];
}

// The w x w stencil sum of one field by exact-width reads: tp points at the
// first tap's cell in the tile, rows BWC floats apart (bw_rt when BWC is 0).
template <int W, int BWC>
__device__ __forceinline__ float exact_sum(const float *tp, int bw_rt, const ExactRow<W> &er,
                                           const float *wy) {
    const int bw = BWC ? BWC : bw_rt;
    const float *p1 = tp + er.o1;
    const float2 *p2 = reinterpret_cast<const float2 *>(tp + er.o2);
    const float4 *p4 = reinterpret_cast<const float4 *>(tp + er.o4);
    float acc = 0.f;
#pragma unroll
    for (int bb = 0; bb < W; ++bb) {
        const float2 g2 = p2[bb * (bw / 2)];
        float rr = er.w1 * p1[bb * bw];
        rr = fmaf(er.w2[0], g2.x, rr);
        rr = fmaf(er.w2[1], g2.y, rr);
#pragma unroll
        for (int c = 0; c < ExactRow<W>::Q4; ++c) {
            const float4 g = p4[bb * (bw / 4) + c];
            rr = fmaf(er.w4[4 * c], g.x, rr);
            rr = fmaf(er.w4[4 * c + 1], g.y, rr);
            rr = fmaf(er.w4[4 * c + 2], g.z, rr);
            rr = fmaf(er.w4[4 * c + 3], g.w, rr);
        }
        acc = fmaf(wy[bb], rr, acc);
    }
    return acc;
}

// Split reads (odd W): the x weights in read order, the single cell's last.
template <int W> struct SplitRow {
    int o2, o1;
    float w2[W - 1], w1;
};

template <int W>
__device__ __forceinline__ void split_weights(float tx, float ty, int odd,
                                              const Horner<float, W> &hw, SplitRow<W> &sr,
                                              float *wy) {
    static_assert(W % 2 == 1, "split reads need odd W");
    float wx[W];
    es_weights_mirror<W>(tx, hw, wx);
    es_weights_mirror<W>(ty, hw, wy);
    sr.o2 = odd;
    sr.o1 = odd ? 0 : W - 1;
#pragma unroll
    for (int i = 0; i < W - 1; ++i) sr.w2[i] = odd ? wx[1 + i] : wx[i];
    sr.w1 = odd ? wx[0] : wx[W - 1];
}

template <int W>
__device__ __forceinline__ float split_sum(const float *tp, int bw, const SplitRow<W> &sr,
                                           const float *wy) {
    const float *p1 = tp + sr.o1;
    const float2 *p2 = reinterpret_cast<const float2 *>(tp + sr.o2);
    float acc = 0.f;
#pragma unroll
    for (int bb = 0; bb < W; ++bb) {
        float rr = sr.w1 * p1[bb * bw];
#pragma unroll
        for (int k = 0; k < (W - 1) / 2; ++k) {
            const float2 g = p2[bb * (bw / 2) + k];
            rr = fmaf(sr.w2[2 * k], g.x, rr);
            rr = fmaf(sr.w2[2 * k + 1], g.y, rr);
        }
        acc = fmaf(wy[bb], rr, acc);
    }
    return acc;
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
        for (int f0 = a.fa; f0 < a.fa + a.fn; f0 += a.FG) {
            const int fg = min(a.FG, a.fa + a.fn - f0);
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
                const int ox = b.x - col0;
                const int odd = ox & 1;
                float wy[W], w8[WP];
                paired_weights<W>(frac[2 * pi], frac[2 * pi + 1], odd, hw, w8, wy);
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

// FP32 with TMA staging.  grid (CTAs per member, members); the CTAs of member
// k claim its sub-tasks from the member's counter work[2k] (one atomic a
// claim), a sub-task being one non-empty bin and one group of FG fields, so
// that SMs whose bins hold fewer points take more of them and all finish
// together.  Claims take the sub-tasks from both ends of the bin list inward
// (ends_inward): the bins of the first and last bin rows, where departure
// points near the poles crowd (up to six times a bin's median count on a
// 2048 x 1024 grid), start first instead of one of them holding up the end of
// the launch.  The last CTA of the member to finish (counter work[2k + 1])
// sets both counters back to zero for the next launch.
//
// Two stages: while a CTA evaluates its sub-task from stage j & 1, the boxes
// of the next one it claimed land in the other stage (claimed and issued by
// thread 0 after the barrier that ends the reads of that stage).  A box starts
// at the bin's first stencil column rounded down to 4 cells (16 bytes, the TMA
// alignment rule), so a point's first tap sits at column ox in [0, tile_x + 2]
// of the box and its reads end below tile_x + 2 + WP <= BW.  BWC, when
// nonzero, is BW as a compile-time constant (the exact-width reads).  A box
// that would leave [0, n1) x [0, n2) (a bin at the torus seam) is not copied
// by TMA: its barrier phase completes on the issuing thread's arrival alone,
// and the CTA stages the tile with wrapped plain loads.  A wait that runs out
// (about a second) sets the status word to DFS_STATUS_TIMEOUT and ends the
// CTA's loop after its copies land.
template <int W, int BWC>
__global__ void __launch_bounds__(128) k_interp_tma(InterpArgs a,
                                                    const __grid_constant__ Horner<float, W> hw,
                                                    const __grid_constant__ CUtensorMap gmap,
                                                    const float *__restrict__ grid,
                                                    const int2 *__restrict__ base,
                                                    const float *__restrict__ frac,
                                                    const int *__restrict__ idx,
                                                    const int *__restrict__ bin_start_all,
                                                    const int *__restrict__ task_all,
                                                    const int *__restrict__ n_tasks,
                                                    const int *__restrict__ pofs,
                                                    float *__restrict__ out_all,
                                                    int *__restrict__ status,
                                                    int *__restrict__ work) {
    dfs_grid_wait();
    constexpr int WP = (W + 2) & ~1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sb = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sb);
    int *s_sub = reinterpret_cast<int *>(sb + 16);   // the sub-task staged in each stage
    float *stage = reinterpret_cast<float *>(sb + 128);
    const int TH = a.tile_y + W - 1;
    const int BWr = BWC ? BWC : a.BW;         // floats per box row
    const int Q = BWr / 2;                    // pairs per box row
    const int k = blockIdx.y;
    const int p0 = pofs[k];
    const int Pk = pofs[k + 1] - p0;
    const int total = n_tasks[k] * a.NG;
    const int *task_bin = task_all + (size_t)k * a.bstride;
    const int *bin_start = bin_start_all + (size_t)k * a.bstride;
    int *wk = work + 2 * k;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const unsigned box_bytes = (unsigned)(a.BW * TH * 4);
    auto wraps = [&](int col0, int row0) {
        return col0 < 0 || col0 + a.BW > a.n1 || row0 < 0 || row0 + TH > a.n2;
    };
    auto issue = [&](int sub, int b) {
        const int task = sub / a.NG;
        const int f0 = a.fa + (sub - task * a.NG) * a.FG;
        const int fg = min(a.FG, a.fa + a.fn - f0);
        const int bin = task_bin[task];
        const int by = bin / a.nbx;
        const int bx = bin - by * a.nbx;
        const int col0 = (bx * a.tile_x - a.c0) & ~3;
        const int row0 = by * a.tile_y - a.c0;
        if (wraps(col0, row0)) {
            mbar_arrive_expect_tx(&bar[b], 0);
            return;
        }
        float *dst = stage + (size_t)b * a.FG * a.box_f;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[b], box_bytes * fg);
        for (int ff = 0; ff < fg; ++ff)
            tma_load_2d(dst + (size_t)ff * a.box_f, &gmap, col0 >> 1,   // 8-byte units
                        (k * a.F + f0 + ff) * a.n2 + row0, &bar[b]);
    };
    uint32_t ph0 = 0, ph1 = 0;
    auto claim = [&]() {
        const int i = atomicAdd(&wk[0], 1);
        return i >= total ? total : ends_inward(i, total);
    };
    if (threadIdx.x == 0) {
        const int first = claim();
        s_sub[0] = first;
        if (first < total) issue(first, 0);
    }
    __syncthreads();
    for (int it = 0;; ++it) {
        const int cur = it & 1;
        const int sub = s_sub[cur];
        if (sub >= total) break;
        int nxt = total;
        if (threadIdx.x == 0) {
            nxt = claim();
            s_sub[cur ^ 1] = nxt;
            if (nxt < total) issue(nxt, cur ^ 1);
        }
        // geometry and the first point's record, fetched while the boxes land
        const int task = sub / a.NG;
        const int f0 = a.fa + (sub - task * a.NG) * a.FG;
        const int fg = min(a.FG, a.fa + a.fn - f0);
        const int bin = task_bin[task];
        const int by = bin / a.nbx;
        const int bx = bin - by * a.nbx;
        const int col0 = (bx * a.tile_x - a.c0) & ~3;
        const int row0 = by * a.tile_y - a.c0;
        const int s = p0 + bin_start[bin];
        const int e = p0 + bin_start[bin + 1];
        int pi = s + threadIdx.x;
        int2 b = make_int2(0, 0);
        float2 t = make_float2(0.f, 0.f);
        int dst = 0;
        if (pi < e) {
            b = base[pi];
            t = reinterpret_cast<const float2 *>(frac)[pi];
            dst = idx[pi];
        }
        const bool ok = mbar_wait_bounded(&bar[cur], cur ? ph1 : ph0);
        if (cur) ph1 ^= 1;
        else ph0 ^= 1;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(status, DFS_STATUS_TIMEOUT);
                mbar_wait_bounded(&bar[cur], cur ? ph1 ^ 1 : ph0 ^ 1);
                if (nxt < total) mbar_wait_bounded(&bar[cur ^ 1], cur ? ph0 : ph1);
            }
            __syncthreads();
            break;
        }
        float *tile = stage + (size_t)cur * a.FG * a.box_f;
        if (wraps(col0, row0)) {
            // seam bin: the same box, gathered with indices taken mod n
            const int nq = fg * TH * Q;
            for (int i = threadIdx.x; i < nq; i += blockDim.x) {
                const int rr = i / Q;
                const int qq = i - rr * Q;
                const int ff = rr / TH;
                const int r = rr - ff * TH;
                const int gr = (row0 + r) & (a.n2 - 1);
                const int gc = (col0 + 2 * qq) & (a.n1 - 1);
                *reinterpret_cast<float2 *>(tile + (size_t)ff * a.box_f + r * BWr + 2 * qq) =
                    *reinterpret_cast<const float2 *>(
                        grid + ((size_t)(k * a.F + f0 + ff) * a.n2 + gr) * a.n1 + gc);
            }
            __syncthreads();
        }
        while (pi < e) {
            const int ox = b.x - col0;
            const int oy = b.y - row0;
            const int d = dst;
            if constexpr (BWC != 0 && W % 4 == 3) {
                ExactRow<W> er;
                float wy[W];
                exact_weights<W>(t.x, t.y, ox & 3, hw, er, wy);
                pi += blockDim.x;
                if (pi < e) {                  // next record in flight during the sums
                    b = base[pi];
                    t = reinterpret_cast<const float2 *>(frac)[pi];
                    dst = idx[pi];
                }
                for (int ff = 0; ff < fg; ++ff) {
                    const float *tp = tile + (size_t)ff * a.box_f + oy * BWr + ox;
                    out_all[(size_t)a.F * p0 + (size_t)(f0 + ff) * Pk + d] =
                        exact_sum<W, BWC>(tp, BWr, er, wy);
                }
                continue;
            }
            if constexpr (W % 2 == 1) {
                SplitRow<W> sr;
                float wy[W];
                split_weights<W>(t.x, t.y, ox & 1, hw, sr, wy);
                pi += blockDim.x;
                if (pi < e) {                  // next record in flight during the sums
                    b = base[pi];
                    t = reinterpret_cast<const float2 *>(frac)[pi];
                    dst = idx[pi];
                }
                for (int ff = 0; ff < fg; ++ff) {
                    const float *tp = tile + (size_t)ff * a.box_f + oy * BWr + ox;
                    out_all[(size_t)a.F * p0 + (size_t)(f0 + ff) * Pk + d] =
                        split_sum<W>(tp, BWr, sr, wy);
                }
                continue;
            }
            const int odd = ox & 1;
            float w8[WP], wy[W];
            paired_weights<W>(t.x, t.y, odd, hw, w8, wy);
            pi += blockDim.x;
            if (pi < e) {                      // next record in flight during the sums
                b = base[pi];
                t = reinterpret_cast<const float2 *>(frac)[pi];
                dst = idx[pi];
            }
            for (int ff = 0; ff < fg; ++ff) {
                const float2 *tp = reinterpret_cast<const float2 *>(
                    tile + (size_t)ff * a.box_f + oy * BWr + (ox - odd));
                float acc = 0.f;
#pragma unroll
                for (int bb = 0; bb < W; ++bb) {
                    float rr = 0.f;
#pragma unroll
                    for (int kk = 0; kk < WP / 2; ++kk) {
                        const float2 g = tp[bb * Q + kk];
                        rr += w8[2 * kk] * g.x + w8[2 * kk + 1] * g.y;
                    }
                    acc += wy[bb] * rr;
                }
                out_all[(size_t)a.F * p0 + (size_t)(f0 + ff) * Pk + d] = acc;
            }
        }
        __syncthreads();                       // stage cur is free for the claim after next
    }
    // the member's last CTA to finish resets its counters for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&wk[1], 1) == (int)gridDim.x - 1) {
            wk[0] = 0;
            wk[1] = 0;
            __threadfence();
        }
    }
}

// Points in the caller's order (DFSNUFFT_KEEP_ORDER): one thread per point,
// member k = blockIdx.y; the stencil rows are read from the fine grid through
// the L1 cache (neighbouring points of a grid-ordered set share rows), indices
// taken mod n.  FP32 reads each row as WP/2 aligned pairs (paired_weights).
template <typename R, int W>
__global__ void __launch_bounds__(256) k_interp_direct(InterpArgs a,
                                                       const __grid_constant__ Horner<R, W> hw,
                                                       const R *__restrict__ grid,
                                                       const int2 *__restrict__ base,
                                                       const R *__restrict__ frac,
                                                       const int *__restrict__ pofs,
                                                       R *__restrict__ out_all) {
    constexpr bool PAIR = sizeof(R) == 4 && W <= 8;
    constexpr int WP = (W + 2) & ~1;
    const int k = blockIdx.y;
    const int p0 = pofs[k];
    const int Pk = pofs[k + 1] - p0;
    const int m1 = a.n1 - 1, m2 = a.n2 - 1;
    for (int pl = blockIdx.x * blockDim.x + threadIdx.x; pl < Pk; pl += gridDim.x * blockDim.x) {
        const int2 b = base[p0 + pl];
        const R tx = frac[2 * (size_t)(p0 + pl)], ty = frac[2 * (size_t)(p0 + pl) + 1];
        R *out = out_all + (size_t)a.F * p0 + pl;
        if constexpr (PAIR) {
            const int odd = b.x & 1;
            const int cx = b.x - odd;                  // even: pairs never straddle a row end
            float w8[WP], wy[W];
            paired_weights<W>(tx, ty, odd, hw, w8, wy);
            for (int f = a.fa; f < a.fa + a.fn; ++f) {
                const float *g = grid + (size_t)(k * a.F + f) * a.n2 * a.n1;
                float acc = 0.f;
#pragma unroll
                for (int bb = 0; bb < W; ++bb) {
                    const float *gr = g + (size_t)((b.y + bb) & m2) * a.n1;
                    float rr = 0.f;
#pragma unroll
                    for (int kk = 0; kk < WP / 2; ++kk) {
                        const float2 v = __ldg(reinterpret_cast<const float2 *>(
                            gr + ((cx + 2 * kk) & m1)));
                        rr += w8[2 * kk] * v.x + w8[2 * kk + 1] * v.y;
                    }
                    acc += wy[bb] * rr;
                }
                out[(size_t)f * Pk] = acc;
            }
        } else {
            R wx[W], wy[W];
            es_weights<R, W>(tx, hw, wx);
            es_weights<R, W>(ty, hw, wy);
            for (int f = a.fa; f < a.fa + a.fn; ++f) {
                const R *g = grid + (size_t)(k * a.F + f) * a.n2 * a.n1;
                R acc = 0;
#pragma unroll
                for (int bb = 0; bb < W; ++bb) {
                    const R *gr = g + (size_t)((b.y + bb) & m2) * a.n1;
                    R rr = 0;
#pragma unroll
                    for (int aa = 0; aa < W; ++aa) rr += wx[aa] * __ldg(gr + ((b.x + aa) & m1));
                    acc += wy[bb] * rr;
                }
                out[(size_t)f * Pk] = acc;
            }
        }
    }
}

// Points in the caller's order, FP32: each warp takes 32 consecutive points of
// a member, finds their stencils' bounding box (coordinates unwrapped around
// lane 0's, so a chunk across the torus seam stays compact) and, when the box
// fits half of its shared-memory slice of WT_CAP floats, stages the fields'
// boxes by asynchronous 8-byte copies (cp.async, indices taken mod n), field
// f + 1 landing in one half while field f is evaluated from the other; a chunk
// whose box does not fit reads its stencils from the fine grid directly.  Points of one arrival row sit about two cells apart, so
// the warp's pair reads fall on consecutive words.  grid (CTAs, members).
#define WT_CAP 1536
template <int W>
__global__ void __launch_bounds__(256) k_interp_wtile(InterpArgs a,
                                                      const __grid_constant__ Horner<float, W> hw,
                                                      const float *__restrict__ grid,
                                                      const int2 *__restrict__ base,
                                                      const float *__restrict__ frac,
                                                      const int *__restrict__ pofs,
                                                      float *__restrict__ out_all) {
    constexpr int WP = (W + 2) & ~1;
    __shared__ __align__(16) float tiles[8][WT_CAP];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float *tile = tiles[wid];
    const int k = blockIdx.y;
    const int p0 = pofs[k];
    const int Pk = pofs[k + 1] - p0;
    const int m1 = a.n1 - 1, m2 = a.n2 - 1;
    const int nchunk = (Pk + 31) >> 5;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    for (int ch = blockIdx.x * (blockDim.x >> 5) + wid; ch < nchunk; ch += wstride) {
        const int pl = (ch << 5) + lane;
        const bool live = pl < Pk;
        int2 b = make_int2(0, 0);
        float2 t = make_float2(0.f, 0.f);
        if (live) {
            b = base[p0 + pl];
            t = reinterpret_cast<const float2 *>(frac)[p0 + pl];
        }
        // unwrap around lane 0's cell, then the chunk's box
        const int bx0 = __shfl_sync(0xffffffffu, b.x, 0), by0 = __shfl_sync(0xffffffffu, b.y, 0);
        const int ux = bx0 + ((((b.x - bx0) + (a.n1 >> 1)) & m1) - (a.n1 >> 1));
        const int uy = by0 + ((((b.y - by0) + (a.n2 >> 1)) & m2) - (a.n2 >> 1));
        const int xmin = __reduce_min_sync(0xffffffffu, live ? ux : INT_MAX);
        const int xmax = __reduce_max_sync(0xffffffffu, live ? ux : INT_MIN);
        const int ymin = __reduce_min_sync(0xffffffffu, live ? uy : INT_MAX);
        const int ymax = __reduce_max_sync(0xffffffffu, live ? uy : INT_MIN);
        const int col0 = xmin & ~1;                        // even: pairs stay aligned
        const int TW = ((xmax - col0) + WP + 1) & ~1;      // pair reads end below TW
        const int TH = ymax - ymin + W;
        const int Q = TW >> 1;
        const bool fits = 2 * TW * TH <= WT_CAP;
        // lanes past the member's last point read the box's first cells
        const int ox = live ? ux - col0 : 0, odd = ox & 1, oy = live ? uy - ymin : 0;
        float w8[WP], wy[W];
        paired_weights<W>(t.x, t.y, odd, hw, w8, wy);
        float *out = out_all + (size_t)a.F * p0 + pl;
        // asynchronous copies of field f's box into half f & 1 of the slice
        auto stage = [&](int f) {
            const float *g = grid + (size_t)(k * a.F + f) * a.n2 * a.n1;
            float *dst = tile + (f & 1) * (WT_CAP / 2);
            for (int r = 0; r < TH; ++r) {
                const float *gr = g + (size_t)((ymin + r) & m2) * a.n1;
                for (int q = lane; q < Q; q += 32)
                    cp_async_8(dst + r * TW + 2 * q, gr + ((col0 + 2 * q) & m1));
            }
            cp_async_commit();
        };
        __syncwarp();                                      // the previous chunk's boxes are consumed
        if (fits) stage(a.fa);
        for (int f = a.fa; f < a.fa + a.fn; ++f) {
            const float *g = grid + (size_t)(k * a.F + f) * a.n2 * a.n1;
            float acc = 0.f;
            if (fits) {
                if (f + 1 < a.fa + a.fn) {
                    __syncwarp();                          // half (f + 1) & 1 was read at f - 1
                    stage(f + 1);
                    cp_async_wait_group<1>();
                } else {
                    cp_async_wait_group<0>();
                }
                __syncwarp();
                const float2 *tp = reinterpret_cast<const float2 *>(
                    tile + (f & 1) * (WT_CAP / 2) + oy * TW + (ox - odd));
#pragma unroll
                for (int bb = 0; bb < W; ++bb) {
                    float rr = 0.f;
#pragma unroll
                    for (int kk = 0; kk < WP / 2; ++kk) {
                        const float2 v = tp[bb * Q + kk];
                        rr += w8[2 * kk] * v.x + w8[2 * kk + 1] * v.y;
                    }
                    acc += wy[bb] * rr;
                }
            } else {
                const int cx = b.x - odd;
#pragma unroll
                for (int bb = 0; bb < W; ++bb) {
                    const float *gr = g + (size_t)((b.y + bb) & m2) * a.n1;
                    float rr = 0.f;
#pragma unroll
                    for (int kk = 0; kk < WP / 2; ++kk) {
                        const float2 v = __ldg(reinterpret_cast<const float2 *>(
                            gr + ((cx + 2 * kk) & m1)));
                        rr += w8[2 * kk] * v.x + w8[2 * kk + 1] * v.y;
                    }
                    acc += wy[bb] * rr;
                }
            }
            if (live) out[(size_t)f * Pk] = acc;
        }
    }
}

template <typename R, int W>
cudaError_t launch_w(dfsnufft_plan p, void *values) {
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
    // a line window (one-member plans) selects fields
    a.fa = p->nwin ? p->win0 : 0;
    a.fn = p->nwin ? p->nwin : a.F;
    a.NG = 1;
    a.BW = 0;
    a.box_f = 0;
    Horner<R, W> hw;
    {
        double hc[W * (W + 1)];
        dfsnufft_es_horner(W, q.beta, hc);
        for (int i = 0; i < W; ++i)
            for (int k = 0; k <= W; ++k) hw.c[i][k] = (R)hc[i * (W + 1) + k];
    }
    const int M = p->n_members;
    constexpr int WP = (W + 2) & ~1;
    if (p->keep_order) {
        int64_t blocks = (p->max_member_points + 255) / 256;
        if (blocks < 1) blocks = 1;
        if constexpr (sizeof(R) == 4 && W <= 8) {
            Horner<float, W> hf;
            for (int i = 0; i < W; ++i)
                for (int kk = 0; kk <= W; ++kk) hf.c[i][kk] = (float)hw.c[i][kk];
            k_interp_wtile<W><<<dim3((unsigned)blocks, M), 256, 0, p->stream>>>(
                a, hf, (const float *)p->d_G, p->d_base, (const float *)p->d_frac, p->d_pofs,
                (float *)values);
            return cudaGetLastError();
        }
        k_interp_direct<R, W><<<dim3((unsigned)blocks, M), 256, 0, p->stream>>>(
            a, hw, (const R *)p->d_G, p->d_base, (const R *)p->d_frac, p->d_pofs, (R *)values);
        return cudaGetLastError();
    }
    if constexpr (sizeof(R) == 4 && W <= 8) {
        Horner<float, W> hf;
        for (int i = 0; i < W; ++i)
            for (int k = 0; k <= W; ++k) hf.c[i][k] = (float)hw.c[i][k];
        // TMA form: plans that own their buffers (status word, fixed d_G)
        const int TH = q.tile_y + W - 1;
        const int BW = (q.tile_x + WP + 2 + 3) & ~3;
        if (p->d_status && p->d_work && BW / 2 <= 256 && TH <= 256) {
            if (!p->tmap_G_ok) {
                if (dfs_encode_tensor_map_2d(&p->tmap_G, p->d_G, (uint64_t)(q.n1 / 2),
                                             (uint64_t)M * a.F * q.n2,
                                             (uint64_t)q.n1 * sizeof(float), (uint32_t)(BW / 2),
                                             (uint32_t)TH) == cudaSuccess)
                    p->tmap_G_ok = 1;
            }
            if (p->tmap_G_ok) {
                a.BW = BW;
                a.box_f = (BW * TH + 31) & ~31;           // 128-byte aligned boxes
                // fields per stage: two stages within about 26 KB
                int fg = (13 * 1024) / (a.box_f * 4);
                if (fg < 1) fg = 1;
                if (fg > a.F) fg = a.F;
                a.FG = fg;
                a.NG = (a.fn + fg - 1) / fg;
                const size_t smem = 128 + 128 + 2 * (size_t)fg * a.box_f * sizeof(float);
                // w = 7 on 32-cell bins (BW = 44): the exact-width reads, in
                // every launch of the plan, so that launches of one field (the
                // host-buffer pipeline) and of all fields give the same bits
                auto kern = k_interp_tma<W, 0>;
                if constexpr (W == 7)
                    if (BW == 44) kern = k_interp_tma<W, 44>;
                cudaError_t e = dfs_allow_smem((const void *)kern, smem);
                if (e) return e;
                if (p->interp_ctas_per_sm <= 0) {
                    int occ = 0;
                    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128,
                                                                      smem) != cudaSuccess ||
                        occ < 1)
                        occ = 1;
                    p->interp_ctas_per_sm = occ;
                }
                int64_t want = ((int64_t)p->num_sms * p->interp_ctas_per_sm + M - 1) / M;
                const int64_t cap = (int64_t)p->nbins * a.NG;
                if (want > cap) want = cap;
                if (want < 1) want = 1;
                return dfs_launch_dependent(
                    kern, dim3((unsigned)want, M), dim3(128), smem, p->stream, a, hf,
                    p->tmap_G, (const float *)p->d_G, (const int2 *)p->d_base,
                    (const float *)p->d_frac, (const int *)p->d_idx,
                    (const int *)p->d_bin_start, (const int *)p->d_task_bin,
                    (const int *)p->d_n_tasks, (const int *)p->d_pofs, (float *)values,
                    p->d_status, p->d_work);
            }
        }
        // plain loads: tile rows of at most 32 pairs
        if ((q.tile_x + WP) / 2 <= 32) {
            const int tw = q.tile_x + WP;
            const size_t per_field = sizeof(float) * (size_t)TH * tw;
            int fg = (int)((96 * 1024) / per_field);
            if (fg < 1) fg = 1;
            if (fg > a.F) fg = a.F;
            a.FG = fg;
            const size_t smem = per_field * fg;
            int per = (152 * 16 + M - 1) / M;
            if (per > p->nbins) per = p->nbins;
            if (per < 1) per = 1;
            cudaError_t e = dfs_allow_smem((const void *)k_interp_f32<W>, smem);
            if (e) return e;
            k_interp_f32<W><<<dim3(per, M), 128, smem, p->stream>>>(
                a, hf, (const float *)p->d_G, p->d_base, (const float *)p->d_frac, p->d_idx,
                p->d_bin_start, p->d_task_bin, p->d_n_tasks, p->d_pofs, (float *)values);
            return cudaGetLastError();
        }
    }
    const int tw = q.tile_x + W - 1;
    const size_t per_field = sizeof(R) * (size_t)(q.tile_y + W - 1) * tw;
    int fg = (int)((96 * 1024) / per_field);
    if (fg < 1) fg = 1;
    if (fg > a.F) fg = a.F;
    a.FG = fg;
    const size_t smem = per_field * fg;
    // blocks per member: enough to fill the GPU across all members
    int per = (152 * 16 + M - 1) / M;
    if (per > p->nbins) per = p->nbins;
    if (per < 1) per = 1;
    if constexpr (sizeof(R) == 8) {
        if (p->gdf) {
            HornerDF<W> hd;
            for (int i = 0; i < W; ++i)
                for (int kk = 0; kk <= W; ++kk) {
                    const double c = (double)hw.c[i][kk];
                    hd.hi[i][kk] = (float)c;
                    hd.lo[i][kk] = (float)(c - (double)hd.hi[i][kk]);
                }
            if (a.FG > DFS_DF_FG) a.FG = DFS_DF_FG;
            const size_t smem_df = per_field * a.FG;
            cudaError_t e = dfs_allow_smem((const void *)k_interp_df<W>, smem_df);
            if (e) return e;
            return dfs_launch_dependent(
                k_interp_df<W>, dim3(per, M), dim3(256), smem_df, p->stream, a, hd,
                (const float2 *)p->d_G, (const int2 *)p->d_base, (const double *)p->d_frac,
                (const int *)p->d_idx, (const int *)p->d_bin_start, (const int *)p->d_task_bin,
                (const int *)p->d_n_tasks, (const int *)p->d_pofs, (double *)values,
                (const int *)p->d_emax);
        }
    }
    cudaError_t e = dfs_allow_smem((const void *)k_interp<R, W>, smem);
    if (e) return e;
    const int threads = sizeof(R) == 4 ? 128 : 256;
    return dfs_launch_dependent(k_interp<R, W>, dim3(per, M), dim3(threads), smem, p->stream, a,
                                hw, (const R *)p->d_G, (const int2 *)p->d_base,
                                (const R *)p->d_frac, (const int *)p->d_idx,
                                (const int *)p->d_bin_start, (const int *)p->d_task_bin,
                                (const int *)p->d_n_tasks, (const int *)p->d_pofs, (R *)values);
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

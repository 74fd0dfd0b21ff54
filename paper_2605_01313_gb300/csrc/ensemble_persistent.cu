// One persistent launch for the transform and interpolation of a whole
// ensemble step: every group (members of one grid size) of an FP32 ensemble,
// its theta pass (deconvolve, pad and column FFTs), phi pass (complex-to-real
// row FFTs) and interpolation, drained by the resident CTAs from one device
// work queue (Sec. 5: the type-2 NUFFT evaluating Eq. 5.3, here for many
// fields and members of uneven grids at once).
//
// The queue lists the theta tasks of all groups, then their phi tasks, then
// their interpolation tasks; a CTA takes the next index with one atomicAdd.
// A phi task of group g waits until every theta task of g is done, an
// interpolation task until every phi task of g is done: per-group completion
// counters, each bumped after a task's stores (fence, then atomicAdd).  Every
// task a wait depends on has a smaller queue index, so it was taken earlier by
// a CTA that is already running and waits only on tasks before it: the waits
// end without any assumption on how many CTAs are resident.  Each wait is
// bounded (a cycle budget, about a second by default): one that runs out
// records DFS_STATUS_TIMEOUT and raises an abort flag, after which every CTA
// skips the remaining tasks and the launch ends.
//
// The transforms are the library's compile-time-length FFT engine: a theta task
// transforms CB columns (two half-length transforms each, as the TMA theta
// pass does) with 256 threads, a phi task CB row pairs; an interpolation task
// evaluates ENS_BINS consecutive bin slots of one member, each bin's tiles of
// all fields staged in shared memory by plain loads.  Data written earlier in
// the launch by other CTAs (the theta-pass buffer, the fine grid) is read
// through L2 only (ld.global.cg).
#include <string.h>

#include "coef_map.cuh"
#include "ensemble_persistent.cuh"
#include "fft_core.cuh"
#include "tma.cuh"

using namespace dfs_fft;
using namespace dfs_coef;

namespace {

constexpr int kThreads = ENS_THREADS;
constexpr int kE = DFS_FFT_E;

__device__ __forceinline__ float2 ldcg2(const float2 *p) { return __ldcg(p); }

// Wait (thread 0) until *ctr >= target, for at most `budget` cycles or until
// the abort flag rises.  Returns false on timeout or abort.
__device__ bool wait_counter(int *ctr, int target, int *ctl, long long budget) {
    const long long t0 = clock64();
    while (true) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        if (*(volatile int *)&ctl[ENS_ABORT]) return false;
        if (clock64() - t0 > budget) {
            atomicExch(&ctl[ENS_STATUS], DFS_STATUS_TIMEOUT);
            atomicExch(&ctl[ENS_ABORT], 1);
            return false;
        }
        __nanosleep(64);
    }
}

// ---- theta task: CB columns of one line, two half-length transforms each
template <int LOGH>
__device__ void theta_task(const EnsGroup &g, int line, int qb, unsigned char *smem) {
    typedef float2 C;
    constexpr int H = 1 << LOGH, TT = H / kE;
    constexpr int CB = kThreads / TT > 0 ? kThreads / TT : 1;
    const int c = threadIdx.x % CB;
    const int t = threadIdx.x / CB;
    C *sm0 = reinterpret_cast<C *>(smem) + (size_t)c * region_stride<C>(H, CB);
    C *sm1 = reinterpret_cast<C *>(smem) + (size_t)(CB + c) * region_stride<C>(H, CB);
    const int half = g.N2 / 2;
    const int q = qb * CB + c;
    const bool col_ok = q < g.tcols;
    const int qa = g.col_base + q;
    const float sq = col_ok ? __ldg(&g.inv1[qa < g.N1 ? qa : 0]) : 0.f;
    const C *cf0 = g.coef + (size_t)line * g.N2 * g.N1;
    const int2 rr = g.rowrange[line / g.F];
    C *dst = g.T + (size_t)line * g.n2 * g.tpitch + q;
    auto cf = [&](int r, int col) -> C {
        return (r < g.N2 && col < g.N1) ? __ldg(&cf0[(size_t)r * g.N1 + col])
                                        : make_float2(0.f, 0.f);
    };
    // deconvolved c_{n,m} (general plans) or h_{n,m} (real-field plans)
    auto coef_nm = [&](int n) -> C {
        const int r = n + half;
        const C v = g.herm ? herm_coef<C>(n, q, half, g.N1, cf) : cf(r, qa);
        return cscale(v, sq * __ldg(&g.inv2[r < g.N2 ? r : 0]));
    };
    // input i = t + e H/E of both halves: y_n and y_n e^{2 pi i n / n2}, the
    // twiddle being e^{2 pi i t / n2} e^{i pi e / E} (negated for n = i - H)
    const C wt = __ldg(&g.tw2[t]);
    auto ld2 = [&](int i, C &y0, C &y1) {
        y0 = y1 = make_float2(0.f, 0.f);
        if (!col_ok) return;
        const int e = (i - t) / TT;
        const C wi = cmul(wt, make_float2((float)c16(e * (8 / kE)), (float)s16(e * (8 / kE))));
        if (i < half) {
            const C y = coef_nm(i);
            y0 = y0 + y;
            y1 = y1 + cmul(y, wi);
        } else if (i >= H - half) {
            const C y = coef_nm(i - H);
            y0 = y0 + y;
            y1 = y1 - cmul(y, wi);
        }
        if (g.herm && i == half) {
            const C y = coef_nm(half);
            y0 = y0 + y;
            y1 = y1 + cmul(y, __ldg(&g.tw2[half]));
        }
    };
    auto needed = [&](int row) { return ((row - rr.x) & (g.n2 - 1)) < rr.y; };
    auto st2 = [&](int qq, C z0, C z1) {
        if (!col_ok) return;
        if (needed(2 * qq)) dst[(size_t)(2 * qq) * g.tpitch] = z0;
        if (needed(2 * qq + 1)) dst[(size_t)(2 * qq + 1) * g.tpitch] = z1;
    };
    auto none = [] {};
    line_fft_ct2<LOGH, kE>(g.stw_theta, sm0, sm1, t, ld2, st2, none);
}

// ---- phi task: NP row pairs of one line (complex-to-real row transforms)
template <int LOGM>
__device__ void phi_task(const EnsGroup &g, int line, int rb, unsigned char *smem) {
    typedef float2 C;
    constexpr int M = 1 << LOGM, T = M / kE;
    constexpr int NP = kThreads / T > 0 ? kThreads / T : 1;
    const int t = threadIdx.x % T;
    const int c = threadIdx.x / T;
    const int row = rb * 2 * NP + 2 * c;
    const int half = g.N1 / 2;
    const int nmask = g.n1 - 1;
    const C *src = g.T + ((size_t)line * g.n2 + row) * g.tpitch;
    float *dst = g.G + ((size_t)line * g.n2 + row) * g.n1;
    C *sm0 = reinterpret_cast<C *>(smem) + (size_t)(2 * c) * region_len<C>(M);
    C *sm1 = sm0 + region_len<C>(M);
    C *srow0 = reinterpret_cast<C *>(smem) + (size_t)(2 * NP) * region_len<C>(M) +
               (size_t)(2 * c) * g.tcols;
    C *srow1 = srow0 + g.tcols;
    for (int i = t; i < g.tcols; i += T) {
        srow0[i] = ldcg2(&src[i]);
        srow1[i] = ldcg2(&src[g.tpitch + i]);
    }
    __syncthreads();
    auto hval = [&](const C *sr, int k) -> C {
        k &= nmask;
        if (g.herm) {
            if (k <= half) return sr[k];
            if (k >= g.n1 - half) {
                const C v = sr[g.n1 - k];
                return make_float2(v.x, -v.y);
            }
            return make_float2(0.f, 0.f);
        }
        auto tv = [&](int kk) -> C {
            kk &= nmask;
            if (kk < half) return sr[kk + half];
            if (kk >= g.n1 - half) return sr[kk - g.n1 + half];
            return make_float2(0.f, 0.f);
        };
        const C p = tv(k), m = tv(-k);
        return make_float2(0.5f * (p.x + m.x), 0.5f * (p.y - m.y));
    };
    auto ld2 = [&](int k, C &z0, C &z1) {
        const C w = __ldg(&g.tw1[k]);
        const C a0 = hval(srow0, k), b0 = hval(srow0, k + M);
        const C a1 = hval(srow1, k), b1 = hval(srow1, k + M);
        const C d0 = cmul(make_float2(a0.x - b0.x, a0.y - b0.y), w);
        const C d1 = cmul(make_float2(a1.x - b1.x, a1.y - b1.y), w);
        z0 = make_float2(a0.x + b0.x - d0.y, a0.y + b0.y + d0.x);
        z1 = make_float2(a1.x + b1.x - d1.y, a1.y + b1.y + d1.x);
    };
    auto st2 = [&](int j, C z0, C z1) {
        reinterpret_cast<C *>(dst)[j] = z0;
        reinterpret_cast<C *>(dst + g.n1)[j] = z1;
    };
    auto none = [] {};
    line_fft_ct2<LOGM, kE>(g.stw_phi, sm0, sm1, t, ld2, st2, none);
}

// Weights by Horner's rule (degree W in s = t - mid), shifted by the parity of
// the first tap into WP paired weights (as the library's FP32 interpolation).
template <int W>
__device__ __forceinline__ void ens_weights(const float *hc, float tx, float ty, int odd,
                                            float *w8, float *wy) {
    constexpr int WP = (W + 2) & ~1;
    const float mid = (W % 2 == 0) ? 0.5f : 0.f;
    float wx[W];
#pragma unroll
    for (int a = 0; a < W; ++a) {
        float ax = hc[a * (W + 1) + W], ay = ax;
#pragma unroll
        for (int k = W - 1; k >= 0; --k) {
            ax = fmaf(ax, tx - mid, hc[a * (W + 1) + k]);
            ay = fmaf(ay, ty - mid, hc[a * (W + 1) + k]);
        }
        wx[a] = ax;
        wy[a] = ay;
    }
#pragma unroll
    for (int k = 0; k < WP; ++k) {
        const float lo = k < W ? wx[k] : 0.f;
        const float hi = (k >= 1 && k - 1 < W) ? wx[k - 1] : 0.f;
        w8[k] = odd ? hi : lo;
    }
}

// ---- interpolation task: ENS_BINS bin slots of one member, all fields
template <int W>
__device__ void interp_task(const EnsGroup &g, int member, int slot0, unsigned char *smem) {
    constexpr int WP = (W + 2) & ~1;
    float *tile = reinterpret_cast<float *>(smem);
    const int TH = g.tile_y + W - 1;
    const int TW = g.tile_x + WP;               // even: rows stay 8-byte aligned
    const int Q = TW / 2;
    const int tsz = TH * TW;
    const int p0 = g.pofs[member];
    const int Pk = g.pofs[member + 1] - p0;
    const int ntask = g.n_tasks[member];
    const int *task_bin = g.task_bin + (size_t)member * g.bstride;
    const int *bin_start = g.bin_start + (size_t)member * g.bstride;
    const float *hc = g.horner;
    for (int slot = slot0; slot < slot0 + ENS_BINS && slot < ntask; ++slot) {
        const int bin = task_bin[slot];
        const int by = bin / g.nbx;
        const int bx = bin - by * g.nbx;
        const int col0 = (bx * g.tile_x - g.c0) & ~1;
        const int row0 = by * g.tile_y - g.c0;
        const int s = p0 + bin_start[bin];
        const int e = p0 + bin_start[bin + 1];
        __syncthreads();                         // the previous bin's reads are done
        const int nq = g.F * TH * Q;
        for (int i = threadIdx.x; i < nq; i += kThreads) {
            const int rr = i / Q;
            const int qq = i - rr * Q;
            const int ff = rr / TH;
            const int r = rr - ff * TH;
            const int gr = (row0 + r) & (g.n2 - 1);
            const int gc = (col0 + 2 * qq) & (g.n1 - 1);
            *reinterpret_cast<float2 *>(tile + (size_t)ff * tsz + r * TW + 2 * qq) =
                ldcg2(reinterpret_cast<const float2 *>(
                    g.G + ((size_t)(member * g.F + ff) * g.n2 + gr) * g.n1 + gc));
        }
        __syncthreads();
        for (int pi = s + threadIdx.x; pi < e; pi += kThreads) {
            const int2 b = g.base[pi];
            const float2 tf = g.frac[pi];
            const int ox = b.x - col0;
            const int odd = ox & 1;
            float w8[WP], wy[W];
            ens_weights<W>(hc, tf.x, tf.y, odd, w8, wy);
            const int oy = b.y - row0;
            const int d = g.idx[pi];
            for (int ff = 0; ff < g.F; ++ff) {
                const float2 *tp = reinterpret_cast<const float2 *>(
                    tile + (size_t)ff * tsz + oy * TW + (ox - odd));
                float acc = 0.f;
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
                g.values[(size_t)g.F * p0 + (size_t)ff * Pk + d] = acc;
            }
        }
    }
}

template <int L, class Fn>
__device__ __forceinline__ void by_log(int l, Fn &&fn) {
    if constexpr (L <= ENS_MAX_LOG) {
        if (l == L) fn(std::integral_constant<int, L>());
        else by_log<L + 1>(l, fn);
    }
}

__global__ void __launch_bounds__(kThreads, 3) k_ensemble_step(const __grid_constant__ EnsArgs a,
                                                            int *__restrict__ ctl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_task, s_go;
    while (true) {
        if (threadIdx.x == 0) s_task = atomicAdd(&ctl[ENS_Q], 1);
        __syncthreads();
        const int task = s_task;
        if (task >= a.total) break;
        // stage and group of the task
        int stage = 0, gi = 0, local = task;
        for (stage = 0; stage < 3; ++stage) {
            bool found = false;
            for (gi = 0; gi < a.ngroups; ++gi) {
                const int n = a.g[gi].ntask[stage];
                if (local < n) {
                    found = true;
                    break;
                }
                local -= n;
            }
            if (found) break;
        }
        const EnsGroup &g = a.g[gi];
        if (threadIdx.x == 0) {
            bool go = !*(volatile int *)&ctl[ENS_ABORT];
            if (go && stage == 1) {
                const int target = g.ntask[0] + (gi == a.poison_group ? 1 : 0);
                go = wait_counter(&ctl[ENS_DONE_T + gi], target, ctl, a.budget);
            } else if (go && stage == 2) {
                go = wait_counter(&ctl[ENS_DONE_P + gi], g.ntask[1], ctl, a.budget);
            }
            s_go = go;
        }
        __syncthreads();
        if (s_go) {
            if (stage == 0) {
                const int line = local / g.nbq;
                by_log<ENS_MIN_LOG>(g.logh, [&](auto L) {
                    theta_task<decltype(L)::value>(g, line, local - line * g.nbq, smem);
                });
            } else if (stage == 1) {
                const int line = local / g.nrb;
                const int rb = local - line * g.nrb;
                // skip row blocks no stencil touches (the needed range is whole
                // DFS_ROW_BLOCK blocks)
                const int2 rr = g.rowrange[line / g.F];
                bool need = false;
                for (int r = rb * g.rows_per_phi; r < (rb + 1) * g.rows_per_phi; r += DFS_ROW_BLOCK)
                    need |= ((r - rr.x) & (g.n2 - 1)) < rr.y;
                if (need)
                    by_log<ENS_MIN_LOG>(g.logm, [&](auto L) {
                        phi_task<decltype(L)::value>(g, line, rb, smem);
                    });
            } else {
                const int member = local / g.nslot;
                const int slot0 = (local - member * g.nslot) * ENS_BINS;
                if (g.W == 6) interp_task<6>(g, member, slot0, smem);
                else interp_task<7>(g, member, slot0, smem);
            }
        }
        __syncthreads();                         // the task's stores are issued
        if (threadIdx.x == 0 && stage < 2) {
            __threadfence();
            atomicAdd(&ctl[(stage == 0 ? ENS_DONE_T : ENS_DONE_P) + gi], 1);
        }
    }
}

}  // namespace

size_t dfs_ensemble_step_smem(const EnsArgs &a) {
    size_t m = 0;
    for (int i = 0; i < a.ngroups; ++i) {
        const EnsGroup &g = a.g[i];
        const int H = 1 << g.logh, Mm = 1 << g.logm;
        const int cb = kThreads / (H / kE) > 0 ? kThreads / (H / kE) : 1;
        const int np = kThreads / (Mm / kE) > 0 ? kThreads / (Mm / kE) : 1;
        const size_t th = sizeof(float2) * 2 * (size_t)cb * region_len<float2>(H);
        const size_t ph = sizeof(float2) * 2 * (size_t)np * (region_len<float2>(Mm) + g.tcols);
        const int WP = (g.W + 2) & ~1;
        const size_t ip = sizeof(float) * (size_t)g.F * (g.tile_y + g.W - 1) * (g.tile_x + WP);
        m = th > m ? th : m;
        m = ph > m ? ph : m;
        m = ip > m ? ip : m;
    }
    return m;
}

cudaError_t dfs_ensemble_step_launch(const EnsArgs &a, int *ctl, int num_sms, cudaStream_t st,
                                     int *resident) {
    const size_t smem = dfs_ensemble_step_smem(a);
    cudaError_t e;
    if (*resident <= 0) {
        // first (uncaptured) launch: shared-memory limit and residency, kept
        // for the launches recorded in a graph later
        e = dfs_allow_smem((const void *)k_ensemble_step, smem);
        if (e) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ensemble_step, kThreads, smem);
        if (e) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
        *resident = occ;
    }
    int grid = num_sms * *resident;
    if (grid > a.total) grid = a.total;
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(ctl, 0, sizeof(int) * ENS_CTL_INTS, st);
    if (e) return e;
    k_ensemble_step<<<grid, kThreads, smem, st>>>(a, ctl);
    return cudaGetLastError();
}

// The persistent step's view of a group's batched plan, or false when the plan
// is not of a kind the step runs (FP32, points sorted, w 6 or 7, FFT lengths
// 2^ENS_MIN_LOG .. 2^ENS_MAX_LOG, at most 64 fields).
bool dfs_ensemble_group(dfsnufft_plan p, EnsGroup &g) {
    const dfsnufft_params &q = p->prm;
    if (q.dtype != DFSNUFFT_F32 || p->keep_order || p->gl || (q.w != 6 && q.w != 7) ||
        !p->d_stw_theta || !p->d_stw_phi)
        return false;
    const int logh = ilog2(q.n2) - 1, logm = ilog2(q.n1) - 1;
    if (logh < ENS_MIN_LOG || logh > ENS_MAX_LOG || logm < ENS_MIN_LOG || logm > ENS_MAX_LOG)
        return false;
    memset(&g, 0, sizeof(g));
    g.N1 = q.N1;
    g.N2 = q.N2;
    g.n1 = q.n1;
    g.n2 = q.n2;
    g.logh = logh;
    g.logm = logm;
    g.herm = p->herm;
    g.tcols = dfs_tcols(p->herm, q.N1);
    g.tpitch = dfs_tpitch(p->herm, q.N1);
    g.col_base = p->herm ? q.N1 / 2 : 0;
    g.members = p->n_members;
    g.F = p->n_fields;
    const int lines = g.members * g.F;
    const int cb = kThreads / ((1 << logh) / kE) > 0 ? kThreads / ((1 << logh) / kE) : 1;
    const int np = kThreads / ((1 << logm) / kE) > 0 ? kThreads / ((1 << logm) / kE) : 1;
    g.nbq = (g.tcols + cb - 1) / cb;
    g.rows_per_phi = 2 * np;
    g.nrb = q.n2 / g.rows_per_phi;
    g.nslot = (p->nbins + ENS_BINS - 1) / ENS_BINS;
    g.ntask[0] = lines * g.nbq;
    g.ntask[1] = lines * g.nrb;
    g.ntask[2] = g.members * g.nslot;
    g.tile_x = q.tile_x;
    g.tile_y = q.tile_y;
    g.nbx = p->nbx;
    g.bstride = p->bstride;
    g.c0 = p->c0;
    g.W = q.w;
    double hc[8 * 9];
    dfsnufft_es_horner(q.w, q.beta, hc);
    for (int i = 0; i < q.w * (q.w + 1); ++i) g.horner[i] = (float)hc[i];
    g.inv1 = (const float *)p->d_inv1;
    g.inv2 = (const float *)p->d_inv2;
    g.tw1 = (const float2 *)p->d_tw1;
    g.tw2 = (const float2 *)p->d_tw2;
    g.stw_theta = (const float2 *)p->d_stw_theta;
    g.stw_phi = (const float2 *)p->d_stw_phi;
    g.T = (float2 *)p->d_T;
    g.G = (float *)p->d_G;
    g.rowrange = p->d_rowrange;
    g.bin_start = p->d_bin_start;
    g.task_bin = p->d_task_bin;
    g.n_tasks = p->d_n_tasks;
    g.pofs = p->d_pofs;
    return true;
}

// Point records of the group's plan as they stand (set_points may reallocate
// them when the point count grows).
void dfs_ensemble_group_points(dfsnufft_plan p, EnsGroup &g) {
    g.base = p->d_base;
    g.frac = (const float2 *)p->d_frac;
    g.idx = p->d_idx;
}

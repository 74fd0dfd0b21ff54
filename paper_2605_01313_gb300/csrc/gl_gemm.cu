// The latitude solve of the Gauss-Legendre form (Sec. 5, interpolation for the
// spherical-harmonic model: the inversion of the DFT matrix of the doubled
// column, split by parity into two real n_lat x n_lat systems whose inverses
// the plan forms once): for each class c, O_c = M_c G_c, with M_c the N x N
// inverse (row-major) and G_c the N x cols row spectra (row-major), in FP32 on
// the fifth-generation tensor cores (tcgen05.mma, kind::tf32).
//
// FP32 accuracy from TF32 products (10-bit significands) by splitting both
// operands: x = x_hi + x_lo with x_hi = x rounded to TF32 and x_lo = (x - x_hi)
// rounded to TF32, so that x_hi + x_lo is x to about 2^-22 relative.  Then
// M G = M_hi G_hi + M_hi G_lo + M_lo G_hi up to the product M_lo G_lo, of
// relative size 2^-22 per term with signs that cancel over K; the three
// products are exact in the tensor core.  The tensor core accumulates in FP32;
// so that its rounding does not grow with the full depth K, tensor memory
// accumulates groups of GROUP K tiles (K = 128) only, two accumulators taking
// turns, and each group's sums are added into FP32 registers while the next
// group runs.  M_hi and M_lo are formed on the host (the matrices are the
// plan's); G is split on the fly.
//
// The tensor core computes the transpose, O^T = G^T M^T, in 128 x 128 tiles:
// the A operand is the split G tile (128 columns of G x 32 k), held in tensor
// memory, where the threads that split it store it directly (no shared-memory
// traffic); the B operand is the M tile (128 rows of M x 32 k, K-major,
// 128-byte swizzle), loaded by TMA.  Accumulator lane n is then column j0 + n
// of O, so that the stores of a warp are coalesced.  The kernel is persistent
// (launched as a dependent of the longitude pass, which it waits for first):
// one CTA per multiprocessor takes output tiles blockIdx.x, blockIdx.x +
// gridDim.x, ..., and its rings and accumulators run on across the tiles, so
// that one tile's last sums are stored while the next one's products run.  K
// runs in tiles of 32 through three rings, deep enough to cover the latency of
// the L2: NM stages of M_hi, M_lo (shared memory), NR stages of raw G tiles
// (32 k x 128 columns, shared memory) and NT stages of G_hi, G_lo (tensor
// memory).  The warps have one job each:
//   warps 0-3   (drain) add each finished accumulator group into registers
//               (`accfull` -> `accempty`) and at the end store the sums;
//   warps 4-7   (producers) read their column of the raw G tile (`rawfull` ->
//               `rawempty`) and, once the MMAs that read the tensor-memory stage
//               are done (`emptyT`), split it into the stage's G_hi and G_lo
//               columns (`fullT`);
//   warp 8      one thread issues the tile's twelve MMAs (four K slices of 8,
//               three products) once `fullM` and `fullT` complete, and commits
//               them to `emptyM` and `emptyT` (and to `accfull` at the end of a
//               group);
//   warp 9      one thread loads M_hi and M_lo tiles by TMA (`emptyM` -> `fullM`);
//   warp 10     one thread loads raw G tiles by TMA (`rawempty` -> `rawfull`).
// Every wait is bounded (about a second) and also ends once another thread of
// the CTA, or another CTA, has given up; then the CTA records
// DFS_STATUS_TIMEOUT, waits (bounded) for its copies and MMAs in flight, frees
// the tensor memory and returns.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "tma.cuh"

namespace {

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int THREADS = 352;                          // 4 drain, 4 producer, MMA, 2 TMA warps
constexpr int TILE = BM * BK * 4;                     // bytes of one 128 x 32 FP32 tile
constexpr int NM = 4, NR = 6, NT = 4;                 // stages: M tiles, raw G tiles, split G
constexpr int GROUP = 4;                              // K tiles per accumulation group
constexpr int MBYTES = NM * 2 * TILE, RBYTES = NR * TILE;
constexpr int SMEM = 1024 + MBYTES + RBYTES + 256;    // alignment slack, rings, barriers
static_assert(SMEM <= 232448, "shared memory of one CTA");
// tensor memory: accumulators at columns 0 and BN, stage s's G_hi at
// ACOL + 2 BK s and G_lo BK further
constexpr int ACOL = 2 * BN, TMEM_COLS = 512;
static_assert(ACOL + NT * 2 * BK <= TMEM_COLS, "tensor memory columns");

// Shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle:
// start address >> 4, leading offset 16 B (unused for this layout), stride
// 1024 B between 8-row groups, descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

// D (tensor memory) (+)= A (tensor memory, lane m = row m, column k) x B (shared)
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                            uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

// mbarrier.try_wait with a suspend-time hint: the thread sleeps until the
// phase completes (or about 0.1 ms pass) instead of polling shared memory,
// where the tensor core reads its B operand.
__device__ __forceinline__ bool try_wait_sleep(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// x rounded to TF32 (10 explicit significand bits), ties away from zero, as
// FP32 bits: half a unit of the 13 dropped bits added to the magnitude, which
// carries into the exponent where it must; finite inputs only.
__device__ __forceinline__ uint32_t tf32_bits(float x) {
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

// acc[u] += accumulator columns col..col+15 of this thread's lane.
__device__ __forceinline__ void tmem_add16(uint32_t taddr, float *acc) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] += __uint_as_float(v[u]);
}

// Columns col..col+31 of this thread's lane = v[0..31].
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
        "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
        "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

struct Bars {
    uint64_t fullM[NM], emptyM[NM], rawfull[NR], rawempty[NR], fullT[NT], emptyT[NT];
    uint64_t accfull[2], accempty[2];
    uint32_t tmem;
    int abort, issuedM, issuedG, committed;   // CTA gave up; M, G tiles loaded; tiles whose
                                              // MMAs were committed
};

// grid: at most one CTA per output tile (ceil(cols / 128) x ceil(N / 128) x 2
// classes), THREADS threads.  mapM_hi, mapM_lo: (N k, N rows, 2 classes), box 32 x 128 x 1, 128-byte
// swizzle.  mapG: G as (cols, N, 2 classes), box 128 x 32 x 1, no swizzle.
// out: 2 x N x cols, class c at c * N * cols.
__global__ void __launch_bounds__(THREADS, 1) k_gl_gemm(const __grid_constant__ CUtensorMap mapM_hi,
                                                         const __grid_constant__ CUtensorMap mapM_lo,
                                                         const __grid_constant__ CUtensorMap mapG,
                                                         float *__restrict__ out, int N, int cols,
                                                         int *__restrict__ status) {
    dfs_grid_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    Bars &B = *reinterpret_cast<Bars *>(base + MBYTES + RBYTES);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int KT = (N + BK - 1) / BK, NG = (KT + GROUP - 1) / GROUP;   // per output tile
    const int ntj = (cols + BN - 1) / BN, nti = (N + BM - 1) / BM, ntiles = 2 * nti * ntj;
    // output tile -> class, first row, first column (tiles of one row band
    // consecutive, so that CTAs running together share M tiles in the L2)
    auto tile_of = [&](int tile, int &cls, int &i0, int &j0) {
        cls = tile / (nti * ntj);
        const int rem = tile - cls * nti * ntj;
        i0 = (rem / ntj) * BM;
        j0 = (rem % ntj) * BN;
    };
    // M stage s, part q: 0 M_hi, 1 M_lo; raw G stage r
    auto part = [&](int s, int q) { return base + (size_t)(s * 2 + q) * TILE; };
    auto raw = [&](int r) { return reinterpret_cast<float *>(base + MBYTES + (size_t)r * TILE); };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&B.tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 256) {
        for (int s = 0; s < NM; ++s) {
            mbar_init(&B.fullM[s], 1);
            mbar_init(&B.emptyM[s], 1);
        }
        for (int r = 0; r < NR; ++r) {
            mbar_init(&B.rawfull[r], 1);
            mbar_init(&B.rawempty[r], 128);
        }
        for (int s = 0; s < NT; ++s) {
            mbar_init(&B.fullT[s], 128);
            mbar_init(&B.emptyT[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&B.accfull[a], 1);
            mbar_init(&B.accempty[a], 128);
        }
        B.abort = 0;
        B.issuedM = 0;
        B.issuedG = 0;
        B.committed = 0;
        fence_mbar_init();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = B.tmem;
    volatile int *vabort = &B.abort;

    // bounded wait that also ends when this CTA gave up, or, once it has lasted
    // about a million cycles, when another CTA did (the status word is global
    // memory: read on every turn it would delay the wake-up by its latency)
    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (try_wait_sleep(bar, parity)) return true;
        const long long t0 = clock64();
        while (!try_wait_sleep(bar, parity)) {
            if (*vabort) return false;
            const long long dt = clock64() - t0;
            if (dt > (1LL << 20) && *(volatile int *)status == DFS_STATUS_TIMEOUT) {
                *vabort = 1;
                return false;
            }
            if (dt > DFS_WAIT_CYCLES) {
                *vabort = 1;
                atomicExch(status, DFS_STATUS_TIMEOUT);
                return false;
            }
        }
        return true;
    };

    if (warp < 4) {
        // ---- drain: the accumulator groups into registers, then the store ----
        const uint32_t trow = (uint32_t)(32 * warp) << 16;
        bool ok = true;
        for (int tile = blockIdx.x, lt = 0; tile < ntiles && ok; tile += gridDim.x, ++lt) {
            int cls, i0, j0;
            tile_of(tile, cls, i0, j0);
            float acc[BM];
#pragma unroll
            for (int u = 0; u < BM; ++u) acc[u] = 0.f;
            for (int gl = 0; gl < NG; ++gl) {
                const int gi = lt * NG + gl;
                if (!__all_sync(0xffffffffu, wait(&B.accfull[gi & 1], (gi >> 1) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int q = 0; q < BM / 16; ++q)
                    tmem_add16(tmem + trow + (uint32_t)((gi & 1) * BN + 16 * q), acc + 16 * q);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&B.accempty[gi & 1]);
            }
            // lane n of the accumulator is column j0 + n of O, column u row i0 + u
            const int j = j0 + tid;
            if (ok && j < cols) {
                float *o = out + ((size_t)cls * N + i0) * cols + j;
                const int rows = N - i0 < BM ? N - i0 : BM;
#pragma unroll
                for (int u = 0; u < BM; ++u)
                    if (u < rows) o[(size_t)u * cols] = acc[u];
            }
        }
    } else if (warp < 8) {
        // ---- producers: raw G column -> G_hi, G_lo in tensor memory ----
        const int n = tid - 128;
        const uint32_t trow = (uint32_t)(32 * (warp - 4)) << 16;   // lane n
        const int its = ((ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x) * KT;
        for (int it = 0; it < its; ++it) {
            const int r = it % NR, s = it % NT;
            if (!__all_sync(0xffffffffu, wait(&B.rawfull[r], (it / NR) & 1))) break;
            float gp[BK];
            const float *src = raw(r) + n;
#pragma unroll
            for (int q = 0; q < BK; ++q) gp[q] = src[q * BN];
            mbar_arrive(&B.rawempty[r]);
            if (it >= NT && !__all_sync(0xffffffffu, wait(&B.emptyT[s], ((it - NT) / NT) & 1)))
                break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t h[BK], l[BK];
#pragma unroll
            for (int q = 0; q < BK; ++q) {
                h[q] = tf32_bits(gp[q]);
                l[q] = tf32_bits(gp[q] - __uint_as_float(h[q]));   // exact difference
            }
            const uint32_t col = tmem + trow + (uint32_t)(ACOL + 2 * BK * s);
            tmem_st32(col, h);
            tmem_st32(col + BK, l);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&B.fullT[s]);
        }
    } else if (tid == 256) {
        // ---- MMA issue ----
        bool ok = true;
        for (int tile = blockIdx.x, lt = 0; tile < ntiles && ok; tile += gridDim.x, ++lt)
            for (int t = 0; t < KT; ++t) {
                const int it = lt * KT + t, gi = lt * NG + t / GROUP;
                const int sm = it % NM, st = it % NT;
                if (t % GROUP == 0 && gi >= 2 &&
                    !wait(&B.accempty[gi & 1], ((gi - 2) >> 1) & 1)) {
                    ok = false;
                    break;
                }
                if (!wait(&B.fullM[sm], (it / NM) & 1) || !wait(&B.fullT[st], (it / NT) & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)((gi & 1) * BN);
                const uint32_t gh = tmem + (uint32_t)(ACOL + 2 * BK * st), gl = gh + BK;
                const uint32_t mh = smem_u32(part(sm, 0)), ml = smem_u32(part(sm, 1));
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {
                    const uint32_t o = kk * 32;                  // 8 TF32 = 32 bytes of K
                    // the small products first; a group's first MMA overwrites
                    mma_tf32_ts(d, gh + 8 * kk, desc_sw128(ml + o),
                                (t % GROUP != 0 || kk > 0) ? 1u : 0u);
                    mma_tf32_ts(d, gl + 8 * kk, desc_sw128(mh + o), 1u);
                    mma_tf32_ts(d, gh + 8 * kk, desc_sw128(mh + o), 1u);
                }
                mma_commit(&B.emptyM[sm]);
                mma_commit(&B.emptyT[st]);
                if (t % GROUP == GROUP - 1 || t == KT - 1) mma_commit(&B.accfull[gi & 1]);
                B.committed = it + 1;
            }
    } else if (tid == 288) {
        // ---- TMA loads of M_hi, M_lo ----
        bool ok = true;
        for (int tile = blockIdx.x, lt = 0; tile < ntiles && ok; tile += gridDim.x, ++lt) {
            int cls, i0, j0;
            tile_of(tile, cls, i0, j0);
            for (int t = 0; t < KT; ++t) {
                const int it = lt * KT + t, s = it % NM;
                if (it >= NM && !wait(&B.emptyM[s], ((it - NM) / NM) & 1)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&B.fullM[s], 2 * TILE);
                tma_load_3d(part(s, 0), &mapM_hi, t * BK, i0, cls, &B.fullM[s]);
                tma_load_3d(part(s, 1), &mapM_lo, t * BK, i0, cls, &B.fullM[s]);
                B.issuedM = it + 1;
            }
        }
    } else if (tid == 320) {
        // ---- TMA loads of raw G tiles (zero outside N x cols) ----
        bool ok = true;
        for (int tile = blockIdx.x, lt = 0; tile < ntiles && ok; tile += gridDim.x, ++lt) {
            int cls, i0, j0;
            tile_of(tile, cls, i0, j0);
            for (int t = 0; t < KT; ++t) {
                const int it = lt * KT + t, r = it % NR;
                if (it >= NR && !wait(&B.rawempty[r], ((it - NR) / NR) & 1)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&B.rawfull[r], TILE);
                tma_load_3d(raw(r), &mapG, j0, t * BK, cls, &B.rawfull[r]);
                B.issuedG = it + 1;
            }
        }
    }
    __syncthreads();
    if (tid == 256 && B.abort) {
        // after giving up: the copies and MMAs in flight land before the CTA leaves
        const int c = B.committed, im = B.issuedM, ig = B.issuedG;
        if (c > 0) mbar_wait_bounded(&B.emptyM[(c - 1) % NM], ((c - 1) / NM) & 1);
        for (int t = im - NM > 0 ? im - NM : 0; t < im; ++t)
            mbar_wait_bounded(&B.fullM[t % NM], (t / NM) & 1);
        for (int t = ig - NR > 0 ? ig - NR : 0; t < ig; ++t)
            mbar_wait_bounded(&B.rawfull[t % NR], (t / NR) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

// Host: the split matrices M_hi, M_lo (2 classes of N x N each, FP32) from the
// FP64 inverses (already scaled), and the tensor maps of the GEMM.
int dfs_gl_tc_setup(dfsnufft_plan p, const double *cm, const double *sm, int N) {
    const size_t nn = (size_t)N * N;
    float *h = (float *)malloc(sizeof(float) * 4 * nn);
    if (!h) return DFSNUFFT_ERR_OOM;
    const double *src[2] = {cm, sm};
    for (int c = 0; c < 2; ++c)
        for (size_t i = 0; i < nn; ++i) {
            const double x = src[c][i];
            // round to TF32 as the kernel does (10 explicit significand bits,
            // ties away from zero)
            const float xf = (float)x;
            uint32_t b;
            memcpy(&b, &xf, 4);
            b = (b + 0x1000u) & 0xFFFFE000u;
            float hi;
            memcpy(&hi, &b, 4);
            h[c * nn + i] = hi;                                   // M_hi, class c
            const float lo = (float)(x - (double)hi);             // the rest, rounded to TF32
            memcpy(&b, &lo, 4);
            b = (b + 0x1000u) & 0xFFFFE000u;
            memcpy(&h[2 * nn + c * nn + i], &b, 4);               // M_lo, class c
        }
    if (cudaMalloc(&p->d_gl_tc, sizeof(float) * 4 * nn) != cudaSuccess) {
        cudaGetLastError();
        p->d_gl_tc = nullptr;
        free(h);
        return DFSNUFFT_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(p->d_gl_tc, h, sizeof(float) * 4 * nn, cudaMemcpyHostToDevice);
    free(h);
    if (e) return DFSNUFFT_ERR_CUDA;
    const uint64_t dims[3] = {(uint64_t)N, (uint64_t)N, 2};
    const uint64_t str[2] = {(uint64_t)N * 4, (uint64_t)nn * 4};
    const uint32_t box[3] = {BK, BM, 1};
    const float *a = (const float *)p->d_gl_tc;
    if (dfs_encode_tensor_map_3d_f32(&p->tmap_gl_hi, a, dims, str, box, 1) ||
        dfs_encode_tensor_map_3d_f32(&p->tmap_gl_lo, a + 2 * nn, dims, str, box, 1))
        return DFSNUFFT_ERR_UNSUPPORTED;
    return DFSNUFFT_OK;
}

// O_c = M_c G_c for both classes: g is 2 x N x cols FP32 (rows of G, cols a
// multiple of 4 and g 16-byte aligned, as TMA requires), out the same shape.
cudaError_t dfs_gl_tc_gemm(dfsnufft_plan p, const float *g, float *out, int N, int cols) {
    cudaError_t e = dfs_allow_smem((const void *)k_gl_gemm, SMEM);
    if (e) return e;
    CUtensorMap mapG;
    const uint64_t dims[3] = {(uint64_t)cols, (uint64_t)N, 2};
    const uint64_t str[2] = {(uint64_t)cols * 4, (uint64_t)N * cols * 4};
    const uint32_t box[3] = {BN, BK, 1};
    if (dfs_encode_tensor_map_3d_f32(&mapG, g, dims, str, box, 0)) return cudaErrorInvalidValue;
    const int ntiles = 2 * ((N + BM - 1) / BM) * ((cols + BN - 1) / BN);
    const int grid = ntiles < p->num_sms ? ntiles : p->num_sms;
    return dfs_launch_dependent(k_gl_gemm, dim3(grid), dim3(THREADS), SMEM, p->stream,
                                p->tmap_gl_hi, p->tmap_gl_lo, mapG, out, N, cols, p->d_status);
}

// Arguments of the persistent ensemble step (ensemble_persistent.cu), filled by
// the ensemble (ensemble.cu) from its groups' batched plans.
#pragma once

#include <type_traits>

#include "common.cuh"

#define ENS_MAXG 16            // groups a persistent step takes
#define ENS_THREADS 256        // threads of its CTAs
#define ENS_BINS 8             // bin slots of one interpolation task
#define ENS_MIN_LOG 7          // half fine lengths n/2 from 2^7 ...
#define ENS_MAX_LOG 11         // ... to 2^11

// Control words (device ints, zeroed before each launch): queue head, status
// word, abort flag, then per group the theta and phi tasks done.
#define ENS_Q 0
#define ENS_STATUS 1
#define ENS_ABORT 2
#define ENS_DONE_T 4
#define ENS_DONE_P (4 + ENS_MAXG)
#define ENS_CTL_INTS (4 + 2 * ENS_MAXG)

struct EnsGroup {
    int N1, N2, n1, n2, logh, logm;   // logh = log2(n2 / 2), logm = log2(n1 / 2)
    int herm, tcols, tpitch, col_base;
    int members, F;
    int nbq;                          // theta tasks (column blocks) per line
    int nrb, rows_per_phi;            // phi tasks (row blocks) per line, rows each
    int nslot;                        // interpolation tasks per member
    int ntask[3];                     // theta, phi and interpolation tasks
    int tile_x, tile_y, nbx, bstride, c0, W;
    float horner[8 * 9];              // kernel weights, dfsnufft_es_horner in FP32
    const float *inv1, *inv2;         // 1 / phihat (plan precision)
    const float2 *tw1, *tw2;          // twiddles of lengths n1 and n2
    const float2 *stw_theta, *stw_phi;   // stage-ordered tables (n2 / 2, n1 / 2)
    float2 *T;                        // theta-pass buffer
    float *G;                         // fine grids
    const int2 *rowrange;
    const int *bin_start, *task_bin, *n_tasks, *pofs;
    const int2 *base;                 // sorted point records
    const float2 *frac;
    const int *idx;
    const float2 *coef;               // this step's coefficients and values
    float *values;
};

struct EnsArgs {
    int ngroups, total;               // groups, tasks of all stages
    long long budget;                 // cycles a dependency wait may last
    int poison_group;                 // self-test: this group's theta target is one too
                                      // high (a wait that cannot end); -1: none
    EnsGroup g[ENS_MAXG];
};

bool dfs_ensemble_group(dfsnufft_plan p, EnsGroup &g);
void dfs_ensemble_group_points(dfsnufft_plan p, EnsGroup &g);
size_t dfs_ensemble_step_smem(const EnsArgs &a);
// resident: CTAs per SM, found on the first launch (*resident <= 0) and kept
cudaError_t dfs_ensemble_step_launch(const EnsArgs &a, int *ctl, int num_sms, cudaStream_t st,
                                     int *resident);

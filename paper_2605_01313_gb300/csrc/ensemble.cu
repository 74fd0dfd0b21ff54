// Ensembles of members on uneven grids: one batched plan per grid size, each
// on its own stream, and one CUDA graph per step.  The step (points and values
// of every member of every group) is recorded by stream capture as a fork/join
// over the group streams, so the groups' kernels overlap on the device, and is
// replayed with one graph launch while the caller's pointers and point counts
// stay the same; when they change, the step runs once uncaptured (it may
// allocate or upload offsets) and is recorded again.
//
// In persistent mode (dfsnufft_ensemble_set_persistent) the groups' set_points
// still run as the graph's fork/join branches, and the transform and
// interpolation of every group then run as one persistent launch that drains a
// device work queue (ensemble_persistent.cu), recorded in the same graph.
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"
#include "ensemble_persistent.cuh"
#include "tma.cuh"

struct dfsnufft_ensemble_s {
    int n_groups;
    int n_fields;
    cudaStream_t stream;                 // caller's stream: the graph runs here
    cudaStream_t origin;                 // recording stream (the legacy stream cannot be captured)
    std::vector<dfsnufft_plan> plans;
    std::vector<cudaStream_t> streams;   // one per group
    std::vector<cudaEvent_t> done;       // group -> main joins
    cudaEvent_t fork;
    cudaGraphExec_t exec;
    // signature of the recorded step
    std::vector<const void *> sig_ptr;
    std::vector<int64_t> sig_counts;
    int status;
    // persistent mode
    int persistent;
    int *d_ctl;                          // the step's control words (ENS_CTL_INTS)
    EnsArgs *args;                       // the groups' views; per-step pointers filled by the step
    int args_ready;                      // args hold a complete step (for the self-test)
    int num_sms;
    int resident;                        // CTAs per SM of the persistent step (0: unknown)
};

namespace {

int ens_fail(dfsnufft_ensemble e, int code) {
    if (!e->status) e->status = code;
    return code;
}

// The step, enqueued on the group streams after a fork from `main` and joined
// back into it; in persistent mode the groups' branches only set their points,
// and one launch on `main` does the rest.
int enqueue_step(dfsnufft_ensemble e, cudaStream_t main, const int64_t *const *counts,
                 const double *const *lon, const double *const *colat, const void *const *coeffs,
                 void *const *values) {
    if (cudaEventRecord(e->fork, main)) return DFSNUFFT_ERR_CUDA;
    for (int g = 0; g < e->n_groups; ++g) {
        if (cudaStreamWaitEvent(e->streams[g], e->fork, 0)) return DFSNUFFT_ERR_CUDA;
        int rc = dfsnufft_set_points_batch(e->plans[g], counts[g], lon[g], colat[g]);
        if (rc) return rc;
        if (!e->persistent) {
            rc = dfsnufft_execute(e->plans[g], coeffs[g], values[g]);
            if (rc) return rc;
        }
        if (cudaEventRecord(e->done[g], e->streams[g])) return DFSNUFFT_ERR_CUDA;
        if (cudaStreamWaitEvent(main, e->done[g], 0)) return DFSNUFFT_ERR_CUDA;
    }
    if (!e->persistent) return DFSNUFFT_OK;
    EnsArgs &a = *e->args;
    a.total = 0;
    for (int g = 0; g < e->n_groups; ++g) {
        dfs_ensemble_group_points(e->plans[g], a.g[g]);     // set_points may reallocate
        a.g[g].coef = static_cast<const float2 *>(coeffs[g]);
        a.g[g].values = static_cast<float *>(values[g]);
        a.total += a.g[g].ntask[0] + a.g[g].ntask[1] + a.g[g].ntask[2];
    }
    a.budget = DFS_WAIT_CYCLES;
    a.poison_group = -1;
    e->args_ready = 1;
    if (dfs_ensemble_step_launch(a, e->d_ctl, e->num_sms, main, &e->resident))
        return DFSNUFFT_ERR_CUDA;
    return DFSNUFFT_OK;
}

void release(dfsnufft_ensemble e) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    for (auto p : e->plans)
        if (p) dfsnufft_destroy(p);
    for (auto s : e->streams)
        if (s) cudaStreamDestroy(s);
    for (auto v : e->done)
        if (v) cudaEventDestroy(v);
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->origin) cudaStreamDestroy(e->origin);
    if (e->d_ctl) cudaFree(e->d_ctl);
    delete e->args;
}

}  // namespace

extern "C" int dfsnufft_ensemble_create(int n_groups, const int *n_members, const int *n_lon,
                                        const int *n_lat, double tol, int dtype, int n_fields,
                                        void *stream, dfsnufft_ensemble *out) {
    return dfsnufft_ensemble_create_opts(n_groups, n_members, n_lon, n_lat, tol, dtype, n_fields,
                                         nullptr, stream, out);
}

extern "C" int dfsnufft_ensemble_create_opts(int n_groups, const int *n_members,
                                             const int *n_lon, const int *n_lat, double tol,
                                             int dtype, int n_fields,
                                             const dfsnufft_options *opts, void *stream,
                                             dfsnufft_ensemble *out) {
    if (!out || n_groups < 1 || n_groups > 64 || !n_members || !n_lon || !n_lat)
        return DFSNUFFT_ERR_INVALID_ARG;
    *out = nullptr;
    dfsnufft_ensemble e = new (std::nothrow) dfsnufft_ensemble_s();
    if (!e) return DFSNUFFT_ERR_OOM;
    e->n_groups = n_groups;
    e->n_fields = n_fields;
    e->stream = (cudaStream_t)stream;
    e->exec = nullptr;
    e->fork = nullptr;
    e->origin = nullptr;
    e->status = 0;
    e->persistent = 0;
    e->d_ctl = nullptr;
    e->args = nullptr;
    e->args_ready = 0;
    e->num_sms = 0;
    e->resident = 0;
    e->plans.assign(n_groups, nullptr);
    e->streams.assign(n_groups, nullptr);
    e->done.assign(n_groups, nullptr);
    int rc = DFSNUFFT_OK;
    if (cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) ||
        cudaStreamCreateWithFlags(&e->origin, cudaStreamNonBlocking))
        rc = DFSNUFFT_ERR_CUDA;
    for (int g = 0; g < n_groups && !rc; ++g) {
        if (cudaStreamCreateWithFlags(&e->streams[g], cudaStreamNonBlocking) ||
            cudaEventCreateWithFlags(&e->done[g], cudaEventDisableTiming)) {
            rc = DFSNUFFT_ERR_CUDA;
            break;
        }
        rc = dfsnufft_plan_create_opts(n_members[g], n_lon[g], n_lat[g], tol, dtype, n_fields,
                                       opts ? &opts[g] : nullptr, e->streams[g], &e->plans[g]);
    }
    if (rc) {
        release(e);
        delete e;
        return rc;
    }
    *out = e;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_ensemble_run(dfsnufft_ensemble e, const int64_t *const *n_points,
                                     const double *const *lon, const double *const *colat,
                                     const void *const *coeffs, void *const *values) {
    if (!e || !n_points || !lon || !colat || !coeffs || !values) return DFSNUFFT_ERR_INVALID_ARG;
    if (e->status) return e->status;
    // signature: every pointer and every member count
    std::vector<const void *> ptr;
    std::vector<int64_t> counts;
    for (int g = 0; g < e->n_groups; ++g) {
        if (!n_points[g] || !lon[g] || !colat[g] || !coeffs[g] || !values[g])
            return DFSNUFFT_ERR_INVALID_ARG;
        ptr.push_back(lon[g]);
        ptr.push_back(colat[g]);
        ptr.push_back(coeffs[g]);
        ptr.push_back(values[g]);
        for (int k = 0; k < e->plans[g]->n_members; ++k) counts.push_back(n_points[g][k]);
    }
    if (e->exec && ptr == e->sig_ptr && counts == e->sig_counts) {
        if (cudaGraphLaunch(e->exec, e->stream)) return ens_fail(e, DFSNUFFT_ERR_CUDA);
        return DFSNUFFT_OK;
    }
    // new shape of step: run it once as is, then record it on the origin stream
    int rc = enqueue_step(e, e->stream, n_points, lon, colat, coeffs, values);
    if (rc) return ens_fail(e, rc);
    if (e->exec) {
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    // the recording stream starts after this run's step (the groups' streams
    // are reused by the recording)
    if (cudaEventRecord(e->fork, e->stream) || cudaStreamWaitEvent(e->origin, e->fork, 0))
        return ens_fail(e, DFSNUFFT_ERR_CUDA);
    if (cudaStreamBeginCapture(e->origin, cudaStreamCaptureModeThreadLocal))
        return ens_fail(e, DFSNUFFT_ERR_CUDA);
    rc = enqueue_step(e, e->origin, n_points, lon, colat, coeffs, values);
    cudaError_t ce = cudaStreamEndCapture(e->origin, &graph);
    if (rc || ce) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return ens_fail(e, rc ? rc : DFSNUFFT_ERR_CUDA);
    }
    ce = cudaGraphInstantiate(&e->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce) {
        e->exec = nullptr;
        return ens_fail(e, DFSNUFFT_ERR_CUDA);
    }
    e->sig_ptr = ptr;
    e->sig_counts = counts;
    return DFSNUFFT_OK;
}

// The persistent step's status word, after synchronising the ensemble's stream.
static int read_ctl_status(dfsnufft_ensemble e) {
    int st = 0;
    if (cudaStreamSynchronize(e->stream) ||
        cudaMemcpy(&st, e->d_ctl + ENS_STATUS, sizeof(int), cudaMemcpyDeviceToHost))
        return DFSNUFFT_ERR_CUDA;
    return st ? DFSNUFFT_ERR_TIMEOUT : DFSNUFFT_OK;
}

extern "C" int dfsnufft_ensemble_check(dfsnufft_ensemble e) {
    if (!e) return DFSNUFFT_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(e->stream)) return ens_fail(e, DFSNUFFT_ERR_CUDA);
    for (auto p : e->plans) {
        int rc = dfsnufft_plan_check(p);
        if (rc) return ens_fail(e, rc);
    }
    if (e->persistent && e->d_ctl) {
        int rc = read_ctl_status(e);
        if (rc) return ens_fail(e, rc);
    }
    return e->status;
}

extern "C" int dfsnufft_ensemble_set_persistent(dfsnufft_ensemble e, int on) {
    if (!e) return DFSNUFFT_ERR_INVALID_ARG;
    if (e->status) return e->status;
    if (on) {
        if (e->n_groups > ENS_MAXG) return DFSNUFFT_ERR_UNSUPPORTED;
        EnsArgs *a = e->args ? e->args : new (std::nothrow) EnsArgs();
        if (!a) return DFSNUFFT_ERR_OOM;
        e->args = a;
        memset(a, 0, sizeof(*a));
        a->ngroups = e->n_groups;
        for (int g = 0; g < e->n_groups; ++g)
            if (!dfs_ensemble_group(e->plans[g], a->g[g])) return DFSNUFFT_ERR_UNSUPPORTED;
        if (!e->d_ctl) {
            if (cudaMalloc(&e->d_ctl, sizeof(int) * ENS_CTL_INTS)) {
                cudaGetLastError();
                e->d_ctl = nullptr;
                return DFSNUFFT_ERR_OOM;
            }
            if (cudaMemset(e->d_ctl, 0, sizeof(int) * ENS_CTL_INTS))
                return ens_fail(e, DFSNUFFT_ERR_CUDA);
        }
        e->num_sms = e->plans[0]->num_sms > 0 ? e->plans[0]->num_sms : 1;
    }
    e->persistent = on ? 1 : 0;
    e->args_ready = 0;
    // the next run records the step again
    if (e->exec) {
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    e->sig_ptr.clear();
    e->sig_counts.clear();
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_ensemble_selftest_queue_timeout(dfsnufft_ensemble e,
                                                        long long cycles) {
    if (!e || cycles < 1 || cycles > 4000000000LL) return DFSNUFFT_ERR_INVALID_ARG;
    if (!e->persistent || !e->args_ready) return DFSNUFFT_ERR_NO_POINTS;
    if (e->status) return e->status;
    EnsArgs a = *e->args;
    a.budget = cycles;
    a.poison_group = 0;
    if (cudaStreamSynchronize(e->stream) ||
        dfs_ensemble_step_launch(a, e->d_ctl, e->num_sms, e->stream, &e->resident))
        return ens_fail(e, DFSNUFFT_ERR_CUDA);
    return read_ctl_status(e);
}

extern "C" int dfsnufft_ensemble_plan(dfsnufft_ensemble e, int group, dfsnufft_plan *out) {
    if (!e || !out || group < 0 || group >= e->n_groups) return DFSNUFFT_ERR_INVALID_ARG;
    *out = e->plans[group];
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_ensemble_destroy(dfsnufft_ensemble e) {
    if (!e) return DFSNUFFT_ERR_INVALID_ARG;
    cudaStreamSynchronize(e->stream);
    if (e->origin) cudaStreamSynchronize(e->origin);
    for (auto s : e->streams)
        if (s) cudaStreamSynchronize(s);
    release(e);
    delete e;
    return DFSNUFFT_OK;
}

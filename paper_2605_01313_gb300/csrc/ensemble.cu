// Ensembles of members on uneven grids: one batched plan per grid size, each
// on its own stream, and one CUDA graph per step.  The step (points and values
// of every member of every group) is recorded by stream capture as a fork/join
// over the group streams, so the groups' kernels overlap on the device, and is
// replayed with one graph launch while the caller's pointers and point counts
// stay the same; when they change, the step runs once uncaptured (it may
// allocate or upload offsets) and is recorded again.
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"

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
};

namespace {

int ens_fail(dfsnufft_ensemble e, int code) {
    if (!e->status) e->status = code;
    return code;
}

// The step, enqueued on the group streams after a fork from `main` and joined
// back into it.
int enqueue_step(dfsnufft_ensemble e, cudaStream_t main, const int64_t *const *counts,
                 const double *const *lon, const double *const *colat, const void *const *coeffs,
                 void *const *values) {
    if (cudaEventRecord(e->fork, main)) return DFSNUFFT_ERR_CUDA;
    for (int g = 0; g < e->n_groups; ++g) {
        if (cudaStreamWaitEvent(e->streams[g], e->fork, 0)) return DFSNUFFT_ERR_CUDA;
        int rc = dfsnufft_set_points_batch(e->plans[g], counts[g], lon[g], colat[g]);
        if (rc) return rc;
        rc = dfsnufft_execute(e->plans[g], coeffs[g], values[g]);
        if (rc) return rc;
        if (cudaEventRecord(e->done[g], e->streams[g])) return DFSNUFFT_ERR_CUDA;
        if (cudaStreamWaitEvent(main, e->done[g], 0)) return DFSNUFFT_ERR_CUDA;
    }
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

extern "C" int dfsnufft_ensemble_check(dfsnufft_ensemble e) {
    if (!e) return DFSNUFFT_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(e->stream)) return ens_fail(e, DFSNUFFT_ERR_CUDA);
    for (auto p : e->plans) {
        int rc = dfsnufft_plan_check(p);
        if (rc) return ens_fail(e, rc);
    }
    return e->status;
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

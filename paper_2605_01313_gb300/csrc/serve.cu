// Serving engine: a request loop with continuous batching under an HBM budget.
//
// A request is one member's interpolation step: its grid, its departure points
// and its n_fields coefficient arrays, all resident in device memory, and a
// device buffer for the values.  submit() queues it and returns a ticket.  A
// dispatcher thread drains the queue, groups pending requests by grid, and
// launches up to max_batch requests of one grid as one batched plan execution
// (set_points + execute) on a free slot: a stream with a batched plan for that
// grid and staging buffers.  Slots are created on demand while the HBM they
// need fits the budget and are kept for reuse (plan state stays resident);
// requests wait in the queue while no slot can take them, and are admitted as
// soon as one frees up, so work from requests that arrive while others run
// overlaps on the device.  Completions are found by polling each slot's event;
// a request's latency runs from submit() to the dispatcher seeing its batch
// complete.
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

typedef std::chrono::steady_clock Clock;

struct Request {
    int64_t ticket;
    dfsnufft_request r;
    Clock::time_point t_submit;
};

struct Done {
    int status;
    double latency_s;
};

struct Slot {
    int n_lon, n_lat;
    int cap_members;
    cudaStream_t stream;
    cudaEvent_t event;
    dfsnufft_plan plan;
    void *coeffs;               // cap_members x F x N2 x N1 (plan precision)
    double *pts;                // lon then colat, 2 x pts_cap
    void *values;               // F x pts_cap
    int64_t pts_cap;
    size_t bytes;               // device bytes this slot holds
    bool busy;
    std::vector<Request> running;
};

}  // namespace

struct dfsnufft_server_s {
    double tol;
    int dtype, n_fields, max_batch;
    dfsnufft_options opts;      // plan options of every slot
    size_t budget, reserved;
    int device;
    std::mutex mu;
    std::condition_variable cv_submit, cv_done;
    std::deque<Request> queue;
    std::map<int64_t, Done> done;
    int64_t next_ticket;
    bool stop;
    std::thread worker;
    std::vector<Slot *> slots;
    dfsnufft_server_stats stats;
};

namespace {

size_t real_size(int dtype) { return dtype == DFSNUFFT_F64 ? sizeof(double) : sizeof(float); }

// Device bytes of a slot for cap members with pts_cap points in total.
size_t slot_bytes(const dfsnufft_params &q, int F, int cap, int64_t pts_cap) {
    const size_t rs = real_size(q.dtype), cs = 2 * rs;
    const size_t lines = (size_t)F * cap;
    size_t b = 0;
    const int herm = (q.flags & DFSNUFFT_REAL_FIELDS) ? 1 : 0;
    b += lines * q.n2 * dfs_tpitch(herm, q.N1) * cs;   // theta-pass output
    b += lines * q.n2 * q.n1 * rs;             // fine grids
    b += lines * q.N2 * q.N1 * cs;             // staged coefficients
    b += (size_t)pts_cap * (16 + 4 + 8 + 2 * rs + 4);   // points, ranks, sorted records
    b += (size_t)F * pts_cap * rs;             // staged values
    b += (size_t)cap * 3 * 4 * (q.n1 / q.tile_x) * (q.n2 / q.tile_y);   // bins
    return b + (4u << 20);                      // tables and slack
}

void free_slot(Slot *s) {
    if (s->plan) dfsnufft_destroy(s->plan);
    if (s->coeffs) cudaFree(s->coeffs);
    if (s->pts) cudaFree(s->pts);
    if (s->values) cudaFree(s->values);
    if (s->event) cudaEventDestroy(s->event);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

// A slot for this grid, or nullptr if the budget cannot hold one.
Slot *make_slot(dfsnufft_server sv, int n_lon, int n_lat, int64_t pts_cap) {
    dfsnufft_params q;
    if (dfsnufft_choose_params_opts(n_lon, n_lat, sv->tol, sv->dtype, &sv->opts, &q))
        return nullptr;
    const int cap = sv->max_batch;
    const size_t need = slot_bytes(q, sv->n_fields, cap, pts_cap);
    if (sv->reserved + need > sv->budget) return nullptr;
    Slot *s = new (std::nothrow) Slot();
    if (!s) return nullptr;
    s->n_lon = n_lon;
    s->n_lat = n_lat;
    s->cap_members = cap;
    s->pts_cap = pts_cap;
    s->busy = false;
    const size_t rs = real_size(sv->dtype), cs = 2 * rs;
    bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->event, cudaEventDisableTiming) == cudaSuccess &&
              dfsnufft_plan_create_opts(cap, n_lon, n_lat, sv->tol, sv->dtype, sv->n_fields,
                                        &sv->opts, s->stream, &s->plan) == DFSNUFFT_OK &&
              cudaMalloc(&s->coeffs, cs * (size_t)cap * sv->n_fields * q.N2 * q.N1) ==
                  cudaSuccess &&
              cudaMalloc((void **)&s->pts, 2 * sizeof(double) * (size_t)pts_cap) == cudaSuccess &&
              cudaMalloc(&s->values, rs * (size_t)sv->n_fields * pts_cap) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_slot(s);
        return nullptr;
    }
    s->bytes = need;
    sv->reserved += need;
    return s;
}

// Launch a batch of same-grid requests on a free slot.
int launch_batch(dfsnufft_server sv, Slot *s, std::vector<Request> &batch) {
    const dfsnufft_params &q = s->plan->prm;
    const size_t rs = real_size(sv->dtype), cs = 2 * rs;
    const int F = sv->n_fields;
    const int M = s->cap_members;
    std::vector<int64_t> counts(M, 1);
    int64_t total = 0;
    const size_t coef_bytes = cs * (size_t)F * q.N2 * q.N1;
    for (size_t k = 0; k < batch.size(); ++k) {
        const dfsnufft_request &r = batch[k].r;
        counts[k] = r.n_points;
        if (cudaMemcpyAsync((char *)s->coeffs + k * coef_bytes, r.coeffs, coef_bytes,
                            cudaMemcpyDeviceToDevice, s->stream) ||
            cudaMemcpyAsync(s->pts + total, r.lon, sizeof(double) * r.n_points,
                            cudaMemcpyDeviceToDevice, s->stream) ||
            cudaMemcpyAsync(s->pts + s->pts_cap + total, r.colat, sizeof(double) * r.n_points,
                            cudaMemcpyDeviceToDevice, s->stream))
            return DFSNUFFT_ERR_CUDA;
        total += r.n_points;
    }
    // unused member places get one point (the first one of the batch): their
    // values are computed and dropped
    for (int k = (int)batch.size(); k < M; ++k) {
        if (cudaMemcpyAsync(s->pts + total, batch[0].r.lon, sizeof(double),
                            cudaMemcpyDeviceToDevice, s->stream) ||
            cudaMemcpyAsync(s->pts + s->pts_cap + total, batch[0].r.colat, sizeof(double),
                            cudaMemcpyDeviceToDevice, s->stream))
            return DFSNUFFT_ERR_CUDA;
        total += 1;
    }
    int rc = dfsnufft_set_points_batch(s->plan, counts.data(), s->pts, s->pts + s->pts_cap);
    if (rc) return rc;
    rc = dfsnufft_execute(s->plan, s->coeffs, s->values);
    if (rc) return rc;
    int64_t off = 0;
    for (size_t k = 0; k < batch.size(); ++k) {
        const dfsnufft_request &r = batch[k].r;
        if (cudaMemcpyAsync(r.values, (char *)s->values + rs * F * off, rs * F * r.n_points,
                            cudaMemcpyDeviceToDevice, s->stream))
            return DFSNUFFT_ERR_CUDA;
        off += r.n_points;
    }
    if (cudaEventRecord(s->event, s->stream)) return DFSNUFFT_ERR_CUDA;
    s->running = batch;
    s->busy = true;
    sv->stats.batches += 1;
    sv->stats.members += (int64_t)batch.size();
    return DFSNUFFT_OK;
}

void finish(dfsnufft_server sv, std::vector<Request> &reqs, int status) {
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lock(sv->mu);
    for (auto &r : reqs) {
        Done d;
        d.status = status;
        d.latency_s = std::chrono::duration<double>(now - r.t_submit).count();
        sv->done[r.ticket] = d;
        sv->stats.completed += 1;
    }
    reqs.clear();
    sv->cv_done.notify_all();
}

void worker_loop(dfsnufft_server sv) {
    cudaSetDevice(sv->device);
    std::map<std::pair<int, int>, std::deque<Request>> pending;   // by grid
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            bool idle = pending.empty();
            for (auto *s : sv->slots) idle = idle && !s->busy;
            if (idle && sv->queue.empty() && !sv->stop)
                sv->cv_submit.wait_for(lock, std::chrono::milliseconds(5));
            if (sv->stop && sv->queue.empty() && idle) break;
            while (!sv->queue.empty()) {
                Request r = sv->queue.front();
                sv->queue.pop_front();
                pending[{r.r.n_lon, r.r.n_lat}].push_back(r);
            }
        }
        // completions
        for (auto *s : sv->slots) {
            if (!s->busy) continue;
            cudaError_t e = cudaEventQuery(s->event);
            if (e == cudaErrorNotReady) continue;
            int st = e == cudaSuccess ? dfsnufft_plan_check(s->plan) : DFSNUFFT_ERR_CUDA;
            s->busy = false;
            finish(sv, s->running, st);
        }
        // admission and dispatch
        for (auto it = pending.begin(); it != pending.end();) {
            std::deque<Request> &q = it->second;
            while (!q.empty()) {
                const int n_lon = it->first.first, n_lat = it->first.second;
                std::vector<Request> batch;
                int64_t pts = 0;
                while (!q.empty() && (int)batch.size() < sv->max_batch) {
                    batch.push_back(q.front());
                    pts += q.front().r.n_points;
                    q.pop_front();
                }
                const int64_t pts_need = pts + sv->max_batch;
                Slot *slot = nullptr;
                for (auto *s : sv->slots)
                    if (!s->busy && s->n_lon == n_lon && s->n_lat == n_lat &&
                        s->pts_cap >= pts_need) {
                        slot = s;
                        break;
                    }
                if (!slot) {
                    // a new slot, sized for a full batch of whole grids
                    const int64_t grid_pts = (int64_t)n_lon * n_lat;
                    int64_t cap = grid_pts * sv->max_batch + sv->max_batch;
                    if (cap < pts_need) cap = pts_need;
                    slot = make_slot(sv, n_lon, n_lat, cap);
                    if (!slot) {
                        // release idle slots of other grids to make room
                        for (size_t i = 0; i < sv->slots.size() && !slot; ++i) {
                            Slot *s = sv->slots[i];
                            if (s->busy) continue;
                            sv->reserved -= s->bytes;
                            free_slot(s);
                            sv->slots.erase(sv->slots.begin() + i);
                            --i;
                            slot = make_slot(sv, n_lon, n_lat, cap);
                        }
                    }
                    if (slot) sv->slots.push_back(slot);
                }
                if (!slot) {
                    bool any_busy = false;
                    for (auto *s : sv->slots) any_busy = any_busy || s->busy;
                    if (!any_busy) {
                        // nothing will free up: the request can never fit
                        finish(sv, batch, DFSNUFFT_ERR_OOM);
                        continue;
                    }
                    for (auto r = batch.rbegin(); r != batch.rend(); ++r) q.push_front(*r);
                    break;
                }
                int rc = launch_batch(sv, slot, batch);
                if (rc) {
                    cudaGetLastError();
                    finish(sv, batch, rc);
                }
            }
            if (q.empty()) it = pending.erase(it);
            else ++it;
        }
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            sv->stats.slots = (int)sv->slots.size();
            sv->stats.reserved_bytes = (int64_t)sv->reserved;
        }
        bool busy = false;
        for (auto *s : sv->slots) busy = busy || s->busy;
        if (busy) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" int dfsnufft_server_create(double tol, int dtype, int n_fields, int64_t hbm_budget,
                                      int max_batch, dfsnufft_server *out) {
    return dfsnufft_server_create_opts(tol, dtype, n_fields, hbm_budget, max_batch, nullptr, out);
}

extern "C" int dfsnufft_server_create_opts(double tol, int dtype, int n_fields,
                                           int64_t hbm_budget, int max_batch,
                                           const dfsnufft_options *opts, dfsnufft_server *out) {
    if (!out || n_fields < 1 || n_fields > 64 || hbm_budget <= 0 || max_batch < 1 ||
        max_batch > 256)
        return DFSNUFFT_ERR_INVALID_ARG;
    dfsnufft_params q;
    int rc = dfsnufft_choose_params_opts(64, 32, tol, dtype, opts, &q);
    if (rc) return rc;
    dfsnufft_server sv = new (std::nothrow) dfsnufft_server_s();
    if (!sv) return DFSNUFFT_ERR_OOM;
    memset(&sv->opts, 0, sizeof(sv->opts));
    if (opts) sv->opts = *opts;
    sv->tol = tol;
    sv->dtype = dtype;
    sv->n_fields = n_fields;
    sv->max_batch = max_batch;
    sv->budget = (size_t)hbm_budget;
    sv->reserved = 0;
    sv->next_ticket = 1;
    sv->stop = false;
    memset(&sv->stats, 0, sizeof(sv->stats));
    if (cudaGetDevice(&sv->device)) {
        delete sv;
        return DFSNUFFT_ERR_CUDA;
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_server_submit(dfsnufft_server sv, const dfsnufft_request *req,
                                      int64_t *ticket) {
    if (!sv || !req || !ticket || req->n_points < 1 || req->n_points > 0x7fffffffLL ||
        !req->lon || !req->colat || !req->coeffs || !req->values)
        return DFSNUFFT_ERR_INVALID_ARG;
    dfsnufft_params q;
    int rc = dfsnufft_choose_params_opts(req->n_lon, req->n_lat, sv->tol, sv->dtype, &sv->opts, &q);
    if (rc) return rc;
    Request r;
    r.r = *req;
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        r.ticket = sv->next_ticket++;
        sv->queue.push_back(r);
        sv->stats.submitted += 1;
    }
    sv->cv_submit.notify_one();
    *ticket = r.ticket;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_server_wait(dfsnufft_server sv, int64_t ticket, double timeout_s,
                                    int *status, double *latency_s) {
    if (!sv || !status) return DFSNUFFT_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(sv->mu);
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(timeout_s));
    while (sv->done.find(ticket) == sv->done.end()) {
        if (sv->cv_done.wait_until(lock, until) == std::cv_status::timeout &&
            sv->done.find(ticket) == sv->done.end())
            return DFSNUFFT_ERR_TIMEOUT;
    }
    const Done d = sv->done[ticket];
    sv->done.erase(ticket);
    *status = d.status;
    if (latency_s) *latency_s = d.latency_s;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_server_stats_get(dfsnufft_server sv, dfsnufft_server_stats *out) {
    if (!sv || !out) return DFSNUFFT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    *out = sv->stats;
    out->budget_bytes = (int64_t)sv->budget;
    return DFSNUFFT_OK;
}

extern "C" int dfsnufft_server_destroy(dfsnufft_server sv) {
    if (!sv) return DFSNUFFT_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
    }
    sv->cv_submit.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (auto *s : sv->slots) {
        cudaStreamSynchronize(s->stream);
        free_slot(s);
    }
    delete sv;
    return DFSNUFFT_OK;
}

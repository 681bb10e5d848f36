// serve.cu -- request loop over the resident graphs of a group.
//
// Update requests (one batch for one graph each) arrive at any time from any
// thread.  One worker thread drains them: every call it makes takes the
// oldest pending request of as many distinct graphs as fit the group's
// per-call limits (continuous batching) and applies them with one
// esc_group_apply, so requests that arrive while a call runs go into the
// next one.  Requests of one graph are applied in the order they were
// submitted.  The paper processes one batch at a time (Alg. 3); this loop
// adds the serving layer around that step and changes nothing in what a
// batch computes: a graph's counts after its requests are those of the same
// batches applied one by one.
#include <time.h>

#include <algorithm>
#include <condition_variable>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <cuda_runtime.h>

#include "escher.h"

namespace esc {
// api.cu: the per-call limits and the device of a group
esc_status group_limits(const esc_group* grp, int32_t* n_graphs, int64_t* max_updates, int64_t* max_nnz,
                        uint32_t* families, int* device);
}  // namespace esc

namespace {

int64_t now_ns() {
    timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return int64_t(t.tv_sec) * 1000000000LL + t.tv_nsec;
}

struct Request {
    int64_t ticket = 0;
    int32_t graph = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> mem;
    std::vector<int64_t> ts;
    std::vector<int32_t> del;
    int32_t* out_ids = nullptr;
    int64_t t_arrival = 0;
    int64_t updates() const { return int64_t(off.empty() ? 0 : off.size() - 1) + int64_t(del.size()); }
};

}  // namespace

struct esc_server {
    esc_group* grp = nullptr;
    int dev = 0;
    int32_t G = 0;
    int64_t max_upd = 0, max_nnz = 0;
    uint32_t families = 0;
    int64_t max_pending = 0;
    int32_t max_per_call = 0;

    std::mutex mu;                      // queue, results, counters
    std::condition_variable cv_work;    // worker: requests pending or stop
    std::condition_variable cv_done;    // waiters: a request finished
    std::list<Request*> pending;        // submitted, not yet taken, in order
    int64_t pending_upd = 0;            // updates submitted and not finished
    int64_t in_flight = 0;              // requests submitted and not finished
    std::unordered_set<int64_t> open;   // submitted, not finished
    std::unordered_map<int64_t, esc_request_info> done;  // finished, not collected
    int64_t next_ticket = 0;
    bool stop = false;
    esc_server_stats stats{};

    std::mutex gmu;  // one user of the group at a time (worker or a query)
    std::thread worker;

    void run();
    void finish(std::vector<Request*>& take, const std::vector<int32_t>& status, int64_t t_start, int64_t t_done,
                int64_t call_updates);
};

void esc_server::finish(std::vector<Request*>& take, const std::vector<int32_t>& status, int64_t t_start,
                        int64_t t_done, int64_t call_updates) {
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < take.size(); ++i) {
        Request* r = take[i];
        esc_request_info inf{};
        inf.status = status[i];
        inf.call_batches = int32_t(take.size());
        inf.t_arrival_ns = r->t_arrival;
        inf.t_start_ns = t_start;
        inf.t_done_ns = t_done;
        inf.call_updates = call_updates;
        done[r->ticket] = inf;
        open.erase(r->ticket);
        pending_upd -= r->updates();
        --in_flight;
        if (status[i] == ESC_OK) {
            ++stats.completed;
            stats.updates += r->updates();
        } else {
            ++stats.failed;
        }
        delete r;
    }
    take.clear();
    cv_done.notify_all();
}

void esc_server::run() {
    cudaSetDevice(dev);
    std::vector<Request*> take;
    std::vector<char> used(size_t(G), 0);
    std::vector<esc_batch> arr;
    std::vector<int32_t> status;
    for (;;) {
        int64_t upd = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !pending.empty(); });
            if (pending.empty()) break;  // stop with nothing left
            // the oldest request of each graph, oldest first, while the call's
            // limits hold; a graph's later requests wait behind its first
            std::fill(used.begin(), used.end(), 0);
            int64_t nnz = 0;
            for (auto it = pending.begin(); it != pending.end();) {
                Request* r = *it;
                if (used[size_t(r->graph)]) {
                    ++it;
                    continue;
                }
                used[size_t(r->graph)] = 1;
                const int64_t u = r->updates(), z = int64_t(r->mem.size());
                if (!take.empty() && (upd + u > max_upd || nnz + z > max_nnz ||
                                      (max_per_call > 0 && int32_t(take.size()) >= max_per_call))) {
                    ++it;
                    continue;
                }
                take.push_back(r);
                upd += u;
                nnz += z;
                it = pending.erase(it);
            }
            ++stats.calls;
        }
        arr.assign(take.size(), esc_batch{});
        for (size_t i = 0; i < take.size(); ++i) {
            Request* r = take[i];
            esc_batch& b = arr[i];
            b.graph = r->graph;
            b.n_ins = r->off.empty() ? 0 : int64_t(r->off.size() - 1);
            b.ins_offsets = r->off.empty() ? nullptr : r->off.data();
            b.ins_members = r->mem.data();
            b.ins_timestamps = r->ts.empty() ? nullptr : r->ts.data();
            b.n_del = int64_t(r->del.size());
            b.del_ids = r->del.empty() ? nullptr : r->del.data();
            b.out_ins_ids = r->out_ids;
        }
        const int64_t t_start = now_ns();
        status.assign(take.size(), ESC_OK);
        esc_status s;
        {
            std::lock_guard<std::mutex> g(gmu);
            s = esc_group_apply(grp, int32_t(arr.size()), arr.data());
            if ((s == ESC_ERR_INVALID_ARG || s == ESC_ERR_NOT_FOUND || s == ESC_ERR_OUT_OF_MEMORY ||
                 s == ESC_ERR_UNSUPPORTED) &&
                arr.size() > 1) {
                // a failed call changes nothing: apply the requests one by one
                // so that only the faulty ones fail
                for (size_t i = 0; i < arr.size(); ++i) status[i] = esc_group_apply(grp, 1, &arr[i]);
            } else {
                std::fill(status.begin(), status.end(), int32_t(s));
            }
        }
        finish(take, status, t_start, now_ns(), upd);
    }
}

extern "C" {

esc_status esc_server_create(esc_group* grp, int64_t max_pending_updates, int32_t max_batches_per_call,
                             esc_server** out) {
    if (!out || !grp || max_pending_updates <= 0 || max_batches_per_call < 0) return ESC_ERR_INVALID_ARG;
    *out = nullptr;
    esc_server* s = new esc_server();
    s->grp = grp;
    esc_status st = esc::group_limits(grp, &s->G, &s->max_upd, &s->max_nnz, &s->families, &s->dev);
    if (st != ESC_OK) {
        delete s;
        return st;
    }
    s->max_pending = max_pending_updates;
    s->max_per_call = max_batches_per_call;
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return ESC_OK;
}

esc_status esc_server_submit(esc_server* s, const esc_batch* b, int64_t t_arrival_ns, int64_t* ticket) {
    if (!s || !b || !ticket) return ESC_ERR_INVALID_ARG;
    *ticket = -1;
    if (b->graph < 0 || b->graph >= s->G || b->n_ins < 0 || b->n_del < 0) return ESC_ERR_INVALID_ARG;
    if (b->n_ins > 0 && (!b->ins_offsets || !b->ins_members)) return ESC_ERR_INVALID_ARG;
    if (b->n_ins > 0 && (s->families & ESC_FAMILY_TEMPORAL) && !b->ins_timestamps) return ESC_ERR_INVALID_ARG;
    if (b->n_del > 0 && !b->del_ids) return ESC_ERR_INVALID_ARG;
    const int64_t u = b->n_ins + b->n_del;
    if (u == 0) return ESC_ERR_INVALID_ARG;
    if (u > s->max_upd) return ESC_ERR_OUT_OF_MEMORY;
    auto host = [](const void* p) {
        if (!p) return true;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return true;
        }
        return a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged;
    };
    if (!host(b->ins_offsets) || !host(b->ins_members) || !host(b->ins_timestamps) || !host(b->del_ids) ||
        !host(b->out_ins_ids))
        return ESC_ERR_INVALID_ARG;
    int64_t nnz = 0;
    if (b->n_ins > 0) {
        if (b->ins_offsets[0] != 0) return ESC_ERR_INVALID_ARG;
        nnz = b->ins_offsets[b->n_ins];
        if (nnz < 0) return ESC_ERR_INVALID_ARG;
        if (nnz > s->max_nnz) return ESC_ERR_OUT_OF_MEMORY;
    }
    {
        // cheap refusal before copying anything
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return ESC_ERR_INVALID_ARG;
        if (s->pending_upd + u > s->max_pending) {
            ++s->stats.rejected;
            return ESC_ERR_BUSY;
        }
    }
    Request* r = new Request();
    r->graph = b->graph;
    r->t_arrival = t_arrival_ns > 0 ? t_arrival_ns : now_ns();
    if (b->n_ins > 0) {
        r->off.assign(b->ins_offsets, b->ins_offsets + b->n_ins + 1);
        r->mem.assign(b->ins_members, b->ins_members + nnz);
        if (b->ins_timestamps) r->ts.assign(b->ins_timestamps, b->ins_timestamps + b->n_ins);
    }
    if (b->n_del > 0) r->del.assign(b->del_ids, b->del_ids + b->n_del);
    r->out_ids = b->n_ins > 0 ? b->out_ins_ids : nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->pending_upd + u > s->max_pending) {
            ++s->stats.rejected;
            delete r;
            return ESC_ERR_BUSY;
        }
        r->ticket = s->next_ticket++;
        s->pending.push_back(r);
        s->open.insert(r->ticket);
        s->pending_upd += u;
        ++s->in_flight;
        ++s->stats.submitted;
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return ESC_OK;
}

esc_status esc_server_wait(esc_server* s, int64_t ticket, esc_request_info* info) {
    if (!s || ticket < 0) return ESC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket >= s->next_ticket) return ESC_ERR_INVALID_ARG;
    auto it = s->done.find(ticket);
    while (it == s->done.end()) {
        if (!s->open.count(ticket)) return ESC_ERR_NOT_FOUND;  // collected before
        s->cv_done.wait(lk);
        it = s->done.find(ticket);
    }
    const esc_request_info inf = it->second;
    s->done.erase(it);
    if (info) *info = inf;
    return esc_status(inf.status);
}

esc_status esc_server_drain(esc_server* s) {
    if (!s) return ESC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->in_flight == 0; });
    return ESC_OK;
}

esc_status esc_server_triads(esc_server* s, int32_t graph, esc_triad_type type, int64_t window, uint64_t* out,
                             int32_t n_out) {
    if (!s) return ESC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->gmu);
    return esc_group_triads(s->grp, graph, type, window, out, n_out);
}

esc_status esc_server_get_stats(esc_server* s, esc_server_stats* out) {
    if (!s || !out) return ESC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->pending_updates = s->pending_upd;
    return ESC_OK;
}

esc_status esc_server_destroy(esc_server* s) {
    if (!s) return ESC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return ESC_OK;
}

}  // extern "C"

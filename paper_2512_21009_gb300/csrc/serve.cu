// serve.cu -- request loop over the resident graphs of one or more groups.
//
// Update requests (one batch for one graph each) arrive at any time from any
// thread.  Each group ("shard") has a worker thread that drains its
// requests: every call it makes takes the oldest pending request of as many
// distinct graphs of the group as fit the group's per-call limits
// (continuous batching) and applies them with one esc_group_apply, so
// requests that arrive while a call runs go into the next one.  Groups can
// be added while the server runs; the workers of different groups run their
// calls at the same time, each on its group's stream, so their device work
// overlaps.  Requests of one graph are applied in the order they were
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

// One group of resident graphs and the worker thread that applies its
// requests.  Graphs are numbered server-wide: the shard's graph i is the
// server's graph first + i.
struct Shard {
    esc_group* grp = nullptr;
    int dev = 0;
    int32_t first = 0, G = 0;
    int64_t max_upd = 0, max_nnz = 0;
    uint32_t families = 0;
    std::list<Request*> pending;        // submitted, not yet taken, in order (server mu)
    std::condition_variable cv_work;    // this shard's worker: requests pending or stop
    std::mutex gmu;                     // one user of the group at a time (worker or a query)
    std::thread worker;
};

struct esc_server {
    int64_t max_pending = 0;
    int32_t max_per_call = 0;

    std::mutex mu;                      // shards list, queues, results, counters
    std::condition_variable cv_done;    // waiters: a request finished
    std::vector<Shard*> shards;         // appended to, never removed while running
    std::vector<int32_t> shard_of;      // server graph -> shard index
    int64_t pending_upd = 0;            // updates submitted and not finished
    int64_t in_flight = 0;              // requests submitted and not finished
    std::unordered_set<int64_t> open;   // submitted, not finished
    std::unordered_map<int64_t, esc_request_info> done;  // finished, not collected
    int64_t next_ticket = 0;
    bool stop = false;
    esc_server_stats stats{};

    void run(Shard* sh);
    void finish(std::vector<Request*>& take, const std::vector<int32_t>& status, int64_t t_start, int64_t t_done,
                int64_t call_updates);
    esc_status add(esc_group* grp, int32_t* first);
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

void esc_server::run(Shard* sh) {
    cudaSetDevice(sh->dev);
    std::vector<Request*> take;
    std::vector<char> used(size_t(sh->G), 0);
    std::vector<esc_batch> arr;
    std::vector<int32_t> status;
    for (;;) {
        int64_t upd = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            sh->cv_work.wait(lk, [&] { return stop || !sh->pending.empty(); });
            if (sh->pending.empty()) break;  // stop with nothing left
            // the oldest request of each graph, oldest first, while the call's
            // limits hold; a graph's later requests wait behind its first
            std::fill(used.begin(), used.end(), 0);
            int64_t nnz = 0;
            for (auto it = sh->pending.begin(); it != sh->pending.end();) {
                Request* r = *it;
                const size_t lg = size_t(r->graph - sh->first);
                if (used[lg]) {
                    ++it;
                    continue;
                }
                used[lg] = 1;
                const int64_t u = r->updates(), z = int64_t(r->mem.size());
                if (!take.empty() && (upd + u > sh->max_upd || nnz + z > sh->max_nnz ||
                                      (max_per_call > 0 && int32_t(take.size()) >= max_per_call))) {
                    ++it;
                    continue;
                }
                take.push_back(r);
                upd += u;
                nnz += z;
                it = sh->pending.erase(it);
            }
            ++stats.calls;
        }
        arr.assign(take.size(), esc_batch{});
        for (size_t i = 0; i < take.size(); ++i) {
            Request* r = take[i];
            esc_batch& b = arr[i];
            b.graph = r->graph - sh->first;
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
            std::lock_guard<std::mutex> g(sh->gmu);
            s = esc_group_apply(sh->grp, int32_t(arr.size()), arr.data());
            if ((s == ESC_ERR_INVALID_ARG || s == ESC_ERR_NOT_FOUND || s == ESC_ERR_OUT_OF_MEMORY ||
                 s == ESC_ERR_UNSUPPORTED) &&
                arr.size() > 1) {
                // a failed call changes nothing: apply the requests one by one
                // so that only the faulty ones fail
                for (size_t i = 0; i < arr.size(); ++i) status[i] = esc_group_apply(sh->grp, 1, &arr[i]);
            } else {
                std::fill(status.begin(), status.end(), int32_t(s));
            }
        }
        finish(take, status, t_start, now_ns(), upd);
    }
}

esc_status esc_server::add(esc_group* grp, int32_t* first) {
    Shard* sh = new Shard();
    sh->grp = grp;
    esc_status st = esc::group_limits(grp, &sh->G, &sh->max_upd, &sh->max_nnz, &sh->families, &sh->dev);
    if (st != ESC_OK) {
        delete sh;
        return st;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        if (stop) {
            delete sh;
            return ESC_ERR_INVALID_ARG;
        }
        for (Shard* o : shards)
            if (o->grp == grp) {
                delete sh;
                return ESC_ERR_INVALID_ARG;  // already served
            }
        sh->first = int32_t(shard_of.size());
        shard_of.insert(shard_of.end(), size_t(sh->G), int32_t(shards.size()));
        shards.push_back(sh);
        if (first) *first = sh->first;
    }
    sh->worker = std::thread([this, sh] { run(sh); });
    return ESC_OK;
}

extern "C" {

esc_status esc_server_create(esc_group* grp, int64_t max_pending_updates, int32_t max_batches_per_call,
                             esc_server** out) {
    if (!out || !grp || max_pending_updates <= 0 || max_batches_per_call < 0) return ESC_ERR_INVALID_ARG;
    *out = nullptr;
    esc_server* s = new esc_server();
    s->max_pending = max_pending_updates;
    s->max_per_call = max_batches_per_call;
    esc_status st = s->add(grp, nullptr);
    if (st != ESC_OK) {
        delete s;
        return st;
    }
    *out = s;
    return ESC_OK;
}

esc_status esc_server_add_group(esc_server* s, esc_group* grp, int32_t* first_graph) {
    if (!s || !grp) return ESC_ERR_INVALID_ARG;
    return s->add(grp, first_graph);
}

esc_status esc_group_fits(const esc_config* shared, int32_t n_graphs, const esc_config* graph_cfg,
                          int64_t reserve_bytes, int32_t* fits) {
    if (!fits || reserve_bytes < 0) return ESC_ERR_INVALID_ARG;
    *fits = 0;
    int64_t need = 0;
    esc_status st = esc_group_bytes(shared, n_graphs, graph_cfg, &need);
    if (st != ESC_OK) return st;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return ESC_ERR_CUDA;
    }
    *fits = int64_t(free_b) - reserve_bytes >= need ? 1 : 0;
    return ESC_OK;
}

esc_status esc_server_submit(esc_server* s, const esc_batch* b, int64_t t_arrival_ns, int64_t* ticket) {
    if (!s || !b || !ticket) return ESC_ERR_INVALID_ARG;
    *ticket = -1;
    Shard* sh = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (b->graph >= 0 && size_t(b->graph) < s->shard_of.size()) sh = s->shards[size_t(s->shard_of[size_t(b->graph)])];
    }
    if (!sh || b->n_ins < 0 || b->n_del < 0) return ESC_ERR_INVALID_ARG;
    if (b->n_ins > 0 && (!b->ins_offsets || !b->ins_members)) return ESC_ERR_INVALID_ARG;
    if (b->n_ins > 0 && (sh->families & ESC_FAMILY_TEMPORAL) && !b->ins_timestamps) return ESC_ERR_INVALID_ARG;
    if (b->n_del > 0 && !b->del_ids) return ESC_ERR_INVALID_ARG;
    const int64_t u = b->n_ins + b->n_del;
    if (u == 0) return ESC_ERR_INVALID_ARG;
    if (u > sh->max_upd) return ESC_ERR_OUT_OF_MEMORY;
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
        if (nnz > sh->max_nnz) return ESC_ERR_OUT_OF_MEMORY;
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
        sh->pending.push_back(r);
        s->open.insert(r->ticket);
        s->pending_upd += u;
        ++s->in_flight;
        ++s->stats.submitted;
        *ticket = r->ticket;
    }
    sh->cv_work.notify_one();
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
    Shard* sh = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (graph >= 0 && size_t(graph) < s->shard_of.size()) sh = s->shards[size_t(s->shard_of[size_t(graph)])];
    }
    if (!sh) return ESC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(sh->gmu);
    return esc_group_triads(sh->grp, graph - sh->first, type, window, out, n_out);
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
    std::vector<Shard*> shards;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        shards = s->shards;
    }
    for (Shard* sh : shards) sh->cv_work.notify_all();
    for (Shard* sh : shards) {
        if (sh->worker.joinable()) sh->worker.join();
        delete sh;
    }
    delete s;
    return ESC_OK;
}

}  // extern "C"

// api.cu -- the C ABI declared in include/escher.h.
//
// Host code here only sizes and allocates device memory, stages host-pointer
// inputs to the device, launches the kernels of store.cu and count.cu in
// order on the graph's stream, and reads back status and counts.  Every step
// of the update and of the counting runs in those kernels.
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "escher.h"
#include "escher_internal.cuh"
#include "store_api.cuh"

namespace esc {

// the message of the last failed call without a handle (esc_last_error(NULL))
thread_local std::string t_create_error;

namespace {

// 0: pageable host memory, 1: page-locked host memory, 2: device memory
int ptr_kind(const void* p) {
    if (!p) return 0;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 2;
    return a.type == cudaMemoryTypeHost ? 1 : 0;
}

bool is_device_ptr(const void* p) { return ptr_kind(p) == 2; }

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

struct Engine {
    int dev = 0;
    cudaStream_t st = nullptr;
    int sm_count = 0;
    esc_config shared{};
    int32_t G = 0;
    std::vector<int64_t> vbase, ebase, ecap;
    std::vector<int32_t> nv;
    int64_t inc_cap = 0;  // incidences of all graphs (capacity)
    Store S{};
    std::vector<void*> allocs;
    unsigned long long* d_dbg = nullptr;  // debug mode: per-graph sums of the invariant check
    FILE* jsonl = nullptr;                // ESC_STATS_JSONL: one record per call
    int64_t n_calls = 0;
    // call staging
    Call C{};
    int64_t max_ins = 0, max_nnz = 0;
    BatchIn* d_batches = nullptr;
    int64_t* d_bins_lo = nullptr;
    int64_t* d_bdel_lo = nullptr;
    BatchIn* h_batches = nullptr;      // pinned
    int64_t* h_lo = nullptr;           // pinned [2*(G+1)]
    Scalars* d_sc = nullptr;
    Scalars* h_sc = nullptr;           // pinned
    uint64_t* h_counts = nullptr;      // pinned [kCStride]
    int32_t* h_ids = nullptr;          // pinned [max_ins]
    int64_t* h_word = nullptr;         // pinned word read back by the counter
    int64_t* h_dims = nullptr;         // pinned [3]: batches, inserts, deletes of the call
    int64_t* d_dims = nullptr;         // device copy
    // device staging for host-pointer inputs
    int64_t* st_off = nullptr;
    int32_t* st_mem = nullptr;
    int64_t* st_ts = nullptr;
    int32_t* st_del = nullptr;
    int32_t* st_pin = nullptr;
    CountScratch cs{};
    int64_t max_u = 0;
    PairTable pairs{};                 // vertex-pair statistics (ESC_FAMILY_VERTEX12)
    // pinned host copies of host-pointer inputs, grown on demand, so that a
    // call with many batches moves each input array with one copy
    struct Pinned {
        void* p = nullptr;
        size_t bytes = 0;
    } hs[5];
    size_t hs_lo[5] = {};  // first element of hs[k] not yet copied in this call
    bool profiling = false;
    cudaEvent_t cev[32] = {};          // centre-kernel launch events (profiling)
    // calls as one replayed CUDA graph (a fixed launch sequence whose kernels
    // read the call's sizes on the device)
    bool graph_mode = false;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t own_st = nullptr;     // capture needs a stream other than the legacy one
    int64_t graph_kernels = 0, graph_count_kernels = 0;
    int n_cev = 0;
    // sizing pass: alloc() only adds up the bytes it would take
    bool dry = false;
    int64_t dry_bytes = 0;
    cudaEvent_t ev[6] = {};
    esc_batch_stats last{};
    LaunchCounter lc;
    std::string err;

    template <typename T>
    cudaError_t alloc(T** p, size_t n, int fill = 0) {
        size_t bytes = n * sizeof(T);
        if (bytes == 0) bytes = 16;
        if (dry) {
            dry_bytes += int64_t((bytes + 511) & ~size_t(511));
            *p = nullptr;
            return cudaSuccess;
        }
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        *p = static_cast<T*>(q);
        return cudaMemsetAsync(q, fill, bytes, st);
    }

    ~Engine() {
        if (st) cudaStreamSynchronize(st);
        if (jsonl) fclose(jsonl);
        for (void* p : allocs) cudaFree(p);
        if (h_batches) cudaFreeHost(h_batches);
        if (h_lo) cudaFreeHost(h_lo);
        if (h_sc) cudaFreeHost(h_sc);
        if (h_counts) cudaFreeHost(h_counts);
        if (h_ids) cudaFreeHost(h_ids);
        if (h_word) cudaFreeHost(h_word);
        if (h_dims) cudaFreeHost(h_dims);
        for (auto& h : hs)
            if (h.p) cudaFreeHost(h.p);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        for (auto& e : cev)
            if (e) cudaEventDestroy(e);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (own_st) cudaStreamDestroy(own_st);
    }

    esc_status fail(esc_status s, const std::string& m) {
        err = m;
        return s;
    }
    esc_status cuda_fail(cudaError_t e, const char* where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return ESC_ERR_CUDA;
    }
};

#define ESC_CU(expr, where)                          \
    do {                                             \
        cudaError_t e__ = (expr);                    \
        if (e__ != cudaSuccess) return E->cuda_fail(e__, where); \
    } while (0)

static esc_status check_cfg(const esc_config* c, bool per_graph_only) {
    if (!c) return ESC_ERR_INVALID_ARG;
    if (c->n_vertices <= 0 || c->capacity_hyperedges <= 0 || c->capacity_incidences <= 0)
        return ESC_ERR_INVALID_ARG;
    if (c->capacity_hyperedges > (int64_t(1) << 30)) return ESC_ERR_UNSUPPORTED;
    if (per_graph_only) return ESC_OK;
    if (c->max_batch_hyperedges <= 0 || c->max_batch_incidences <= 0) return ESC_ERR_INVALID_ARG;
    if (c->max_batch_incidences > 0x7fffffffLL) return ESC_ERR_UNSUPPORTED;
    if (c->families == 0 || (c->families & ~15u)) return ESC_ERR_INVALID_ARG;
    if ((c->families & kFamV) && (c->families & kFamV12)) return ESC_ERR_INVALID_ARG;
    if (c->delta < 0) return ESC_ERR_INVALID_ARG;
    if (c->debug != 0 && c->debug != 1) return ESC_ERR_INVALID_ARG;
    return ESC_OK;
}

// Graph mode: calls replay one captured launch sequence.  Capture needs a
// stream other than the legacy default one, so an engine created on that
// stream gets its own (every call still synchronises before it returns).
static cudaError_t set_graph_mode(Engine* E, bool on) {
    if (E->gexec) {
        cudaGraphExecDestroy(E->gexec);
        E->gexec = nullptr;
    }
    E->graph_mode = on;
    if (on && !E->st) {
        if (!E->own_st) {
            cudaError_t e = cudaStreamCreate(&E->own_st);
            if (e != cudaSuccess) return e;
        }
        E->st = E->own_st;
    }
    return cudaSuccess;
}

static esc_status build_engine(Engine* E, const esc_config& shared, int32_t G, const esc_config* per,
                               cudaStream_t st) {
    E->shared = shared;
    E->G = G;
    E->st = st;
    ESC_CU(cudaGetDevice(&E->dev), "cudaGetDevice");
    ESC_CU(cudaDeviceGetAttribute(&E->sm_count, cudaDevAttrMultiProcessorCount, E->dev), "attribute");
    const bool dry = E->dry;
    E->vbase.resize(G);
    E->ebase.resize(G);
    E->ecap.resize(G);
    E->nv.resize(G);
    int64_t V = 0, Ecap = 0, inc = 0;
    for (int g = 0; g < G; ++g) {
        E->vbase[g] = V;
        E->nv[g] = per[g].n_vertices;
        E->ebase[g] = Ecap;
        E->ecap[g] = round_up(per[g].capacity_hyperedges, 32);
        V += per[g].n_vertices;
        Ecap += E->ecap[g];
        inc += per[g].capacity_incidences;
    }
    if (V > 0x7fffffffLL || Ecap > 0x7fffffffLL) return E->fail(ESC_ERR_UNSUPPORTED, "ID spaces exceed int32");
    int64_t pair_cap = 0;
    for (int g = 0; g < G; ++g) pair_cap += per[g].capacity_vertex_pairs;
    if (shared.families & kFamV12) {
        if (pair_cap <= 0) return E->fail(ESC_ERR_INVALID_ARG, "ESC_FAMILY_VERTEX12 needs capacity_vertex_pairs");
        // a pair's hyperedge count and size sum share one 64-bit word (24 + 40 bits)
        if (Ecap >= (int64_t(1) << 24))
            return E->fail(ESC_ERR_UNSUPPORTED, "ESC_FAMILY_VERTEX12 holds at most 2^24 hyperedge IDs");
    }
    E->inc_cap = inc;
    Store& S = E->S;
    S.n_graphs = G;
    S.nv_total = V;
    S.e_total = Ecap;
    S.fam = shared.families;
    S.delta = shared.delta;
    int64_t *vb, *eb, *ec;
    int32_t* nvp;
    ESC_CU(E->alloc(&vb, G), "alloc");
    ESC_CU(E->alloc(&eb, G), "alloc");
    ESC_CU(E->alloc(&ec, G), "alloc");
    ESC_CU(E->alloc(&nvp, G), "alloc");
    if (!dry) {
        ESC_CU(cudaMemcpyAsync(vb, E->vbase.data(), G * 8, cudaMemcpyHostToDevice, st), "copy");
        ESC_CU(cudaMemcpyAsync(eb, E->ebase.data(), G * 8, cudaMemcpyHostToDevice, st), "copy");
        ESC_CU(cudaMemcpyAsync(ec, E->ecap.data(), G * 8, cudaMemcpyHostToDevice, st), "copy");
        ESC_CU(cudaMemcpyAsync(nvp, E->nv.data(), G * 4, cudaMemcpyHostToDevice, st), "copy");
        ESC_CU(cudaStreamSynchronize(st), "sync");
    }
    S.vbase = vb;
    S.ebase = eb;
    S.ecap = ec;
    S.nv = nvp;
    ESC_CU(E->alloc(&S.hw, G), "alloc");
    ESC_CU(E->alloc(&S.n_live, G), "alloc");
    ESC_CU(E->alloc(&S.counts, int64_t(G) * kCStride), "alloc");
    ESC_CU(E->alloc(&S.dcounts, int64_t(2) * G * kCStride), "alloc");
    ESC_CU(E->alloc(&S.h_off, Ecap), "alloc");
    ESC_CU(E->alloc(&S.h_card, Ecap), "alloc");
    ESC_CU(E->alloc(&S.h_ts, Ecap), "alloc");
    ESC_CU(E->alloc(&S.live, Ecap / 32), "alloc");
    ESC_CU(E->alloc(&S.delb, Ecap / 32), "alloc");
    ESC_CU(E->alloc(&S.insb, Ecap / 32), "alloc");
    ESC_CU(E->alloc(&S.v_off, V), "alloc");
    ESC_CU(E->alloc(&S.v_deg, V), "alloc");
    ESC_CU(E->alloc(&S.v_cap, V), "alloc");
    ESC_CU(E->alloc(&S.v_ndel, V), "alloc");
    ESC_CU(E->alloc(&S.v_nins, V), "alloc");
    ESC_CU(E->alloc(&S.v_touch, V), "alloc");
    ESC_CU(E->alloc(&S.v_base, V), "alloc");
    ESC_CU(E->alloc(&S.v_newoff, V), "alloc");
    ESC_CU(E->alloc(&S.v_newcap, V), "alloc");
    ESC_CU(E->alloc(&S.realloc_v, V), "alloc");
    ESC_CU(E->alloc(&S.vbig, V), "alloc");
    // slab arenas: power-of-two classes at most double a list, plus the
    // smallest slab per hyperedge / vertex; v2h gets extra room because a
    // vertex that outgrows its slab leaves the old one on a free stack
    auto make_pool = [&](SlabPool& P, int64_t cap) -> esc_status {
        P.cap = cap;
        ESC_CU(E->alloc(&P.arena, cap), "alloc arena");
        ESC_CU(E->alloc(&P.tail, 1), "alloc");
        ESC_CU(E->alloc(&P.top, kNumClasses), "alloc");
        int64_t tot = 0;
        for (int c = 0; c < kNumClasses; ++c) {
            P.base[c] = tot;
            tot += cap / slab_size(c) + 1;
        }
        P.base[kNumClasses] = tot;
        ESC_CU(E->alloc(&P.stack, tot), "alloc stack");
        return ESC_OK;
    };
    esc_status s;
    if ((s = make_pool(S.hp, 2 * inc + 8 * Ecap)) != ESC_OK) return s;
    if ((s = make_pool(S.vp, 3 * inc + 8 * V)) != ESC_OK) return s;
    // call staging
    E->max_ins = shared.max_batch_hyperedges;
    E->max_nnz = shared.max_batch_incidences;
    Call& C = E->C;
    C.max_nnz = E->max_nnz;
    ESC_CU(E->alloc(&E->d_batches, G), "alloc");
    ESC_CU(E->alloc(&E->d_bins_lo, G + 1), "alloc");
    ESC_CU(E->alloc(&E->d_bdel_lo, G + 1), "alloc");
    ESC_CU(E->alloc(&C.nnz_lo, G + 1), "alloc");
    ESC_CU(E->alloc(&C.ins_off, E->max_ins + 1), "alloc");
    ESC_CU(E->alloc(&C.raw, E->max_nnz), "alloc");
    ESC_CU(E->alloc(&C.sorted, E->max_nnz), "alloc");
    ESC_CU(E->alloc(&C.slot, E->max_nnz), "alloc");
    ESC_CU(E->alloc(&C.ts, E->max_ins), "alloc");
    ESC_CU(E->alloc(&C.ins_g, E->max_ins), "alloc");
    ESC_CU(E->alloc(&C.card, E->max_ins), "alloc");
    ESC_CU(E->alloc(&C.ids, E->max_ins), "alloc");
    ESC_CU(E->alloc(&C.out_local, E->max_ins), "alloc");
    ESC_CU(E->alloc(&C.big, E->max_ins), "alloc");
    ESC_CU(E->alloc(&C.del, E->max_ins), "alloc");
    ESC_CU(E->alloc(&C.del_g, E->max_ins), "alloc");
    ESC_CU(E->alloc(&C.touched, V), "alloc");
    ESC_CU(E->alloc(&E->d_sc, 1), "alloc");
    ESC_CU(E->alloc(&E->d_dims, 3), "alloc");
    C.sc = E->d_sc;
    C.batches = E->d_batches;
    ESC_CU(E->alloc(&E->st_off, E->max_ins + G + 1), "alloc");
    ESC_CU(E->alloc(&E->st_mem, E->max_nnz), "alloc");
    ESC_CU(E->alloc(&E->st_ts, E->max_ins), "alloc");
    ESC_CU(E->alloc(&E->st_del, E->max_ins), "alloc");
    ESC_CU(E->alloc(&E->st_pin, E->max_ins), "alloc");
    if (!dry) {
        ESC_CU(cudaMallocHost(&E->h_batches, sizeof(BatchIn) * G), "pinned");
        ESC_CU(cudaMallocHost(&E->h_lo, sizeof(int64_t) * 2 * (G + 1)), "pinned");
        ESC_CU(cudaMallocHost(&E->h_sc, sizeof(Scalars)), "pinned");
        ESC_CU(cudaMallocHost(&E->h_counts, sizeof(uint64_t) * kCStride), "pinned");
        ESC_CU(cudaMallocHost(&E->h_ids, sizeof(int32_t) * E->max_ins), "pinned");
        ESC_CU(cudaMallocHost(&E->h_dims, sizeof(int64_t) * 3), "pinned");
    }
    // counter scratch: neighbour lists for a run of changed hyperedges (runs
    // are split when the lists would not fit), per-ID inversion arrays, and
    // per-block overflow hash tables
    CountShape sh;
    sh.cap = E->max_ins;
    // neighbour-list arena of one count run (24 B per entry): a batch whose
    // lists do not fit is counted in several runs, each rebuilding the N(g1)
    // it needs, so the arena is sized for whole batches
    sh.list_cap = std::min<int64_t>(std::max<int64_t>(int64_t(1) << 22, 512 * sh.cap), int64_t(1) << 29);
    if (const char* env = getenv("ESC_COUNT_LIST")) {
        long long v = atoll(env);
        if (v >= 4096) sh.list_cap = v;
    }
    sh.e_cap = Ecap;
    int64_t slots = int64_t(1) << 15;
    while (slots < 2 * std::min<int64_t>(inc, int64_t(1) << 20) && slots < (int64_t(1) << 16)) slots <<= 1;
    sh.gs_nh = slots;
    sh.gs_c = slots < (int64_t(1) << 16) ? slots : (int64_t(1) << 17);
    if (const char* env = getenv("ESC_COUNT_TABLE_SLOTS")) {
        long long v = atoll(env);
        if (v >= 1024 && (v & (v - 1)) == 0) sh.gs_nh = sh.gs_c = v;
    }
    sh.n_cta_nh = E->sm_count * 2;
    sh.n_cta_c = E->sm_count;
    sh.with_ts = (shared.families & kFamT) != 0;
    sh.c_per_sm = 3;
    // restricted-list pool of a count run (int32 entries, below 2^31): none
    // unless asked for -- building the lists costs more than the probes they
    // save on the measured workloads
    sh.r_cap = 0;
    if (const char* env = getenv("ESC_COUNT_RPOOL")) {
        long long v = atoll(env);
        if (v >= 0 && v < (1ll << 31)) sh.r_cap = v;
    }
    if (dry) {
        E->dry_bytes += int64_t(count_scratch_bytes(sh));
        if (shared.families & kFamV12) E->dry_bytes += int64_t(pair_table_bytes(pair_cap, E->max_ins));
        return ESC_OK;
    }
    void* csmem = nullptr;
    ESC_CU(cudaMalloc(&csmem, count_scratch_bytes(sh)), "alloc count scratch");
    E->allocs.push_back(csmem);
    ESC_CU(cudaMallocHost(&E->h_word, sizeof(int64_t)), "pinned");
    ESC_CU(count_scratch_init(&E->cs, csmem, sh, E->h_word, st), "scratch init");
    E->max_u = count_max_u(sh);
    // test knobs: shrink the shared-memory tables so that the global-table
    // and partitioned paths run on small inputs; lower the neighbourhood size
    // from which restricted lists are built
    if (const char* env = getenv("ESC_CENTER_SMALL")) E->cs.center_small = atoi(env);
    if (const char* env = getenv("ESC_CALL_GRAPH"))
        if (atoi(env) != 0) ESC_CU(set_graph_mode(E, true), "graph mode");
    if (const char* env = getenv("ESC_COUNT_BIGNH")) {
        long long v = atoll(env);
        if (v >= 16) E->cs.big_nh = v;
    }
    if (const char* env = getenv("ESC_COUNT_M1PCT")) {
        long long v = atoll(env);
        if (v >= 1) E->cs.m1_pct = v;
    }
    if (const char* env = getenv("ESC_COUNT_RMIN")) {
        long long v = atoll(env);
        if (v >= 1) E->cs.r_min = v;
    }
    if (const char* env = getenv("ESC_COUNT_ORIENT")) E->cs.orient = atoi(env) != 0;
    if (const char* env = getenv("ESC_COUNT_OPEN_MAX")) {
        long long v = atoll(env);
        if (v >= 0 && v <= 65536) E->cs.oh_max = int(v);
    }
    if (const char* env = getenv("ESC_COUNT_OPEN_SMEM")) {
        long long v = atoll(env);
        if (v >= 0 && v <= 8192) E->cs.oh_smem = int(v);
    }
    if (const char* env = getenv("ESC_COUNT_SMEM_SLOTS")) {
        long long v = atoll(env);
        if (v >= 64 && (v & (v - 1)) == 0) E->cs.smem_slots = v;
    }
    if (shared.families & kFamV12) {
        void* pm = nullptr;
        ESC_CU(cudaMalloc(&pm, pair_table_bytes(pair_cap, E->max_ins)), "alloc pair table");
        E->allocs.push_back(pm);
        ESC_CU(pair_table_init(&E->pairs, pm, pair_cap, E->max_ins, st), "pair table init");
    }
    ESC_CU(upload_tables(st), "tables");
    if (shared.debug) ESC_CU(E->alloc(&E->d_dbg, 3 * int64_t(G)), "alloc");
    if (const char* env = getenv("ESC_STATS_JSONL"))
        if (*env) E->jsonl = fopen(env, "a");
    for (auto& e : E->ev) ESC_CU(cudaEventCreate(&e), "event");
    for (auto& e : E->cev) ESC_CU(cudaEventCreate(&e), "event");
    E->cs.max_cev = 16;
    E->cs.n_cev = &E->n_cev;
    ESC_CU(cudaStreamSynchronize(st), "sync");
    return ESC_OK;
}

static std::string describe(const Scalars& s) {
    char buf[256];
    const int b = s.detail[0], i = s.detail[1], v = s.detail[2];
    switch (s.status) {
        case kErrInvalid:
            if (b >= 0) snprintf(buf, sizeof buf, "batch %d: invalid input at element %d (value %d)", b, i, v);
            else if (b == -5) snprintf(buf, sizeof buf, "insert with ID %d, which holds a live hyperedge", v);
            else snprintf(buf, sizeof buf, "duplicate delete of hyperedge %d", v);
            break;
        case kErrNotFound:
            if (b == -6) snprintf(buf, sizeof buf, "ID %d is outside the graph's hyperedge ID range", v);
            else snprintf(buf, sizeof buf, "delete of hyperedge %d, which is not live", v);
            break;
        case kErrNoMem:
            if (b == -1) snprintf(buf, sizeof buf, "inserted members (%d) exceed max_batch_incidences (%d)", i, v);
            else if (b == -2) snprintf(buf, sizeof buf, "h2v arena full");
            else if (b == -3) snprintf(buf, sizeof buf, "v2h arena full");
            else snprintf(buf, sizeof buf, "batch %d: hyperedge ID capacity exceeded", b);
            break;
        case kErrUnsupported:
            if (b == -4 || b == -8)
                snprintf(buf, sizeof buf,
                         "a changed hyperedge meets %d vertex-hyperedge entries, above the counter's limit", v);
            else if (b >= 0) snprintf(buf, sizeof buf, "batch %d: hyperedge %d has %d members (max %d)", b, i, v, kMaxCard);
            else snprintf(buf, sizeof buf, "counter hash table overflow (%d)", b);
            break;
        default:
            snprintf(buf, sizeof buf, "device error %d (%d, %d, %d)", s.status, b, i, v);
    }
    return buf;
}

// Copy the packed elements [hs_lo[k], used) of hs[k] to the device.
template <typename T>
static esc_status flush_staged(Engine* E, T* dst_area, int k, size_t used) {
    const size_t lo = E->hs_lo[k];
    if (used > lo)
        ESC_CU(cudaMemcpyAsync(dst_area + lo, static_cast<T*>(E->hs[k].p) + lo, (used - lo) * sizeof(T),
                               cudaMemcpyHostToDevice, E->st),
               "stage");
    E->hs_lo[k] = used;
    return ESC_OK;
}

// Stage one input array: a device pointer is used in place; page-locked host
// memory is copied directly to dst_area + used; pageable host memory is
// packed into the pinned buffer hs[k] at element offset `used`, and the packed
// runs go to the device by flush_staged() (one copy per run, normally one per
// array per call).
template <typename T>
static esc_status stage(Engine* E, const T* src, size_t n, T* dst_area, int k, size_t& used, size_t cap,
                        const T** out) {
    if (n == 0 || src == nullptr) {
        *out = src;
        return ESC_OK;
    }
    const int kind = ptr_kind(src);
    if (kind == 2) {
        *out = src;
        return ESC_OK;
    }
    if (used + n > cap) return E->fail(ESC_ERR_OUT_OF_MEMORY, "batch larger than the staging capacity");
    if (kind == 1) {
        // page-locked already: copy straight from the caller's buffer (the
        // call synchronises before it returns), after the packed run before it
        esc_status s = flush_staged(E, dst_area, k, used);
        if (s != ESC_OK) return s;
        E->hs_lo[k] = used + n;
        ESC_CU(cudaMemcpyAsync(dst_area + used, src, n * sizeof(T), cudaMemcpyHostToDevice, E->st), "stage");
        *out = dst_area + used;
        used += n;
        return ESC_OK;
    }
    Engine::Pinned& h = E->hs[k];
    const size_t need = (used + n) * sizeof(T);
    if (need > h.bytes) {
        // earlier calls have synchronised; a run of this call already sent
        // from the old buffer must land before the buffer is freed
        if (E->hs_lo[k] > 0) ESC_CU(cudaStreamSynchronize(E->st), "sync");
        size_t nb = std::max(need, std::max(2 * h.bytes, size_t(1) << 20));
        nb = std::min(nb, std::max(need, cap * sizeof(T)));
        void* q = nullptr;
        ESC_CU(cudaMallocHost(&q, nb), "pinned staging");
        if (h.p) {
            memcpy(q, h.p, used * sizeof(T));
            cudaFreeHost(h.p);
        }
        h.p = q;
        h.bytes = nb;
    }
    memcpy(static_cast<T*>(h.p) + used, src, n * sizeof(T));
    *out = dst_area + used;
    used += n;
    return ESC_OK;
}

constexpr int kFixedRuns = 1;  // count runs per side in the captured sequence (the arena holds a batch)

// NVTX range around the host-side launch of one stage (header-only NVTX v3:
// it costs nothing unless a profiler is attached)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// The device work of one call, in order: ingest, count on the old graph,
// delete, insert, count on the new graph, fold.  fixed: the sequence does not
// depend on the call's sizes (every kernel reads them on the device; count
// runs planned on the device), so it can be captured once into a CUDA graph.
static cudaError_t launch_sequence(Engine* E, const Call& C, bool fixed, cudaStream_t st, LaunchCounter& lc,
                                   bool prof = false) {
    const Store& S = E->S;
    cudaError_t e;
    const bool nbh = (S.fam & (kFamH | kFamV | kFamT)) != 0;  // a family counted from neighbourhoods
    const bool pairs = (S.fam & kFamV12) != 0;
    {
        Range r("escher: ingest");
        // the neighbourhood-size limit binds only the families counted from
        // neighbourhoods
        if ((e = store_ingest(S, C, E->d_bins_lo, E->d_bdel_lo, nbh ? E->max_u : INT64_MAX, E->sm_count, st, lc)))
            return e;
        if (pairs) {
            if ((e = pairs_check(E->pairs, C, st, lc))) return e;
            if ((e = store_latch(C, st, lc))) return e;
        }
    }
    if (fixed && nbh) {
        // the inserted side's runs must fit the sequence before anything changes
        if ((e = count_precheck_fixed(S, C, E->cs, E->max_u, kFixedRuns, st, lc))) return e;
        if ((e = store_latch(C, st, lc))) return e;
    }
    if (prof) cudaEventRecord(E->ev[1], st);
    if (nbh) {
        Range r("escher: count, deleted side");
        if (fixed)
            e = count_launch_fixed(S, C.sc, C.del, C.del_g, S.delb, C.dims + 2, 0, S.dcounts, E->cs, E->max_u,
                                   kFixedRuns, st, lc);
        else
            e = count_launch(S, C.sc, C.del, C.del_g, S.delb, 0, C.n_del, 0, S.dcounts, E->cs, E->max_u, st, lc);
    }
    if (e) return e;
    if (fixed) {
        // a failed count (the retry status) must leave the store unchanged
        if ((e = store_latch(C, st, lc))) return e;
    }
    if (pairs) {
        // vertex-pair statistics: the deleted hyperedges leave (their members
        // are still in the store) and the inserted ones arrive, in one pass
        Range r("escher: vertex pairs");
        if ((e = pairs_update(S, C, E->pairs, E->sm_count, st, lc))) return e;
    }
    if (prof) cudaEventRecord(E->ev[2], st);
    {
        Range r("escher: store update");
        if ((e = store_delete(S, C, E->sm_count, st, lc))) return e;
        if ((e = store_insert(S, C, E->sm_count, st, lc))) return e;
    }
    if (prof) cudaEventRecord(E->ev[3], st);
    uint64_t* dins = S.dcounts + int64_t(S.n_graphs) * kCStride;
    if (nbh) {
        Range r("escher: count, inserted side");
        if (fixed)
            e = count_launch_fixed(S, C.sc, C.ids, C.ins_g, S.insb, C.dims + 1, 1, dins, E->cs, E->max_u,
                                   kFixedRuns, st, lc);
        else
            e = count_launch(S, C.sc, C.ids, C.ins_g, S.insb, 0, C.n_ins, 1, dins, E->cs, E->max_u, st, lc);
    }
    if (e) return e;
    if (prof) cudaEventRecord(E->ev[4], st);
    Range r("escher: fold counts");
    return store_finish(S, C, E->sm_count, st, lc);
}

// pins: per batch, the IDs its inserts keep (a horizontal update), or null
static esc_status run_call(Engine* E, int n, const esc_batch* bs, const int32_t* const* pins = nullptr) {
    if (n == 0) return ESC_OK;
    if (n < 0 || n > E->G || !bs) return E->fail(ESC_ERR_INVALID_ARG, "bad batch list");
    std::vector<char> seen(E->G, 0);
    int64_t tot_ins = 0, tot_del = 0;
    for (int b = 0; b < n; ++b) {
        const esc_batch& x = bs[b];
        if (x.graph < 0 || x.graph >= E->G || seen[x.graph]) return E->fail(ESC_ERR_INVALID_ARG, "bad or repeated graph");
        seen[x.graph] = 1;
        if (x.n_ins < 0 || x.n_del < 0) return E->fail(ESC_ERR_INVALID_ARG, "negative count");
        if (x.n_ins > 0 && (!x.ins_offsets || !x.ins_members))
            return E->fail(ESC_ERR_INVALID_ARG, "missing insert arrays");
        if (x.n_ins > 0 && (E->shared.families & kFamT) && !x.ins_timestamps && !(pins && pins[b]))
            return E->fail(ESC_ERR_INVALID_ARG, "timestamps required by the temporal family");
        if (x.n_del > 0 && !x.del_ids) return E->fail(ESC_ERR_INVALID_ARG, "missing delete IDs");
        tot_ins += x.n_ins;
        tot_del += x.n_del;
    }
    if (tot_ins + tot_del > E->max_ins)
        return E->fail(ESC_ERR_OUT_OF_MEMORY, "batch larger than max_batch_hyperedges");
    cudaStream_t st = E->st;
    // stage host inputs
    size_t u_off = 0, u_mem = 0, u_ts = 0, u_del = 0, u_pin = 0;
    for (auto& lo : E->hs_lo) lo = 0;
    int64_t* bins = E->h_lo;
    int64_t* bdel = E->h_lo + (E->G + 1);
    bins[0] = bdel[0] = 0;
    for (int b = 0; b < n; ++b) {
        const esc_batch& x = bs[b];
        BatchIn& B = E->h_batches[b];
        B.graph = x.graph;
        B.n_ins = x.n_ins;
        B.n_del = x.n_del;
        B.ins_lo = bins[b];
        B.del_lo = bdel[b];
        bins[b + 1] = bins[b] + x.n_ins;
        bdel[b + 1] = bdel[b] + x.n_del;
        esc_status s;
        B.off = nullptr;
        B.mem = nullptr;
        B.ts = nullptr;
        B.del = nullptr;
        B.pin = nullptr;
        if (x.n_ins > 0 && pins && pins[b])
            if ((s = stage(E, pins[b], size_t(x.n_ins), E->st_pin, 4, u_pin, size_t(E->max_ins), &B.pin)) != ESC_OK)
                return s;
        if (x.n_ins > 0) {
            bool off_dev = is_device_ptr(x.ins_offsets);
            if ((s = stage(E, x.ins_offsets, size_t(x.n_ins + 1), E->st_off, 0, u_off,
                           size_t(E->max_ins + E->G + 1), &B.off)) != ESC_OK)
                return s;
            if (!off_dev) {
                int64_t nnz = x.ins_offsets[x.n_ins] - x.ins_offsets[0];
                if (x.ins_offsets[0] != 0 || nnz < 0) return E->fail(ESC_ERR_INVALID_ARG, "offsets must start at 0");
                if (nnz > E->max_nnz) return E->fail(ESC_ERR_OUT_OF_MEMORY, "batch members exceed max_batch_incidences");
                if ((s = stage(E, x.ins_members, size_t(nnz), E->st_mem, 1, u_mem, size_t(E->max_nnz), &B.mem)) !=
                    ESC_OK)
                    return s;
            } else {
                if (is_device_ptr(x.ins_members)) B.mem = x.ins_members;
                else return E->fail(ESC_ERR_INVALID_ARG, "device offsets need device members");
            }
            if ((s = stage(E, x.ins_timestamps, size_t(x.n_ins), E->st_ts, 2, u_ts, size_t(E->max_ins), &B.ts)) !=
                ESC_OK)
                return s;
        }
        if (x.n_del > 0)
            if ((s = stage(E, x.del_ids, size_t(x.n_del), E->st_del, 3, u_del, size_t(E->max_ins), &B.del)) != ESC_OK)
                return s;
    }
    {
        esc_status s;
        if ((s = flush_staged(E, E->st_off, 0, u_off)) != ESC_OK || (s = flush_staged(E, E->st_mem, 1, u_mem)) != ESC_OK ||
            (s = flush_staged(E, E->st_ts, 2, u_ts)) != ESC_OK || (s = flush_staged(E, E->st_del, 3, u_del)) != ESC_OK ||
            (s = flush_staged(E, E->st_pin, 4, u_pin)) != ESC_OK)
            return s;
    }
    ESC_CU(cudaMemcpyAsync(E->d_batches, E->h_batches, sizeof(BatchIn) * n, cudaMemcpyHostToDevice, st), "copy");
    ESC_CU(cudaMemcpyAsync(E->d_bins_lo, bins, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st), "copy");
    ESC_CU(cudaMemcpyAsync(E->d_bdel_lo, bdel, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st), "copy");
    E->h_dims[0] = n;
    E->h_dims[1] = tot_ins;
    E->h_dims[2] = tot_del;
    Call C = E->C;
    C.n_batches = n;
    C.n_ins = tot_ins;
    C.n_del = tot_del;
    C.dims = E->d_dims;
    C.pinned = pins != nullptr;
    LaunchCounter lc;
    const bool prof = E->profiling;
    // graph mode: one replay of the fixed launch sequence; a call whose lists
    // need more count runs than the sequence holds fails inside it with the
    // retry status (changing nothing) and runs again with host-planned runs
    for (int attempt = 0; attempt < 2; ++attempt) {
        const bool fixed = E->graph_mode && attempt == 0;
        ESC_CU(cudaMemsetAsync(E->d_sc, 0, sizeof(Scalars), st), "memset");
        ESC_CU(cudaMemcpyAsync(E->d_dims, E->h_dims, sizeof(int64_t) * 3, cudaMemcpyHostToDevice, st), "copy");
        C.fixed = fixed;
        C.grid_batches = fixed ? E->G : n;
        C.grid_ins = fixed ? E->max_ins : tot_ins;
        C.grid_del = fixed ? E->max_ins : tot_del;
        E->cs.cev = prof && !fixed ? E->cev : nullptr;
        E->n_cev = 0;
        if (prof) cudaEventRecord(E->ev[0], st);
        if (fixed) {
            if (!E->gexec) {
                // capture once; every later call replays the same graph
                LaunchCounter lg;
                cudaGraph_t graph = nullptr;
                store_prepare();
                count_prepare();
                ESC_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "capture");
                cudaError_t e = launch_sequence(E, C, true, st, lg);
                cudaError_t e2 = cudaStreamEndCapture(st, &graph);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&E->gexec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (e != cudaSuccess) return E->cuda_fail(e, "graph capture");
                E->graph_kernels = lg.total;
                E->graph_count_kernels = lg.count;
            }
            ESC_CU(cudaGraphLaunch(E->gexec, st), "graph launch");
            lc.total += E->graph_kernels;
            lc.count += E->graph_count_kernels;
        } else {
            ESC_CU(launch_sequence(E, C, false, st, lc, prof), "launch");
        }
        if (prof) cudaEventRecord(E->ev[5], st);
        ESC_CU(cudaMemcpyAsync(E->h_sc, E->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st), "status");
        if (tot_ins > 0)
            ESC_CU(cudaMemcpyAsync(E->h_ids, C.out_local, sizeof(int32_t) * tot_ins, cudaMemcpyDeviceToHost, st),
                   "ids");
        ESC_CU(cudaStreamSynchronize(st), "sync");
        if (E->h_sc->status != kErrRetry) break;
    }
    E->lc.total += lc.total;
    E->lc.count += lc.count;
    if (prof) {
        esc_batch_stats& L = E->last;
        cudaEventElapsedTime(&L.ms_total, E->ev[0], E->ev[5]);
        L.ms_ingest = L.ms_count_del = L.ms_store = L.ms_count_ins = 0.f;
        if (!E->graph_mode || E->h_sc->status == 0) {
            cudaEventElapsedTime(&L.ms_ingest, E->ev[0], E->ev[1]);
            cudaEventElapsedTime(&L.ms_count_del, E->ev[1], E->ev[2]);
            cudaEventElapsedTime(&L.ms_store, E->ev[2], E->ev[3]);
            cudaEventElapsedTime(&L.ms_count_ins, E->ev[3], E->ev[4]);
        }
        L.ms_center = 0.f;
        for (int k = 0; k < E->n_cev; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, E->cev[2 * k], E->cev[2 * k + 1]);
            L.ms_center += ms;
        }
        L.center_launches = E->n_cev;
    }
    E->last.launches = lc.total;
    E->last.count_launches = lc.count;
    E->last.v2h_reads = int64_t(E->h_sc->stats[0]);
    E->last.h2v_reads = int64_t(E->h_sc->stats[1]);
    E->last.meta_reads = int64_t(E->h_sc->stats[2]);
    E->last.triads = int64_t(E->h_sc->stats[3]);
    E->last.alg_entries = int64_t(E->h_sc->stats[4]);
    for (int k = 0; k < 6; ++k) E->last.work[k] = int64_t(E->h_sc->stats[5 + k]);
    E->last.alg_center = int64_t(E->h_sc->stats[11]);
    E->last.alg_open = int64_t(E->h_sc->stats[12]);
    E->last.alg_closed = int64_t(E->h_sc->stats[13]);
    E->last.alg_build = int64_t(E->h_sc->stats[14]);
    E->last.alg_store = int64_t(E->h_sc->stats[15]);
    int status = E->h_sc->status;
    if (status == 0 && E->d_dbg) {
        // debug mode: the store's invariants after the call
        ESC_CU(cudaMemsetAsync(E->d_sc, 0, sizeof(Scalars), st), "memset");
        ESC_CU(store_debug_check(E->S, E->d_sc, E->d_dbg, E->sm_count, st), "debug check");
        ESC_CU(cudaMemcpyAsync(E->h_sc, E->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st), "status");
        ESC_CU(cudaStreamSynchronize(st), "sync");
        status = E->h_sc->status;
    }
    ++E->n_calls;
    if (E->jsonl) {
        const esc_batch_stats& L = E->last;
        fprintf(E->jsonl,
                "{\"call\": %lld, \"batches\": %d, \"inserts\": %lld, \"deletes\": %lld, \"status\": %d, "
                "\"launches\": %lld",
                (long long)E->n_calls, n, (long long)tot_ins, (long long)tot_del, status, (long long)lc.total);
        if (prof)
            fprintf(E->jsonl,
                    ", \"ms_total\": %.4f, \"ms_ingest\": %.4f, \"ms_count_del\": %.4f, \"ms_store\": %.4f, "
                    "\"ms_count_ins\": %.4f, \"ms_center\": %.4f, \"triads\": %lld, \"work\": [%lld, %lld, %lld, "
                    "%lld, %lld, %lld]",
                    L.ms_total, L.ms_ingest, L.ms_count_del, L.ms_store, L.ms_count_ins, L.ms_center,
                    (long long)L.triads, (long long)L.work[0], (long long)L.work[1], (long long)L.work[2],
                    (long long)L.work[3], (long long)L.work[4], (long long)L.work[5]);
        fprintf(E->jsonl, "}\n");
        fflush(E->jsonl);
    }
    if (status != 0) {
        E->err = status == kErrInternal ? "store invariant check failed: " + describe(*E->h_sc) : describe(*E->h_sc);
        return esc_status(status);
    }
    for (int b = 0; b < n; ++b) {
        const esc_batch& x = bs[b];
        if (!x.out_ins_ids || x.n_ins == 0) continue;
        const int32_t* src = E->h_ids + bins[b];
        if (is_device_ptr(x.out_ins_ids))
            ESC_CU(cudaMemcpy(x.out_ins_ids, src, sizeof(int32_t) * x.n_ins, cudaMemcpyHostToDevice), "ids out");
        else
            memcpy(x.out_ins_ids, src, sizeof(int32_t) * x.n_ins);
    }
    return ESC_OK;
}

// Copy n int32 IDs (host or device) to the host and check they are distinct.
static esc_status host_ids(Engine* E, int64_t n, const int32_t* ids, std::vector<int32_t>& out) {
    out.resize(static_cast<size_t>(n));
    if (is_device_ptr(ids))
        ESC_CU(cudaMemcpy(out.data(), ids, sizeof(int32_t) * n, cudaMemcpyDeviceToHost), "ids");
    else
        memcpy(out.data(), ids, sizeof(int32_t) * n);
    std::vector<int32_t> sorted(out);
    std::sort(sorted.begin(), sorted.end());
    for (size_t i = 1; i < sorted.size(); ++i)
        if (sorted[i] == sorted[i - 1])
            return E->fail(ESC_ERR_INVALID_ARG, "hyperedge ID " + std::to_string(sorted[i]) + " repeated");
    return ESC_OK;
}

// Horizontal update (incident vertices inserted into / deleted from live
// hyperedges): each hyperedge ids[j] of graph g gets a new vertex set and
// keeps its ID and timestamp.  As a call: the old hyperedges are deleted and
// the new sets inserted with their IDs kept, so both counts of Alg. 3 see the
// change (triads holding an updated hyperedge leave their old class and
// join their new one).
static esc_status update_members(Engine* E, int32_t g, int64_t n, const int32_t* ids, const int64_t* offsets,
                                 const int32_t* members) {
    if (g < 0 || g >= E->G || n < 0 || (n > 0 && (!ids || !offsets || !members)))
        return E->fail(ESC_ERR_INVALID_ARG, "bad update");
    if (n == 0) return ESC_OK;
    std::vector<int32_t> pin;
    esc_status s = host_ids(E, n, ids, pin);
    if (s != ESC_OK) return s;
    std::vector<int32_t> del(pin);
    std::sort(del.begin(), del.end());
    esc_batch b{};
    b.graph = g;
    b.n_ins = n;
    b.ins_offsets = offsets;
    b.ins_members = members;
    b.ins_timestamps = nullptr;
    b.n_del = n;
    b.del_ids = del.data();
    const int32_t* pins[1] = {pin.data()};
    return run_call(E, 1, &b, pins);
}

// Inserts whose IDs the caller gives (a restored checkpoint; with pin null,
// the ID rule picks them as for any insert): hyperedge j
// takes ID pin[j] (which must be free) and its triads are counted like any
// insert's (the inserted side of Alg. 3).  The graph's high-water mark rises
// to cover the IDs, so later inserts follow the ID rule as if the hyperedges
// had been inserted one by one: free IDs below the mark first, smallest
// first, then fresh ones.  One call per chunk of at most max_ins hyperedges
// and max_nnz members; with chunked set, a failed chunk leaves the earlier
// ones in place (callers that need all-or-nothing pass chunked = false).
static esc_status insert_pinned(Engine* E, int32_t g, int64_t n, const int32_t* pin, const int64_t* offsets,
                                const int32_t* members, const int64_t* timestamps, bool chunked) {
    if (n == 0) return ESC_OK;
    std::vector<int64_t> hoff(size_t(n) + 1);
    if (is_device_ptr(offsets))
        ESC_CU(cudaMemcpy(hoff.data(), offsets, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost), "offsets");
    else
        memcpy(hoff.data(), offsets, sizeof(int64_t) * (n + 1));
    if (hoff[0] != 0) return E->fail(ESC_ERR_INVALID_ARG, "offsets must start at 0");
    std::vector<int64_t> zero_ts;
    if (!timestamps) {
        if (E->shared.families & kFamT) return E->fail(ESC_ERR_INVALID_ARG, "timestamps required by the temporal family");
        zero_ts.assign(static_cast<size_t>(n), 0);
        timestamps = zero_ts.data();
    }
    std::vector<int64_t> rebased;
    int64_t i0 = 0;
    while (i0 < n) {
        int64_t i1 = n;
        if (chunked) {
            i1 = i0;
            while (i1 < n && i1 - i0 < E->max_ins && hoff[i1 + 1] - hoff[i0] <= E->max_nnz) ++i1;
            if (i1 == i0) return E->fail(ESC_ERR_OUT_OF_MEMORY, "a hyperedge is larger than max_batch_incidences");
        }
        rebased.resize(size_t(i1 - i0) + 1);
        for (int64_t i = i0; i <= i1; ++i) rebased[i - i0] = hoff[i] - hoff[i0];
        esc_batch b{};
        b.graph = g;
        b.n_ins = i1 - i0;
        b.ins_offsets = rebased.data();
        b.ins_members = members + hoff[i0];
        b.ins_timestamps = timestamps + i0;
        const int32_t* pins[1] = {pin ? pin + i0 : nullptr};
        esc_status s = run_call(E, 1, &b, pin ? pins : nullptr);
        if (s != ESC_OK) return s;
        i0 = i1;
    }
    return ESC_OK;
}

static esc_status insert_with_ids(Engine* E, int32_t g, int64_t n, const int32_t* ids, const int64_t* offsets,
                                  const int32_t* members, const int64_t* timestamps) {
    if (g < 0 || g >= E->G || n < 0 || (n > 0 && (!ids || !offsets || !members)))
        return E->fail(ESC_ERR_INVALID_ARG, "bad insert");
    if (n == 0) return ESC_OK;
    std::vector<int32_t> pin;
    esc_status s = host_ids(E, n, ids, pin);
    if (s != ESC_OK) return s;
    return insert_pinned(E, g, n, pin.data(), offsets, members, timestamps, false);
}

// Graph g's live hyperedges and vertex lists, in the graph's own IDs.
static esc_status export_graph(Engine* E, int32_t g, int64_t* n_live, int64_t* n_incidences, int32_t* ids,
                               int64_t* timestamps, int64_t* offsets, int32_t* members, int64_t* v_offsets,
                               int32_t* v_members) {
    if (g < 0 || g >= E->G) return E->fail(ESC_ERR_INVALID_ARG, "bad graph");
    ESC_CU(cudaStreamSynchronize(E->st), "sync");
    const Store& S = E->S;
    const int64_t eb = E->ebase[g], vb = E->vbase[g];
    const size_t ne = size_t(E->ecap[g]), nvt = size_t(E->nv[g]);  // ebase and ecap are multiples of 32
    std::vector<int32_t> card(ne);
    std::vector<uint32_t> live(ne / 32);
    ESC_CU(cudaMemcpy(card.data(), S.h_card + eb, ne * 4, cudaMemcpyDeviceToHost), "export");
    ESC_CU(cudaMemcpy(live.data(), S.live + eb / 32, live.size() * 4, cudaMemcpyDeviceToHost), "export");
    if (n_live || n_incidences) {
        int64_t nl = 0, ni = 0;
        for (size_t i = 0; i < ne; ++i)
            if (live[i >> 5] >> (i & 31) & 1) {
                ++nl;
                ni += card[i];
            }
        if (n_live) *n_live = nl;
        if (n_incidences) *n_incidences = ni;
    }
    if (!ids && !timestamps && !offsets && !members && !v_offsets && !v_members) return ESC_OK;
    std::vector<int32_t> vdeg(nvt);
    std::vector<int64_t> hoff(ne), hts(ne), voff(nvt);
    int64_t htail = 0, vtail = 0;
    ESC_CU(cudaMemcpy(hoff.data(), S.h_off + eb, ne * 8, cudaMemcpyDeviceToHost), "export");
    ESC_CU(cudaMemcpy(hts.data(), S.h_ts + eb, ne * 8, cudaMemcpyDeviceToHost), "export");
    if (nvt) {
        ESC_CU(cudaMemcpy(vdeg.data(), S.v_deg + vb, nvt * 4, cudaMemcpyDeviceToHost), "export");
        ESC_CU(cudaMemcpy(voff.data(), S.v_off + vb, nvt * 8, cudaMemcpyDeviceToHost), "export");
    }
    ESC_CU(cudaMemcpy(&htail, S.hp.tail, 8, cudaMemcpyDeviceToHost), "export");
    ESC_CU(cudaMemcpy(&vtail, S.vp.tail, 8, cudaMemcpyDeviceToHost), "export");
    std::vector<int32_t> harena(static_cast<size_t>(htail)), varena(static_cast<size_t>(vtail));
    if (htail) ESC_CU(cudaMemcpy(harena.data(), S.hp.arena, size_t(htail) * 4, cudaMemcpyDeviceToHost), "export");
    if (vtail) ESC_CU(cudaMemcpy(varena.data(), S.vp.arena, size_t(vtail) * 4, cudaMemcpyDeviceToHost), "export");
    int64_t k = 0, p = 0;
    if (offsets) offsets[0] = 0;
    for (size_t i = 0; i < ne; ++i) {
        if (!(live[i >> 5] >> (i & 31) & 1)) continue;
        if (ids) ids[k] = int32_t(i);
        if (timestamps) timestamps[k] = hts[i];
        for (int j = 0; j < card[i]; ++j, ++p)
            if (members) members[p] = int32_t(harena[size_t(hoff[i]) + j] - vb);
        ++k;
        if (offsets) offsets[k] = p;
    }
    int64_t q = 0;
    if (v_offsets) v_offsets[0] = 0;
    for (size_t v = 0; v < nvt; ++v) {
        std::vector<int32_t> l(varena.begin() + voff[v], varena.begin() + voff[v] + vdeg[v]);
        std::sort(l.begin(), l.end());
        if (v_members)
            for (int32_t x : l) v_members[q++] = int32_t(x - eb);
        else
            q += int64_t(l.size());
        if (v_offsets) v_offsets[v + 1] = q;
    }
    return ESC_OK;
}

// The h2h mapping (line graph) of graph g, assembled on the host from a copy
// of the store: for each live hyperedge in ascending ID order, the other live
// hyperedges sharing at least s of its vertices, ascending, with the number
// shared.  s = 1 gives the line graph, s > 1 the s-line graph.
static esc_status export_h2h(Engine* E, int32_t g, int32_t s, int64_t* n_entries, int64_t* offsets,
                             int32_t* neighbours, int32_t* overlaps) {
    if (s < 1) return E->fail(ESC_ERR_INVALID_ARG, "s must be at least 1");
    int64_t nl = 0, ni = 0;
    esc_status st = export_graph(E, g, &nl, &ni, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st != ESC_OK) return st;
    const size_t nvt = size_t(E->nv[g]);
    std::vector<int32_t> ids(size_t(nl) + 1), mem(size_t(ni) + 1), vmem(size_t(ni) + 1);
    std::vector<int64_t> off(size_t(nl) + 1), voff(nvt + 1);
    st = export_graph(E, g, nullptr, nullptr, ids.data(), nullptr, off.data(), mem.data(), voff.data(), vmem.data());
    if (st != ESC_OK) return st;
    std::vector<int32_t> pos(size_t(E->ecap[g]), -1), cnt(size_t(nl), 0), touched;
    for (int64_t k = 0; k < nl; ++k) pos[size_t(ids[k])] = int32_t(k);
    int64_t q = 0;
    if (offsets) offsets[0] = 0;
    for (int64_t k = 0; k < nl; ++k) {
        touched.clear();
        for (int64_t j = off[k]; j < off[k + 1]; ++j) {
            const int32_t x = mem[j];
            for (int64_t e = voff[x]; e < voff[x + 1]; ++e) {
                const int32_t p = pos[size_t(vmem[e])];
                if (p == k) continue;
                if (cnt[p]++ == 0) touched.push_back(p);
            }
        }
        std::sort(touched.begin(), touched.end());
        for (int32_t p : touched) {
            if (cnt[p] >= s) {
                if (neighbours) neighbours[q] = ids[p];
                if (overlaps) overlaps[q] = cnt[p];
                ++q;
            }
            cnt[p] = 0;
        }
        if (offsets) offsets[k + 1] = q;
    }
    if (n_entries) *n_entries = q;
    return ESC_OK;
}

static esc_status read_counts(Engine* E, int32_t g, esc_triad_type type, int64_t window, uint64_t* out,
                              int32_t n_out) {
    if (g < 0 || g >= E->G || !out) return E->fail(ESC_ERR_INVALID_ARG, "bad graph or output");
    int off, len;
    uint32_t fam;
    switch (type) {
        case ESC_TRIAD_HYPEREDGE: off = 0; len = kNH; fam = kFamH; break;
        case ESC_TRIAD_VERTEX: off = kOffV; len = kNV; fam = kFamV | kFamV12; break;
        case ESC_TRIAD_TEMPORAL: off = kOffT; len = kNT; fam = kFamT; break;
        default: return E->fail(ESC_ERR_INVALID_ARG, "bad triad type");
    }
    if (n_out < len) return E->fail(ESC_ERR_INVALID_ARG, "output too small");
    if (!(E->shared.families & fam)) return E->fail(ESC_ERR_UNSUPPORTED, "family not maintained");
    if (type == ESC_TRIAD_TEMPORAL && window != E->shared.delta)
        return E->fail(ESC_ERR_UNSUPPORTED, "temporal counts are kept for the configured delta only");
    ESC_CU(cudaMemcpyAsync(E->h_counts, E->S.counts + int64_t(g) * kCStride, sizeof(uint64_t) * kCStride,
                           cudaMemcpyDeviceToHost, E->st),
           "counts");
    ESC_CU(cudaStreamSynchronize(E->st), "sync");
    memcpy(out, E->h_counts + off, sizeof(uint64_t) * len);
    return ESC_OK;
}

namespace {

__global__ void k_mark_sel(Store S, Scalars* sc, const int32_t* ids, int64_t n, int32_t* out_global) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t h = ids[i];
    if (h < 0 || h >= S.e_total || !bit_test(S.live, h)) {
        set_error(sc, kErrNotFound, -1, i, h);
        out_global[i] = 0;
        return;
    }
    out_global[i] = h;
    uint32_t old = atomicOr(&S.insb[h >> 5], 1u << (h & 31));
    if (old & (1u << (h & 31))) set_error(sc, kErrInvalid, -1, i, h);
}

__global__ void k_unmark_sel(Store S, const int32_t* ids, int64_t n) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t h = ids[i];
    if (h >= 0 && h < S.e_total) atomicAnd(&S.insb[h >> 5], ~(1u << (h & 31)));
}

__global__ void k_latch_api(Scalars* sc) { sc->gate = sc->status; }

}  // namespace

static esc_status local_triads(Engine* E, int64_t n, const int32_t* ids, uint64_t* oh, uint64_t* ov, uint64_t* ot,
                               float* ms_out = nullptr) {
    if (n < 0 || (n > 0 && !ids)) return E->fail(ESC_ERR_INVALID_ARG, "bad id list");
    cudaStream_t st = E->st;
    const Store& S = E->S;
    E->cs.cev = nullptr;  // not timed
    int32_t* d_ids = nullptr;
    int32_t* d_glob = nullptr;
    ESC_CU(cudaMalloc(&d_ids, sizeof(int32_t) * (n > 0 ? n : 1)), "alloc");
    ESC_CU(cudaMalloc(&d_glob, sizeof(int32_t) * (n > 0 ? n : 1)), "alloc");
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        cudaFree(d_ids);
        cudaFree(d_glob);
    };
    if (n > 0) {
        cudaError_t e = cudaMemcpyAsync(d_ids, ids, sizeof(int32_t) * n, cudaMemcpyDefault, st);
        if (e != cudaSuccess) { cleanup(); return E->cuda_fail(e, "copy ids"); }
    }
    cudaMemsetAsync(E->d_sc, 0, sizeof(Scalars), st);
    uint64_t* dside = S.dcounts + int64_t(S.n_graphs) * kCStride;
    cudaMemsetAsync(dside, 0, sizeof(uint64_t) * kCStride, st);
    LaunchCounter lc;
    if (ms_out) cudaEventRecord(E->ev[0], st);
    // local counts are whole counts, whatever work split the graph has
    CountScratch whole = E->cs;
    whole.split_world = 1;
    if (n > 0) {
        k_mark_sel<<<unsigned((n + 255) / 256), 256, 0, st>>>(S, E->d_sc, d_ids, n, d_glob);
        k_latch_api<<<1, 1, 0, st>>>(E->d_sc);
        for (int64_t lo = 0; lo < n; lo += E->cs.cap) {
            int64_t hi = lo + E->cs.cap < n ? lo + E->cs.cap : n;
            cudaError_t e = count_launch(S, E->d_sc, d_glob, nullptr, S.insb, lo, hi, 1, dside, whole,
                                         E->max_u, st, lc);
            if (e != cudaSuccess) { cleanup(); return E->cuda_fail(e, "count"); }
        }
        k_unmark_sel<<<unsigned((n + 255) / 256), 256, 0, st>>>(S, d_glob, n);
    }
    if (ms_out) cudaEventRecord(E->ev[1], st);
    cudaMemcpyAsync(E->h_counts, dside, sizeof(uint64_t) * kCStride, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(E->h_sc, E->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
    cudaMemsetAsync(dside, 0, sizeof(uint64_t) * kCStride, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return E->cuda_fail(e, "sync");
    if (ms_out) cudaEventElapsedTime(ms_out, E->ev[0], E->ev[1]);
    E->lc.total += lc.total + (n > 0 ? 3 : 0);
    E->lc.count += lc.count;
    if (E->h_sc->status) {
        E->err = describe(*E->h_sc);
        return esc_status(E->h_sc->status);
    }
    if (oh && (E->shared.families & kFamH)) memcpy(oh, E->h_counts, sizeof(uint64_t) * kNH);
    if (ov && (E->shared.families & kFamV)) memcpy(ov, E->h_counts + kOffV, sizeof(uint64_t) * kNV);
    if (ot && (E->shared.families & kFamT)) memcpy(ot, E->h_counts + kOffT, sizeof(uint64_t) * kNT);
    return ESC_OK;
}

// Time the counter's launch shapes (and, without the temporal family, the
// restricted lists) on the engine's own data -- the triads of a sample of
// live hyperedges, counted and discarded -- and keep the fastest.
static esc_status autotune(Engine* E, int64_t n, const int32_t* ids, int32_t reps, esc_tune_result* out) {
    if (n <= 0 || !ids || reps <= 0 || !out) return E->fail(ESC_ERR_INVALID_ARG, "bad sample");
    CountScratch& cs = E->cs;
    const int shapes[4] = {0, 1, 2, 3};
    const int64_t r_cap0 = cs.r_cap;
    int32_t* const r_pool0 = cs.r_pool;
    int32_t* extra = nullptr;
    const bool try_r = !(E->shared.families & kFamT);
    if (try_r && r_cap0 == 0) {
        const int64_t want =
            std::min<int64_t>(std::max<int64_t>(16 * E->inc_cap, int64_t(1) << 24), (int64_t(1) << 31) - 64);
        if (cudaMalloc(&extra, sizeof(int32_t) * want) != cudaSuccess) {
            cudaGetLastError();
            extra = nullptr;
        } else {
            cs.r_pool = extra;
            cs.r_cap = want;
        }
    }
    for (int k = 0; k < 8; ++k) out->ms[k] = -1.f;
    for (int k = 0; k < 3; ++k) out->ms_table[k] = out->ms_m1[k] = -1.f;
    float best = 3.4e38f;
    int best_shape = cs.center_small, best_r = r_cap0 > 0 ? 1 : 0;
    for (int r = 0; r < 2; ++r) {
        if (r == 1 && (!try_r || cs.r_cap == 0)) break;
        const int64_t cap_now = cs.r_cap;
        if (r == 0) cs.r_cap = 0;
        for (int k = 0; k < 4; ++k) {
            cs.center_small = shapes[k];
            float t = 3.4e38f;
            for (int rep = 0; rep <= reps; ++rep) {  // the first run warms up
                float ms = 0.f;
                esc_status s = local_triads(E, n, ids, nullptr, nullptr, nullptr, &ms);
                if (s != ESC_OK) {
                    cs.r_cap = r_cap0;
                    cs.r_pool = r_pool0;
                    if (extra) cudaFree(extra);
                    return s;
                }
                if (rep > 0) t = std::min(t, ms);
            }
            out->ms[r * 4 + k] = t;
            if (t < best) {
                best = t;
                best_shape = shapes[k];
                best_r = r;
            }
        }
        if (r == 0) cs.r_cap = cap_now;
    }
    cs.center_small = best_shape;
    if (best_r == 1) {
        if (extra) E->allocs.push_back(extra);  // kept for the engine's life
        extra = nullptr;
    } else {
        cs.r_cap = r_cap0;
        cs.r_pool = r_pool0;
    }
    // the intersection strategy by neighbourhood size, then the per-pair
    // side weight, each with the choices made so far
    auto time_now = [&](float* best_ms) -> esc_status {
        float t = 3.4e38f;
        for (int rep = 0; rep <= reps; ++rep) {
            float ms = 0.f;
            esc_status s = local_triads(E, n, ids, nullptr, nullptr, nullptr, &ms);
            if (s != ESC_OK) return s;
            if (rep > 0) t = std::min(t, ms);
        }
        *best_ms = t;
        return ESC_OK;
    };
    const int tables[3] = {256, 512, 1024}, m1s[3] = {50, 100, 200};
    float bt = 3.4e38f, bm = 3.4e38f;
    int64_t best_table = cs.big_nh, best_m1 = cs.m1_pct;
    for (int k = 0; k < 3; ++k) {
        cs.big_nh = tables[k];
        esc_status s = time_now(&out->ms_table[k]);
        if (s != ESC_OK) {
            if (extra) cudaFree(extra);
            return s;
        }
        if (out->ms_table[k] < bt) {
            bt = out->ms_table[k];
            best_table = tables[k];
        }
    }
    cs.big_nh = best_table;
    for (int k = 0; k < 3; ++k) {
        cs.m1_pct = m1s[k];
        esc_status s = time_now(&out->ms_m1[k]);
        if (s != ESC_OK) {
            if (extra) cudaFree(extra);
            return s;
        }
        if (out->ms_m1[k] < bm) {
            bm = out->ms_m1[k];
            best_m1 = m1s[k];
        }
    }
    cs.m1_pct = best_m1;
    if (extra) cudaFree(extra);
    if (E->gexec) {  // a captured sequence holds the old shape
        cudaGraphExecDestroy(E->gexec);
        E->gexec = nullptr;
    }
    out->center_shape = best_shape;
    out->restricted = best_r;
    out->table_from = int32_t(best_table);
    out->m1_pct = int32_t(best_m1);
    return ESC_OK;
}

}  // namespace esc

using esc::Engine;

struct esc_graph {
    Engine* e;
};
struct esc_group {
    Engine* e;
};

namespace esc {
esc_status group_limits(const esc_group* grp, int32_t* n_graphs, int64_t* max_updates, int64_t* max_nnz,
                        uint32_t* families, int* device) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    const Engine* E = grp->e;
    *n_graphs = E->G;
    *max_updates = E->max_ins;
    *max_nnz = E->max_nnz;
    *families = E->shared.families;
    *device = E->dev;
    return ESC_OK;
}
}  // namespace esc

namespace esc {
static esc_status set_split(Engine* E, int32_t rank, int32_t world) {
    if (world < 2 || rank < 0 || rank >= world) return E->fail(ESC_ERR_INVALID_ARG, "bad rank or world size");
    if (E->cs.split_world > 1) return E->fail(ESC_ERR_UNSUPPORTED, "the work split is already set");
    if (E->graph_mode) return E->fail(ESC_ERR_UNSUPPORTED, "the work split needs graph launch off");
    if (rank != 0) {
        // the counts held now stay with rank 0; the other ranks' shares start at zero
        ESC_CU(cudaMemsetAsync(E->S.counts, 0, sizeof(uint64_t) * int64_t(E->G) * kCStride, E->st), "zero counts");
        ESC_CU(cudaStreamSynchronize(E->st), "sync");
    }
    E->cs.split_rank = rank;
    E->cs.split_world = world;
    return ESC_OK;
}
}  // namespace esc

extern "C" {

const char* esc_version(void) { return "escher-gb300 0.1 (sm_103a)"; }

esc_status esc_group_create(const esc_config* shared, int32_t n_graphs, const esc_config* graph_cfg,
                            void* cuda_stream, esc_group** out) {
    if (!out) return ESC_ERR_INVALID_ARG;
    *out = nullptr;
    esc_status s = esc::check_cfg(shared, false);
    if (s != ESC_OK || n_graphs <= 0 || !graph_cfg) {
        esc::t_create_error = "invalid configuration";
        return s != ESC_OK ? s : ESC_ERR_INVALID_ARG;
    }
    for (int g = 0; g < n_graphs; ++g)
        if ((s = esc::check_cfg(&graph_cfg[g], true)) != ESC_OK) {
            esc::t_create_error = "invalid graph configuration " + std::to_string(g);
            return s;
        }
    Engine* E = new Engine();
    s = esc::build_engine(E, *shared, n_graphs, graph_cfg, static_cast<cudaStream_t>(cuda_stream));
    if (s != ESC_OK) {
        esc::t_create_error = E->err;
        delete E;
        return s;
    }
    *out = new esc_group{E};
    return ESC_OK;
}

esc_status esc_group_bytes(const esc_config* shared, int32_t n_graphs, const esc_config* graph_cfg,
                           int64_t* out_bytes) {
    if (!out_bytes) return ESC_ERR_INVALID_ARG;
    *out_bytes = 0;
    esc_status s = esc::check_cfg(shared, false);
    if (s != ESC_OK || n_graphs <= 0 || !graph_cfg) return s != ESC_OK ? s : ESC_ERR_INVALID_ARG;
    for (int g = 0; g < n_graphs; ++g)
        if ((s = esc::check_cfg(&graph_cfg[g], true)) != ESC_OK) return s;
    Engine E;
    E.dry = true;
    s = esc::build_engine(&E, *shared, n_graphs, graph_cfg, nullptr);
    if (s != ESC_OK) return s;
    *out_bytes = E.dry_bytes;
    return ESC_OK;
}

esc_status esc_group_apply(esc_group* grp, int32_t n, const esc_batch* batches) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    return esc::run_call(grp->e, n, batches);
}

esc_status esc_group_update_members(esc_group* grp, int32_t graph, int64_t n, const int32_t* ids,
                                    const int64_t* offsets, const int32_t* members) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    return esc::update_members(grp->e, graph, n, ids, offsets, members);
}

esc_status esc_group_insert_with_ids(esc_group* grp, int32_t graph, int64_t n, const int32_t* ids,
                                     const int64_t* offsets, const int32_t* members, const int64_t* timestamps) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    return esc::insert_with_ids(grp->e, graph, n, ids, offsets, members, timestamps);
}

esc_status esc_group_export_sizes(esc_group* grp, int32_t graph, int64_t* n_live, int64_t* n_incidences) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    return esc::export_graph(grp->e, graph, n_live, n_incidences, nullptr, nullptr, nullptr, nullptr, nullptr,
                             nullptr);
}

esc_status esc_group_export(esc_group* grp, int32_t graph, int32_t* ids, int64_t* timestamps, int64_t* offsets,
                            int32_t* members, int64_t* v_offsets, int32_t* v_members) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    return esc::export_graph(grp->e, graph, nullptr, nullptr, ids, timestamps, offsets, members, v_offsets,
                             v_members);
}

esc_status esc_group_export_h2h(esc_group* grp, int32_t graph, int32_t s, int64_t* n_entries, int64_t* offsets,
                                int32_t* neighbours, int32_t* overlaps) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    return esc::export_h2h(grp->e, graph, s, n_entries, offsets, neighbours, overlaps);
}

esc_status esc_group_triads(esc_group* grp, int32_t graph, esc_triad_type type, int64_t window, uint64_t* out,
                            int32_t n_out) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    return esc::read_counts(grp->e, graph, type, window, out, n_out);
}

esc_status esc_group_autotune(esc_group* grp, int32_t graph, int64_t n_ids, const int32_t* ids, int32_t reps,
                              esc_tune_result* out) {
    if (!grp || graph < 0 || graph >= grp->e->G || n_ids <= 0 || !ids) return ESC_ERR_INVALID_ARG;
    // the sample's IDs are the graph's own; the counter works on global IDs
    std::vector<int32_t> glob(ids, ids + n_ids);
    const int64_t base = grp->e->ebase[graph];
    for (auto& h : glob) h = int32_t(h + base);
    return esc::autotune(grp->e, n_ids, glob.data(), reps, out);
}

esc_status esc_group_set_split(esc_group* grp, int32_t rank, int32_t world) {
    return grp ? esc::set_split(grp->e, rank, world) : ESC_ERR_INVALID_ARG;
}

esc_status esc_group_set_graph_launch(esc_group* grp, int32_t on) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    if (on && grp->e->cs.split_world > 1) return grp->e->fail(ESC_ERR_UNSUPPORTED, "graph launch with a work split");
    cudaError_t e = esc::set_graph_mode(grp->e, on != 0);
    return e == cudaSuccess ? ESC_OK : grp->e->cuda_fail(e, "graph mode");
}

esc_status esc_group_destroy(esc_group* grp) {
    if (!grp) return ESC_OK;
    delete grp->e;
    delete grp;
    return ESC_OK;
}

const char* esc_group_last_error(const esc_group* grp) {
    return grp ? grp->e->err.c_str() : esc::t_create_error.c_str();
}

esc_status esc_group_set_profiling(esc_group* grp, int32_t on) {
    if (!grp) return ESC_ERR_INVALID_ARG;
    grp->e->profiling = on != 0;
    return ESC_OK;
}

esc_status esc_group_last_stats(esc_group* grp, esc_batch_stats* out) {
    if (!grp || !out) return ESC_ERR_INVALID_ARG;
    *out = grp->e->last;
    return ESC_OK;
}

int64_t esc_group_launch_count(const esc_group* grp) { return grp ? grp->e->lc.total : 0; }

esc_status esc_create(const esc_config* cfg, int64_t n_he, const int64_t* offsets, const int32_t* members,
                      const int64_t* timestamps, void* cuda_stream, esc_graph** out) {
    if (!out) return ESC_ERR_INVALID_ARG;
    *out = nullptr;
    esc_status s = esc::check_cfg(cfg, false);
    if (s != ESC_OK) {
        esc::t_create_error = "invalid configuration";
        return s;
    }
    if (n_he < 0 || (n_he > 0 && (!offsets || !members))) {
        esc::t_create_error = "invalid initial hypergraph";
        return ESC_ERR_INVALID_ARG;
    }
    if (n_he > 0 && (cfg->families & esc::kFamT) && !timestamps) {
        esc::t_create_error = "timestamps required by the temporal family";
        return ESC_ERR_INVALID_ARG;
    }
    Engine* E = new Engine();
    s = esc::build_engine(E, *cfg, 1, cfg, static_cast<cudaStream_t>(cuda_stream));
    if (s != ESC_OK) {
        esc::t_create_error = E->err;
        delete E;
        return s;
    }
    esc_graph* g = new esc_graph{E};
    if (n_he > 0) {
        // initial hyperedges enter as insert batches, in order, so they get
        // IDs 0..n_he-1 and their triads are counted by the same kernels
        s = esc::insert_pinned(E, 0, n_he, nullptr, offsets, members, timestamps, true);
        if (s != ESC_OK) {
            esc::t_create_error = E->err;
            esc_destroy(g);
            return s;
        }
    }
    *out = g;
    return ESC_OK;
}

esc_status esc_apply_batch(esc_graph* g, int64_t n_ins, const int64_t* ins_offsets, const int32_t* ins_members,
                           const int64_t* ins_timestamps, int64_t n_del, const int32_t* del_ids, int32_t* out_ins_ids) {
    if (!g) return ESC_ERR_INVALID_ARG;
    if (n_ins == 0 && n_del == 0) return ESC_OK;
    esc_batch b{};
    b.graph = 0;
    b.n_ins = n_ins;
    b.ins_offsets = ins_offsets;
    b.ins_members = ins_members;
    b.ins_timestamps = ins_timestamps;
    b.n_del = n_del;
    b.del_ids = del_ids;
    b.out_ins_ids = out_ins_ids;
    return esc::run_call(g->e, 1, &b);
}

esc_status esc_update_members(esc_graph* g, int64_t n, const int32_t* ids, const int64_t* offsets,
                              const int32_t* members) {
    if (!g) return ESC_ERR_INVALID_ARG;
    return esc::update_members(g->e, 0, n, ids, offsets, members);
}

esc_status esc_triads(esc_graph* g, esc_triad_type type, int64_t window, uint64_t* out, int32_t n_out) {
    if (!g) return ESC_ERR_INVALID_ARG;
    return esc::read_counts(g->e, 0, type, window, out, n_out);
}

esc_status esc_local_triads(esc_graph* g, int64_t n_ids, const int32_t* ids, uint64_t* out_hyperedge,
                            uint64_t* out_vertex, uint64_t* out_temporal) {
    if (!g) return ESC_ERR_INVALID_ARG;
    return esc::local_triads(g->e, n_ids, ids, out_hyperedge, out_vertex, out_temporal);
}

esc_status esc_autotune(esc_graph* g, int64_t n_ids, const int32_t* ids, int32_t reps, esc_tune_result* out) {
    if (!g) return ESC_ERR_INVALID_ARG;
    return esc::autotune(g->e, n_ids, ids, reps, out);
}

esc_status esc_set_split(esc_graph* g, int32_t rank, int32_t world) {
    return g ? esc::set_split(g->e, rank, world) : ESC_ERR_INVALID_ARG;
}

esc_status esc_set_graph_launch(esc_graph* g, int32_t on) {
    if (!g) return ESC_ERR_INVALID_ARG;
    if (on && g->e->cs.split_world > 1) return g->e->fail(ESC_ERR_UNSUPPORTED, "graph launch with a work split");
    cudaError_t e = esc::set_graph_mode(g->e, on != 0);
    return e == cudaSuccess ? ESC_OK : g->e->cuda_fail(e, "graph mode");
}

esc_status esc_destroy(esc_graph* g) {
    if (!g) return ESC_OK;
    delete g->e;
    delete g;
    return ESC_OK;
}

const char* esc_last_error(const esc_graph* g) { return g ? g->e->err.c_str() : esc::t_create_error.c_str(); }

esc_status esc_set_profiling(esc_graph* g, int32_t on) {
    if (!g) return ESC_ERR_INVALID_ARG;
    g->e->profiling = on != 0;
    return ESC_OK;
}

esc_status esc_last_stats(esc_graph* g, esc_batch_stats* out) {
    if (!g || !out) return ESC_ERR_INVALID_ARG;
    *out = g->e->last;
    return ESC_OK;
}

int64_t esc_launch_count(const esc_graph* g) { return g ? g->e->lc.total : 0; }

esc_status esc_export_sizes(esc_graph* g, int64_t* n_live, int64_t* n_incidences) {
    if (!g) return ESC_ERR_INVALID_ARG;
    return esc::export_graph(g->e, 0, n_live, n_incidences, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

esc_status esc_export(esc_graph* g, int32_t* ids, int64_t* timestamps, int64_t* offsets, int32_t* members,
                      int64_t* v_offsets, int32_t* v_members) {
    if (!g) return ESC_ERR_INVALID_ARG;
    return esc::export_graph(g->e, 0, nullptr, nullptr, ids, timestamps, offsets, members, v_offsets, v_members);
}

esc_status esc_export_h2h(esc_graph* g, int32_t s, int64_t* n_entries, int64_t* offsets, int32_t* neighbours,
                          int32_t* overlaps) {
    if (!g) return ESC_ERR_INVALID_ARG;
    return esc::export_h2h(g->e, 0, s, n_entries, offsets, neighbours, overlaps);
}

esc_status esc_insert_with_ids(esc_graph* g, int64_t n, const int32_t* ids, const int64_t* offsets,
                               const int32_t* members, const int64_t* timestamps) {
    if (!g) return ESC_ERR_INVALID_ARG;
    return esc::insert_with_ids(g->e, 0, n, ids, offsets, members, timestamps);
}

esc_status esc_restore(const esc_config* cfg, int64_t n_he, const int32_t* ids, const int64_t* offsets,
                       const int32_t* members, const int64_t* timestamps, void* cuda_stream, esc_graph** out) {
    if (!out) return ESC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_he < 0 || (n_he > 0 && (!ids || !offsets || !members))) {
        esc::t_create_error = "invalid checkpoint";
        return ESC_ERR_INVALID_ARG;
    }
    esc_graph* g = nullptr;
    esc_status s = esc_create(cfg, 0, nullptr, nullptr, nullptr, cuda_stream, &g);
    if (s != ESC_OK) return s;
    std::vector<int32_t> pin;
    if (n_he > 0) {
        s = esc::host_ids(g->e, n_he, ids, pin);
        if (s == ESC_OK) s = esc::insert_pinned(g->e, 0, n_he, pin.data(), offsets, members, timestamps, true);
    }
    if (s != ESC_OK) {
        esc::t_create_error = g->e->err;
        esc_destroy(g);
        return s;
    }
    *out = g;
    return ESC_OK;
}

}  // extern "C"

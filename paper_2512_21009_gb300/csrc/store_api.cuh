// store_api.cuh -- host-side launch entry points of the store and counter
// kernels, called by the C ABI layer (api.cu).
#pragma once

#include <algorithm>

#include "escher_internal.cuh"

namespace esc {

struct LaunchCounter {
    int64_t total = 0;   // kernels launched
    int64_t count = 0;   // triad-count kernels launched
};

// store.cu
cudaError_t store_ingest(const Store& S, const Call& C, const int64_t* b_ins_lo, const int64_t* b_del_lo,
                         int64_t max_u, int sm_count, cudaStream_t st, LaunchCounter& lc);
cudaError_t store_delete(const Store& S, const Call& C, int sm_count, cudaStream_t st, LaunchCounter& lc);
cudaError_t store_insert(const Store& S, const Call& C, int sm_count, cudaStream_t st, LaunchCounter& lc);
cudaError_t store_finish(const Store& S, const Call& C, int sm_count, cudaStream_t st, LaunchCounter& lc);
// kernel attributes, set once before any launch (and before a capture)
void store_prepare();
void count_prepare();
// latch the status into the gate (later kernels then change nothing)
cudaError_t store_latch(const Call& C, cudaStream_t st, LaunchCounter& lc);

// count.cu
struct CountScratch {
    // per changed hyperedge of one run
    int64_t cap = 0;                 // changed hyperedges per run
    int32_t* sizes = nullptr;        // [cap] sum of member degrees (entries of N(h) with repeats)
    int64_t* nh_off = nullptr;       // [cap+1] start of each N(h) list
    int32_t* nh_n = nullptr;         // [cap] length of each N(h) list
    int64_t* nh_toff = nullptr;      // [cap] start of the hash table of a large N(h)
    int32_t* nh_tcap = nullptr;      // [cap] its slots (0: no table)
    int32_t* order = nullptr;        // [cap] processing order of k_nh_build: large neighbourhoods first
    int32_t* oflag = nullptr;        // [cap]
    int64_t* opre = nullptr;         // [cap+1]
    // neighbour lists N(h) and the inverted candidate lists L(g1)
    int64_t list_cap = 0;            // entries
    int32_t* nh_g = nullptr;         // [list_cap] neighbour g
    uint64_t* nh_xv = nullptr;       // [list_cap] |h & g| (bits 0-15), |g| (16-30), g changed (31),
                                     // smallest shared vertex (32-63); a table slot holds |h & g| and the vertex
    int64_t* nh_ts = nullptr;        // [list_cap] timestamp of g (temporal family only)
    int32_t* l_i = nullptr;          // [list_cap] index of h in the run
    uint64_t* l_xv = nullptr;        // [list_cap] as nh_xv
    int32_t* l_q = nullptr;          // [list_cap] position of g1 in the list of N(h)
    int32_t* nh_flag = nullptr;      // [cap] bit 0: N(h)'s list is sorted by (|g|, g)
    // per hyperedge ID
    int64_t e_cap = 0;
    int32_t* lcnt = nullptr;         // [e_cap] candidate pairs (g1, .) per g1; zero between runs
    int32_t* lfill = nullptr;        // [e_cap]
    int64_t* loffg = nullptr;        // [e_cap] start of L(g1)
    int32_t* d_list = nullptr;       // [e_cap] distinct g1 of the run
    int32_t* d_cnt = nullptr;        // [e_cap] |L(d_list[j])|
    int32_t* d_items = nullptr;      // [e_cap] work items of d_list[j]
    int64_t* d_loff = nullptr;       // [e_cap+1]
    int64_t* d_item_start = nullptr; // [e_cap+1]
    // per distinct g1 (oriented counter): its size, sum of member degrees and
    // h2v offset; and for each centre item its g1's index j
    int32_t* d_k1 = nullptr;         // [e_cap]
    int64_t* d_u1 = nullptr;         // [e_cap]
    int64_t* d_hoff = nullptr;       // [e_cap]
    int32_t* item_j = nullptr;       // [items_cap]
    int64_t items_cap = 0;
    int64_t* block_sums = nullptr;   // scan scratch
    int64_t n_block_sums = 0;
    // per-block overflow hash tables
    int n_cta_nh = 0, n_cta_c = 0;   // persistent grids of the two counting kernels
    int64_t gs_nh = 0, gs_c = 0;     // slots of one overflow table
    int32_t* onh_keys = nullptr;
    uint32_t* onh_vals = nullptr;
    int32_t* onh_aux = nullptr;
    int32_t* onh_list = nullptr;
    uint32_t* onh_hist = nullptr;    // per block: x histograms for |h| above the shared-memory limit
    int32_t* oc_keys = nullptr;
    uint32_t* oc_vals = nullptr;
    uint32_t* oc_mark = nullptr;
    int32_t* oc_list = nullptr;
    int32_t* oc_lk = nullptr;
    int64_t* oc_lts = nullptr;
    int32_t* oc_lkey = nullptr;      // keys of a global N(g1) in list order
    int32_t* oc_pf = nullptr;        // the part of a global N(g1) above g1 in (|f|, f) order: f
    uint32_t* oc_pm = nullptr;       // ... and |g1 & f| | |f| << 16 | f changed << 31
    // restricted incidence lists of a large N(h): for each vertex u of the
    // graph, the neighbours f of h that hold u (a dense index over the
    // graph's vertices, then the lists)
    int32_t* r_pool = nullptr;       // [r_cap] int32 entries
    int64_t r_cap = 0;
    int64_t* r_off = nullptr;        // [cap] start of h's index in the pool, -1: none
    int64_t r_min = 4096;            // sum of member degrees from which h gets the lists
    int64_t big_nh = 512;            // sum of member degrees above which N(h) gets a table and a filter
    int64_t m1_pct = 100;            // visit N(g1) instead of N(h) when |N(g1)| * 100 < |N(h)| * m1_pct
    int64_t smem_slots = 1 << 30;    // cap on shared-memory table sizes (tests lower it)
    int center_small = 3;            // centre blocks per SM x threads: 3: 3 x 256, 1: 2 x 256, 0: 1 x 512, 2: 2 x 512
    bool orient = true;              // search closed pairs in (|g|, g) order (not with restricted lists)
    // temporal family, open triads centred at h (k_open_h): lists of at most
    // oh_smem entries are sorted in shared memory, longer ones of at most
    // min(oh_max, oh_cap) in the block's global scratch (oh_cap a power of
    // two, the arrays strided by oh_cap + 1); longer ones are left to the
    // centre kernel
    int oh_smem = 8192;
    int oh_max = 65536;
    int64_t oh_cap = 0;
    int64_t* oh_t = nullptr;
    int32_t* oh_i = nullptr;
    int32_t* oh_p = nullptr;
    uint32_t* oh_k = nullptr;
    uint32_t* oh_p1 = nullptr;
    uint32_t* oh_pc = nullptr;
    // work split of one hypergraph across ranks: count_launch counts only
    // this rank's contiguous share (by neighbourhood size) of a side
    int split_rank = 0, split_world = 1;
    int c_per_sm = 4;                // centre blocks per SM the overflow tables were sized for
    int64_t* h_total = nullptr;      // pinned host word for the list total
    // profiling: events around each centre-kernel launch of a call
    cudaEvent_t* cev = nullptr;      // [2 * max_cev] or null
    int max_cev = 0;
    int* n_cev = nullptr;            // launches recorded in the current call
};

struct CountShape {
    int64_t cap;        // changed hyperedges per run
    int64_t list_cap;   // N(h) entries per run
    int64_t e_cap;      // hyperedge IDs of the store
    int64_t gs_nh, gs_c;
    int n_cta_nh, n_cta_c;
    int64_t r_cap;      // int32 entries of the restricted-list pool (0: none)
    bool with_ts;       // keep the neighbours' timestamps in the lists (temporal family)
    int c_per_sm;       // centre blocks per SM the overflow tables are sized for (2 or 3)
    bool open_global = true;  // temporal family: global scratch for k_open_h's long lists
};

// pairs.cu: vertex-pair statistics for incident-vertex types 1 and 2
constexpr unsigned long long kPairEmpty = 0;  // no pair key is 0 (u < v)
struct PairTable {
    unsigned long long* kv = nullptr;    // [2 (mask+1)] per slot: key u << 32 | v (u < v; 0 when unused)
                                         // and word m << 40 | S (hyperedges holding the pair, their sizes)
    unsigned long long* used = nullptr;  // device: keys taken
    int64_t* poff = nullptr;             // [n_cap+1] per call: first member pair of each changed hyperedge
    int64_t* tsum = nullptr;             // scan tiles of poff
    uint64_t mask = 0;
    unsigned long long limit = 0;        // keys allowed (the configured capacity)
    int64_t n_cap = 0;                   // changed hyperedges per call
};
// slots for `pairs` keys at a load of at most 0.8
inline uint64_t pair_table_slots(int64_t pairs) {
    uint64_t s = 1024;
    while (s < uint64_t(pairs) + uint64_t(pairs) / 4) s <<= 1;
    return s;
}
size_t pair_table_bytes(int64_t pairs, int64_t n_cap);
cudaError_t pair_table_init(PairTable* P, void* mem, int64_t pairs, int64_t n_cap, cudaStream_t st);
// admission: the batch's inserted pairs must fit the table (status OUT_OF_MEMORY otherwise)
cudaError_t pairs_check(const PairTable& P, const Call& C, cudaStream_t st, LaunchCounter& lc);
// both sides of a batch into the pair statistics and the type 1 / type 2
// terms of each side (run before the store deletes)
cudaError_t pairs_update(const Store& S, const Call& C, const PairTable& P, int sm_count, cudaStream_t st,
                         LaunchCounter& lc);

// debug.cu: the store's invariants (esc_config.debug); acc: 3 * n_graphs words
cudaError_t store_debug_check(const Store& S, Scalars* sc, unsigned long long* acc, int sm_count, cudaStream_t st);

// Largest neighbour-entry count sum(deg) of a changed hyperedge the counter
// accepts with the given shape.
inline int64_t count_max_u(const CountShape& sh) {
    // a neighbourhood takes at most 5 u list entries (list + table)
    return sh.list_cap / 8;
}

// entries of the per-block global scratch of k_open_h (0: none)
inline int64_t open_h_cap(const CountShape& sh) {
    if (!sh.with_ts || !sh.open_global) return 0;
    const int64_t want = std::min<int64_t>(count_max_u(sh), 65536);
    if (want <= 8192) return 0;
    int64_t c = 8192;
    while (c < want) c <<= 1;
    return c;
}

size_t count_scratch_bytes(const CountShape& sh);
cudaError_t count_scratch_init(CountScratch* cs, void* mem, const CountShape& sh, int64_t* pinned_word,
                               cudaStream_t st);
cudaError_t upload_tables(cudaStream_t st);

// Count, for every family of the store, the triads of the current graph that
// hold at least one of the changed hyperedges, attributing each triad to its
// changed member of smallest ID, into dcounts_side[g][...] of each graph g.
// changed[i] / changed_g[i]: global ID and graph of changed hyperedge i
// (changed_g may be null: graph 0); chg_bits marks every changed ID (also
// those outside [lo, hi)).  Only changed[lo, hi) are enumerated by this call.
// side selects the work queues.  The call reads one word back from the
// device (the size of the neighbour lists) and splits [lo, hi) when the lists
// would not fit.  With cs.split_world > 1 only this rank's share of [lo, hi)
// is counted: the contiguous range whose neighbourhood sizes (plus one per
// hyperedge) fall in the rank's equal part of their total, so that the
// shares of all ranks, each counting on an identical replica, sum to the
// whole (every triad is still counted at its changed member of smallest ID).
cudaError_t count_launch(const Store& S, Scalars* sc, const int32_t* changed, const int32_t* changed_g,
                         const uint32_t* chg_bits, int64_t lo, int64_t hi, int side, uint64_t* dcounts_side,
                         const CountScratch& cs, int64_t max_u, cudaStream_t st, LaunchCounter& lc);

// For the fixed sequence, before the store changes: the retry status if the
// inserted side will need more than `runs` count runs.
cudaError_t count_precheck_fixed(const Store& S, const Call& C, const CountScratch& cs, int64_t max_u, int runs,
                                 cudaStream_t st, LaunchCounter& lc);

// The same as a fixed launch sequence (every kernel reads the side's size
// n_side and its run ranges on the device, so the sequence can be captured
// once and replayed): `runs` count runs per side; if the lists need more, the
// call fails with the internal retry status and changes nothing.
cudaError_t count_launch_fixed(const Store& S, Scalars* sc, const int32_t* changed, const int32_t* changed_g,
                               const uint32_t* chg_bits, const int64_t* n_side, int side, uint64_t* dcounts_side,
                               const CountScratch& cs, int64_t max_u, int runs, cudaStream_t st, LaunchCounter& lc);

}  // namespace esc

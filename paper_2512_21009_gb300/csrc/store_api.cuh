// store_api.cuh -- host-side launch entry points of the store and counter
// kernels, called by the C ABI layer (api.cu).
#pragma once

#include "escher_internal.cuh"

namespace esc {

struct LaunchCounter {
    int64_t total = 0;   // kernels launched
    int64_t count = 0;   // triad-count kernels launched
};

// store.cu
cudaError_t store_ingest(const Store& S, const Call& C, const int64_t* b_ins_lo, const int64_t* b_del_lo,
                         int64_t max_u, int sm_count, cudaStream_t st, LaunchCounter& lc);
cudaError_t store_delete(const Store& S, const Call& C, cudaStream_t st, LaunchCounter& lc);
cudaError_t store_insert(const Store& S, const Call& C, int sm_count, cudaStream_t st, LaunchCounter& lc);
cudaError_t store_finish(const Store& S, const Call& C, int sm_count, cudaStream_t st, LaunchCounter& lc);

// count.cu
struct CountScratch {
    int32_t* chunks = nullptr;       // [cap]
    int64_t* item_start = nullptr;   // [cap+1]
    int64_t* block_sums = nullptr;   // scan scratch
    int64_t cap = 0;                 // changed hyperedges per count launch
    int32_t* g_keys = nullptr;       // per-CTA overflow hash tables (2 per CTA)
    uint32_t* g_vals = nullptr;
    int32_t* g_aux = nullptr;
    int32_t* g_list = nullptr;
    int64_t g_slots = 0;             // slots of one overflow table
    int n_cta = 0;                   // persistent grid of the counter
    int64_t smem_slots = 1 << 30;    // cap on shared-memory table sizes (tests lower it)
};

// Largest neighbour-entry count sum(deg) of a changed hyperedge the counter
// accepts with the given overflow table size.
inline int64_t count_max_u(int64_t g_slots) { return g_slots / 2; }

size_t count_scratch_bytes(int64_t cap, int64_t g_slots, int n_cta);
cudaError_t count_scratch_init(CountScratch* cs, void* mem, int64_t cap, int64_t g_slots, int n_cta,
                               cudaStream_t st);
cudaError_t upload_tables(cudaStream_t st);

// Count, for every family of the store, the triads of the current graph that
// hold at least one of the changed hyperedges, attributing each triad to its
// changed member of smallest ID, into dcounts_side[g][...] of each graph g.
// changed[i] / changed_g[i]: global ID and graph of changed hyperedge i;
// chg_bits marks every changed ID (also those outside [lo, hi)).  Only
// changed[lo, hi) are enumerated by this launch.  side selects the work queue.
cudaError_t count_launch(const Store& S, Scalars* sc, const int32_t* changed, const int32_t* changed_g,
                         const uint32_t* chg_bits, int64_t lo, int64_t hi, int side, uint64_t* dcounts_side,
                         const CountScratch& cs, int64_t max_u, cudaStream_t st, LaunchCounter& lc);

}  // namespace esc

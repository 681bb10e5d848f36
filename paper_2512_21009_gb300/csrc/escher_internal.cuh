// escher_internal.cuh -- device-side layout of the incidence store and the
// helpers shared by the store-update and triad-count kernels.
//
// One "store" holds every hypergraph of a group (a single esc_graph is a
// group of one).  Graph g owns the hyperedge IDs [ebase[g], ebase[g]+ecap[g])
// and the vertices [vbase[g], vbase[g]+nv[g]) of the store's global ID
// spaces; batches are translated to global IDs when they are gathered, so the
// store kernels never need to know which graph an element belongs to, and
// triads never span two graphs because no two graphs share a vertex.
//
// h2v (paper Section III-A, memory blocks): each live hyperedge owns one slab
// of the h2v arena holding its members sorted ascending.  v2h: each vertex
// owns one slab of the v2h arena holding the IDs of its hyperedges (in no
// particular order).  Slabs come in power-of-two size classes of 8 << c int32
// slots; freed slabs go to a per-class free stack and are reused before the
// arena's bump tail grows (the paper's reuse of freed blocks, Section III-B).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace esc {

constexpr int kMinSlabLog = 3;           // smallest slab: 8 int32 slots
constexpr int kNumClasses = 28;          // largest slab: 8 << 27 slots
constexpr int kMaxCard = 16384;          // ESC_MAX_CARDINALITY
constexpr int kNH = 30;                  // hyperedge classes
constexpr int kNV = 3;                   // vertex types
constexpr int kNT = 96;                  // temporal classes
constexpr int kOffV = kNH;               // counter layout: [H 30][V 3][T 96]
constexpr int kOffT = kNH + kNV;
constexpr int kNCount = kNH + kNV + kNT; // 129
constexpr int kCStride = 136;            // counters per graph, padded

constexpr uint32_t kFamH = 1u, kFamV = 2u, kFamT = 4u, kFamV12 = 8u;

// status codes, identical to esc_status
constexpr int kOk = 0, kErrInvalid = 1, kErrNotFound = 2, kErrNoMem = 3, kErrUnsupported = 4,
              kErrTimeout = 5, kErrCuda = 6, kErrInternal = 8;
// internal: the neighbour lists of a side needed more count runs than a
// fixed launch sequence holds; nothing changed and the call is run again
// with runs planned on the host (never returned to a caller)
constexpr int kErrRetry = 9;

__host__ __device__ inline int slab_class(int64_t n) {
    int c = 0;
    while ((int64_t(1) << (c + kMinSlabLog)) < n) ++c;
    return c;
}
__host__ __device__ inline int64_t slab_size(int c) { return int64_t(1) << (c + kMinSlabLog); }

struct SlabPool {
    int32_t* arena;       // int32 slots
    int64_t cap;          // slots
    int64_t* tail;        // device scalar: slots handed out by the bump tail
    int32_t* top;         // device [kNumClasses]: free-stack heights
    uint32_t* stack;      // device: all free stacks, entry = slot offset >> kMinSlabLog
    int64_t base[kNumClasses + 1];  // free stack of class c is stack[base[c] .. base[c+1])
};

// device scalars of one call
struct Scalars {
    int32_t status;       // first error of the call (0 = ok)
    int32_t gate;         // status latched at fixed points; kernels that change the store read this
    int32_t ran;          // 1 once the validation kernels have run (their marks need clearing)
    int32_t detail[3];    // where: batch, element, value
    int64_t nnz;          // total inserted members of the call
    int32_t n_touched;    // touched vertices
    int32_t n_big;        // inserted hyperedges sorted by the block sorter
    int32_t n_realloc;    // vertices whose v2h slab moves
    int32_t n_vbig;       // touched vertices whose v2h list is rewritten by a whole block
    int32_t max_u;        // largest neighbour-entry count of a changed hyperedge
    int32_t need_h[kNumClasses];
    int32_t freed_h[kNumClasses];
    int32_t need_v[kNumClasses];
    unsigned long long queue[2];  // centre work queues (deleted side, inserted side)
    unsigned long long qnh[2];    // neighbourhood-build queues
    unsigned long long qoh[2];    // queues of the temporal open-at-h counts (long lists)
    unsigned long long qos[2];    // ... and of the short lists
    int64_t items[2];     // centre work items
    int32_t n_d[2];       // distinct candidate neighbours g1 of one count run
    unsigned long long r_used[2];  // int32 entries of the restricted-list pool taken in this run
    // count runs planned on the device (per side): the changed hyperedges
    // [run_lo, run_lo + run_n) of the side's n_side, their lists starting at
    // neighbour-list position run_base
    int64_t run_lo[2], run_n[2], run_base[2];
    int32_t n_side[2], run_n32[2];
    unsigned long long stats[16]; // v2h, h2v, meta reads, triads, algorithmic entries, then counter work
};

struct Store {
    int32_t n_graphs;
    int64_t nv_total, e_total;
    uint32_t fam;
    int64_t delta;
    // per graph
    const int64_t* vbase;
    const int32_t* nv;
    const int64_t* ebase;   // multiple of 32
    const int64_t* ecap;    // multiple of 32
    int64_t* hw;            // high-water mark, local IDs
    int64_t* n_live;
    uint64_t* counts;       // [G][kCStride]
    uint64_t* dcounts;      // [2][G][kCStride]: deleted side, inserted side
    // hyperedges, global IDs
    int64_t* h_off;
    int32_t* h_card;        // 0 when not live
    int64_t* h_ts;
    uint32_t* live;         // bit per ID
    uint32_t* delb;         // deleted in the current call
    uint32_t* insb;         // inserted in the current call
    // vertices, global IDs
    int64_t* v_off;
    int32_t* v_deg;
    int32_t* v_cap;
    int32_t* v_ndel;        // per-call scratch (kept zero between calls)
    int32_t* v_nins;
    int32_t* v_touch;
    int32_t* v_base;
    int64_t* v_newoff;
    int32_t* v_newcap;
    int32_t* realloc_v;     // vertices whose slab moves this call
    int32_t* vbig;          // touched vertices of degree >= kVBig this call (their v2h lists are long)
    SlabPool hp, vp;
};

// one batch of a call, as handed in (device pointers) plus its place in the
// concatenated call arrays
struct BatchIn {
    int32_t graph;
    int64_t n_ins, n_del;
    const int64_t* off;
    const int32_t* mem;
    const int64_t* ts;
    const int32_t* del;
    const int32_t* pin;      // [n_ins] IDs the inserts keep (a horizontal update), or null: the ID rule
    int64_t ins_lo, del_lo;  // position in the concatenated arrays
};

struct Call {
    int32_t n_batches;
    const BatchIn* batches;  // device [n_batches]
    int64_t* nnz_lo;         // device [n_batches+1]: member offsets of each batch
    int64_t n_ins, n_del;    // totals (host copies, for launch decisions)
    const int64_t* dims;     // device [3]: n_batches, n_ins, n_del (what the kernels read)
    // sizes the launch grids are made for: the call's own, or, for a launch
    // sequence that serves calls of any size (a CUDA graph), the limits
    int64_t grid_batches, grid_ins, grid_del;
    bool fixed;              // launch every kernel even when its part of the call is empty
    bool pinned;             // some batch gives the IDs of its inserts
    int64_t max_nnz;         // staging capacity
    int64_t* ins_off;        // [n_ins+1]
    int32_t* raw;            // [max_nnz] members, global vertex IDs
    int32_t* sorted;         // [max_nnz] sorted, deduplicated members
    int64_t* ts;             // [n_ins]
    int32_t* ins_g;          // [n_ins] graph of each insert
    int32_t* card;           // [n_ins] cardinality after deduplication
    int32_t* ids;            // [n_ins] assigned global IDs
    int32_t* out_local;      // [n_ins] assigned local IDs
    int32_t* slot;           // [max_nnz] place of each inserted member in its v2h append run
    int32_t* big;            // [n_ins] inserts sorted by the block sorter
    int32_t* del;            // [n_del] global IDs
    int32_t* del_g;          // [n_del]
    int32_t* touched;        // [nv_total]
    Scalars* sc;
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool bit_test(const uint32_t* b, int64_t i) {
    return (b[i >> 5] >> (i & 31)) & 1u;
}

__device__ __forceinline__ void set_error(Scalars* sc, int code, int a, int64_t b, int64_t c) {
    if (atomicCAS(&sc->status, 0, code) == 0) {
        sc->detail[0] = a;
        sc->detail[1] = int32_t(b);
        sc->detail[2] = int32_t(c);
    }
}

__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Upper bound in a sorted array: first index with a[idx] > key.
template <typename T>
__device__ __forceinline__ int64_t upper_bound_dev(const T* a, int64_t n, T key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Block-wide exclusive scan of one int per thread (blockDim.x <= 1024).
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int* total, int* warp_tmp) {
    const int lane = lane_id(), w = warp_id();
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = (lane < NT / 32) ? warp_tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) warp_tmp[lane] = s;
    }
    __syncthreads();
    int prefix = (w > 0 ? warp_tmp[w - 1] : 0) + x - v;
    if (total) *total = warp_tmp[NT / 32 - 1];
    __syncthreads();
    return prefix;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// class tables uploaded for the counting kernels, built on the host from the
// definitions (see tables.cu)
struct ClassTables {
    int8_t cls30[128];       // hyperedge class of a pattern, -1 if not a triad
    int8_t cls96[128];       // temporal class of an ordered pattern, -1 if not a triad
    uint8_t perm[6][128];    // pattern after reordering (a,b,c) by permutation q
};
void build_class_tables(ClassTables* t);
// the permutation index of an order (x, y, z) of labels {0,1,2}: new label
// k is old label order[k]
__host__ __device__ inline int perm_index(int o0, int o1) {
    // orders: 012 021 102 120 201 210
    return o0 * 2 + ((o1 == ((o0 == 0) ? 1 : 0)) ? 0 : 1);
}

}  // namespace esc

// count.cu -- incremental triad counting (paper Algorithm 3, steps 2 and 5).
//
// The paper counts the triads of the affected regions before and after the
// update.  Here the same change is computed exactly as
//     new = old - T_old(holding >= 1 deleted) + T_new(holding >= 1 inserted),
// since a triad of unchanged hyperedges keeps its class.  For one set X of
// changed hyperedges, every triad holding a member of X is counted once, at
// its member of X with the smallest ID (the "attribution" rule).
//
// For a changed h with neighbourhood N(h) (hyperedges sharing a vertex with
// h), the connected triples holding h are exactly
//   (i)  {h, g1, g2}, g1 < g2 both in N(h)     -- closed if g1 meets g2,
//                                                 else open with centre h;
//   (ii) {h, g1, f},  g1 in N(h), f in N(g1) outside N(h), f != h
//                                              -- open with centre g1.
// Both are enumerated from the pair (h, g1).  The work is organised by g1
// (centre-major): one block builds N(g1) once, with x = |g1 & f| and the
// size, changed flag (and timestamp) of every f, and then serves the changed
// h that have g1 as a candidate neighbour:
//   1. k_nh_build   per changed h (largest first): N(h) with x_hg and the
//                   smallest shared vertex, written as a list that also
//                   carries |g|, whether g changed and its timestamp; a large
//                   N(h) also as its hash table and a membership filter; the
//                   incident-vertex types 1 and 2; candidate pairs (g1, h)
//                   counted per g1; without the temporal family the open
//                   triads centred at h, in aggregate;
//   2. scans and k_scatter invert the pairs into lists L(g1), ordered by |g1|;
//   3. k_center     per (g1, up to 8 chunks of 32 of L(g1)): N(g1) in shared
//                   memory (or a global table with a shared filter); for
//                   each h, (i) the pairs {g1, g2}: N(h) probing N(g1), or
//                   N(g1) probing N(h)'s filter and table, whichever is
//                   smaller (marking N(h) inside N(g1)); then (ii) the open
//                   triads centred at g1: in aggregate from totals over
//                   N(g1) minus the marked entries, or, with the temporal
//                   family, counted per h by time position and bucket.
// t = |h & g1 & g2| for a closed triple comes from the smallest shared
// vertices: if |h & g1| = 1 it is [that vertex is in g2], and symmetrically;
// otherwise the members of h are tested against g1 and g2.
//
// Venn region sizes follow from |a|, |b|, |c|, the three pairwise
// intersections and t by inclusion-exclusion; the 7-bit pattern is mapped to
// its class by the tables of tables.cu.  The incident-vertex types (Sec. II):
//   type 1 = sum over h of C(|h|, 3)
//   type 2 = sum over hyperedge pairs {h, g} of C(x_hg, 2) (|h| + |g| - 4)
//   type 3 = sum over closed triples {a, b, c} of
//            x_ab x_bc x_ac - t (x_ab + x_bc + x_ac) + 2 t
// (a vertex in each pairwise intersection, all three distinct).
#include <algorithm>
#include <climits>
#include <mutex>
#include <vector>

#include "escher_internal.cuh"
#include "store_api.cuh"

namespace esc {

namespace {

constexpr int32_t EMPTY = -1;
constexpr int kHistT = kNH;          // temporal bins start here in the shared histograms
constexpr int kHistN = kNH + kNT;
constexpr uint32_t kXMask = 0xffffu;

// neighbourhood build
constexpr int NT_NH = 256;
constexpr int NH_S = 4096;           // shared-memory N(h) table slots
// centre kernel: threads NT and shared N(g1) table slots TS are template
// parameters (CenterBig: one 512-thread block per SM; CenterSmall: two
// 256-thread blocks per SM with half the table)
constexpr int LCH = 32;              // changed hyperedges per chunk of a centre work item
constexpr int kSuper = 8;            // chunks of one g1 served by one build of N(g1)
constexpr int kWin = 64;             // |h & g1| values served from the histogram window
constexpr int kIC = 32;              // |h & g1| up to which h & g1 is listed for the triple sizes
constexpr int kHistSmem = 1024;      // |h| up to which the open-at-h histograms live in shared memory

__constant__ ClassTables c_tables;

// MurmurHash3's 32-bit finaliser (Appleby, public domain), used as the slot hash.
__device__ __forceinline__ uint32_t fmix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

// word of key k in the membership filter of a large N(h), and its two bits
// there: a blocked filter of 4 bits per table slot (tcap / 8 words) with both
// of a key's bits in one word, so that a query is one load
__device__ __forceinline__ uint32_t filter_word(int32_t k, uint32_t tcap, uint32_t& bits) {
    const uint32_t x = fmix32(uint32_t(k) ^ 0x27d4eb2fu);
    bits = (1u << (x & 31u)) | (1u << ((x >> 5) & 31u));
    return (x >> 10) & (tcap / 8u - 1u);
}

// bit of key k in a shared-memory filter of N(g1) of w words (w a power of two)
__device__ __forceinline__ uint32_t bloom_bit(int32_t k, int w) {
    return fmix32(uint32_t(k) ^ 0x5bd1e995u) & (uint32_t(w) * 32u - 1u);
}

__device__ __forceinline__ int part_of(int32_t k, int P) {
    return int((fmix32(uint32_t(k) ^ 0x9e3779b9u) >> 8) % uint32_t(P));
}

// Open-addressing table (linear probing).  keys EMPTY / vals 0 / aux INT_MAX
// in unused slots; list[] names the slots taken since the last clear.
struct Tab {
    int32_t* keys;
    uint32_t* vals;
    int32_t* aux;   // may be null
    int32_t* list;
    int* n;
    uint32_t mask;
    int list_cap;
};

__device__ __forceinline__ int tab_insert(const Tab& T, int32_t k, uint32_t inc, int32_t aux_min, Scalars* sc) {
    uint32_t s = fmix32(uint32_t(k)) & T.mask;
    volatile int32_t* vk = T.keys;
    for (uint32_t probe = 0;; ++probe) {
        int32_t cur = vk[s];
        if (cur == k) break;
        if (cur == EMPTY) {
            int32_t old = atomicCAS(&T.keys[s], EMPTY, k);
            if (old == EMPTY) {
                int p = atomicAdd(T.n, 1);
                if (p < T.list_cap) T.list[p] = int32_t(s);
                else set_error(sc, kErrUnsupported, -6, p, T.list_cap);
                break;
            }
            if (old == k) break;
        }
        s = (s + 1) & T.mask;
        if (probe > T.mask) {
            set_error(sc, kErrUnsupported, -7, k, T.mask);
            return -1;
        }
    }
    if (inc) atomicAdd(&T.vals[s], inc);
    if (T.aux) atomicMin(&T.aux[s], aux_min);
    return int(s);
}

// Insert into a table kept in the neighbour-list arena: key in keys[s], and
// x (count) and the smallest shared vertex packed into one 64-bit word xv[s]
// (x in the low half, the vertex in the high half) -- the layout in which a
// large N(h) is handed to k_center, so the table needs no copy.
__device__ __forceinline__ void tab_insert_packed(const Tab& T, uint64_t* xv, int32_t k, int32_t aux_min,
                                                  Scalars* sc) {
    uint32_t s = fmix32(uint32_t(k)) & T.mask;
    volatile int32_t* vk = T.keys;
    for (uint32_t probe = 0;; ++probe) {
        int32_t cur = vk[s];
        if (cur == k) break;
        if (cur == EMPTY) {
            int32_t old = atomicCAS(&T.keys[s], EMPTY, k);
            if (old == EMPTY) {
                int p = atomicAdd(T.n, 1);
                if (p < T.list_cap) T.list[p] = int32_t(s);
                else set_error(sc, kErrUnsupported, -6, p, T.list_cap);
                break;
            }
            if (old == k) break;
        }
        s = (s + 1) & T.mask;
        if (probe > T.mask) {
            set_error(sc, kErrUnsupported, -7, k, T.mask);
            return;
        }
    }
    unsigned int* w = reinterpret_cast<unsigned int*>(xv + s);  // little-endian halves
    atomicAdd(w, 1u);
    atomicMin(w + 1, unsigned(aux_min));
}

__device__ __forceinline__ int tab_find(const Tab& T, int32_t k) {
    uint32_t s = fmix32(uint32_t(k)) & T.mask;
    for (uint32_t probe = 0; probe <= T.mask; ++probe) {
        int32_t cur = T.keys[s];
        if (cur == k) return int(s);
        if (cur == EMPTY) return -1;
        s = (s + 1) & T.mask;
    }
    return -1;
}

template <int NT>
__device__ __forceinline__ void tab_clear(const Tab& T, int n) {
    for (int i = threadIdx.x; i < n; i += NT) {
        int s = T.list[i];
        T.keys[s] = EMPTY;
        T.vals[s] = 0;
        if (T.aux) T.aux[s] = INT_MAX;
    }
}

__device__ __forceinline__ uint32_t pow2_at_least(long long n) {
    uint32_t c = 64;
    while ((long long)c < n) c <<= 1;
    return c;
}

__device__ __forceinline__ bool contains_sorted(const int32_t* a, int n, int32_t v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && a[lo] == v;
}

template <int NT>
__device__ __forceinline__ long long block_sum(long long v, long long* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    long long t = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Members mem[0..n) (n <= NT) of one segment: v2h offset, vertex, and the
// exclusive prefix of their degrees.  Returns the segment's entry count.
template <int NT>
__device__ __forceinline__ int load_segment(const Store& S, const int32_t* mem, int n, int64_t* seg_off,
                                            int32_t* seg_v, int32_t* seg_pre, int* warp_tmp) {
    int d = 0;
    if (int(threadIdx.x) < n) {
        int32_t v = mem[threadIdx.x];
        d = S.v_deg[v];
        seg_off[threadIdx.x] = S.v_off[v];
        if (seg_v) seg_v[threadIdx.x] = v;
    }
    int tot;
    int pre = block_exclusive_scan<NT>(d, &tot, warp_tmp);
    if (int(threadIdx.x) < n) seg_pre[threadIdx.x] = pre;
    if (threadIdx.x == 0) seg_pre[n] = tot;
    __syncthreads();
    return tot;
}

// member of incidence entry e of a loaded segment: largest m with pre[m] <= e
__device__ __forceinline__ int seg_member(const int32_t* pre, int n, int e) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct Accum {
    unsigned long long v1, v2, v3;
    unsigned long long n_v2h, n_h2v, n_meta, n_tri, n_alg;
    unsigned long long w[6];  // items, build entries, pair visits, closed pairs, slow t steps, agg visits
    unsigned long long n_alg_c;  // the part of n_alg counted by the centre kernel
    // algorithmic int32 entries by term: open paths (sum of member degrees
    // of g1 per pair (h, g1)), closed pairs (min(|g1|, |g2|) per closed
    // pair), neighbour build (sum of member degrees of h per changed h) and
    // store (2 |h| + a 4-entry header per changed h)
    unsigned long long n_open, n_closed, n_build, n_store;
};

struct Tables {
    int8_t cls30[128];
    int8_t cls96[128];
    uint8_t perm[6][128];
};

__device__ __forceinline__ void load_tables(Tables& t, int nt) {
    for (int i = threadIdx.x; i < 128; i += nt) {
        t.cls30[i] = c_tables.cls30[i];
        t.cls96[i] = c_tables.cls96[i];
        for (int q = 0; q < 6; ++q) t.perm[q][i] = c_tables.perm[q][i];
    }
}

// Classify the triad (a, b, c) with sizes ka, kb, kc, pairwise intersections
// xab, xbc, xac and triple intersection t into the warp's histogram.
// Class bins of the triad (a, b, c) with sizes ka, kb, kc, pairwise
// intersections xab, xbc, xac and triple intersection t: bh the hyperedge
// class, bt the temporal class (or -1: family not kept, outside the window).
__device__ __forceinline__ void classify_bins(const Tables& tb, uint32_t fam, int64_t delta, int32_t ia, int32_t ib,
                                              int32_t ic, int ka, int kb, int kc, int xab, int xbc, int xac, int t,
                                              int64_t ta, int64_t tbb, int64_t tc, int& bh, int& bt, Accum& acc) {
    int ra = ka - xab - xac + t, rb = kb - xab - xbc + t, rc = kc - xbc - xac + t;
    int m = (ra > 0) | ((rb > 0) << 1) | ((rc > 0) << 2) | ((xab - t > 0) << 3) | ((xbc - t > 0) << 4) |
            ((xac - t > 0) << 5) | ((t > 0) << 6);
    ++acc.n_tri;
    bh = (fam & kFamH) ? tb.cls30[m] : -1;
    bt = -1;
    if (fam & kFamT) {
        // order the labels 0 (a), 1 (b), 2 (c) by (timestamp, ID)
        int64_t T[3] = {ta, tbb, tc};
        int32_t I[3] = {ia, ib, ic};
        int o0 = 0, o1 = 1, o2 = 2, tmp;
#define ESC_BEFORE(x, y) (T[x] < T[y] || (T[x] == T[y] && I[x] < I[y]))
        if (ESC_BEFORE(o1, o0)) { tmp = o0; o0 = o1; o1 = tmp; }
        if (ESC_BEFORE(o2, o1)) { tmp = o1; o1 = o2; o2 = tmp; }
        if (ESC_BEFORE(o1, o0)) { tmp = o0; o0 = o1; o1 = tmp; }
#undef ESC_BEFORE
        if (T[o2] - T[o0] <= delta) bt = tb.cls96[tb.perm[perm_index(o0, o1)][m]];
    }
}

struct CountArgs {
    Store S;
    Scalars* sc;
    const int32_t* changed;
    const int32_t* changed_g;
    const uint32_t* chg;
    int64_t lo, n;
    int side;
    uint64_t* dc;               // [G][kCStride]
    CountScratch cs;
    uint32_t nh_smem_cap, c_smem_cap;
    bool dev;                   // the run's range comes from the device (planned by k_run_plan)
    bool orient;                // closed pairs searched in (|g|, g) order (k_center_o)
};

// The changed hyperedges of one count run, [lo, lo + n) of the side, and the
// neighbour-list position their lists start at.
struct RunRange {
    int64_t lo, n, base;
};

__device__ __forceinline__ RunRange run_of(const CountArgs& A) {
    if (A.dev) return RunRange{A.sc->run_lo[A.side], A.sc->run_n[A.side], A.sc->run_base[A.side]};
    return RunRange{0, A.n, 0};
}

template <int NT>
__device__ void flush(const CountArgs& A, unsigned long long* acc_bins, uint32_t (*hist)[128], int nw, int g,
                      Accum& acc, long long* red) {
    uint64_t* out = A.dc + int64_t(g) * kCStride;
    for (int b = threadIdx.x; b < kHistN; b += NT) {
        unsigned long long v = acc_bins ? acc_bins[b] : 0;
        if (hist)
            for (int w = 0; w < nw; ++w) {
                v += hist[w][b];
                hist[w][b] = 0;
            }
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(b < kNH ? &out[b] : &out[kOffT + (b - kHistT)]), v);
        if (acc_bins) acc_bins[b] = 0;
    }
    long long v1 = block_sum<NT>((long long)acc.v1, red);
    long long v2 = block_sum<NT>((long long)acc.v2, red);
    long long v3 = block_sum<NT>((long long)acc.v3, red);
    if (threadIdx.x == 0) {
        if (v1) atomicAdd(reinterpret_cast<unsigned long long*>(&out[kOffV + 0]), (unsigned long long)v1);
        if (v2) atomicAdd(reinterpret_cast<unsigned long long*>(&out[kOffV + 1]), (unsigned long long)v2);
        if (v3) atomicAdd(reinterpret_cast<unsigned long long*>(&out[kOffV + 2]), (unsigned long long)v3);
    }
    acc.v1 = acc.v2 = acc.v3 = 0;
    __syncthreads();
}

template <int NT>
__device__ void flush_stats(const CountArgs& A, Accum& acc, long long* red) {
    long long r0 = block_sum<NT>((long long)acc.n_v2h, red);
    long long r1 = block_sum<NT>((long long)acc.n_h2v, red);
    long long r2 = block_sum<NT>((long long)acc.n_meta, red);
    long long r3 = block_sum<NT>((long long)acc.n_tri, red);
    long long r4 = block_sum<NT>((long long)acc.n_alg, red);
    long long r5 = block_sum<NT>((long long)acc.n_alg_c, red);
    long long wk[6];
    for (int k = 0; k < 6; ++k) wk[k] = block_sum<NT>((long long)acc.w[k], red);
    const long long r6 = block_sum<NT>((long long)acc.n_open, red);
    const long long r7 = block_sum<NT>((long long)acc.n_closed, red);
    const long long r8 = block_sum<NT>((long long)acc.n_build, red);
    const long long r9 = block_sum<NT>((long long)acc.n_store, red);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k)
            if (wk[k]) atomicAdd(&A.sc->stats[5 + k], (unsigned long long)wk[k]);
        if (r6) atomicAdd(&A.sc->stats[12], (unsigned long long)r6);
        if (r7) atomicAdd(&A.sc->stats[13], (unsigned long long)r7);
        if (r8) atomicAdd(&A.sc->stats[14], (unsigned long long)r8);
        if (r9) atomicAdd(&A.sc->stats[15], (unsigned long long)r9);
        atomicAdd(&A.sc->stats[0], (unsigned long long)r0);
        atomicAdd(&A.sc->stats[1], (unsigned long long)r1);
        atomicAdd(&A.sc->stats[2], (unsigned long long)r2);
        atomicAdd(&A.sc->stats[3], (unsigned long long)r3);
        atomicAdd(&A.sc->stats[4], (unsigned long long)r4);
        if (r5) atomicAdd(&A.sc->stats[11], (unsigned long long)r5);
    }
}

// ---------------------------------------------------------------------------
// 1. sizes and N(h)
// ---------------------------------------------------------------------------

__global__ void k_nh_size(Store S, Scalars* sc, const int32_t* changed, int64_t lo, int64_t n_host,
                          const int32_t* n_dev, int32_t* sizes, int64_t max_u, int64_t big_nh) {
    const int64_t n = n_dev ? *n_dev : n_host;
    const int lane = lane_id();
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n;
         i += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    if (sc->gate) {  // the call failed earlier: the changed list may hold invalid IDs
        if (lane == 0) sizes[i] = 0;
        continue;
    }
    int32_t h = changed[lo + i];
    int k = S.h_card[h];
    const int32_t* m = S.hp.arena + S.h_off[h];
    long long u = 0;
    for (int t = lane; t < k; t += 32) u += S.v_deg[m[t]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (lane == 0) {
        if (u > max_u) {
            set_error(sc, kErrUnsupported, -4, h, u);
            u = 0;
        }
        // list of up to u entries; a large N(h) also gets its hash table
        // (2u rounded up to a power of two slots) and a membership filter of
        // 4 bits per slot (an eighth of the slots, as words)
        const long long t = u > big_nh ? (long long)pow2_at_least(2 * u) : 0;
        sizes[i] = int32_t(u + t + t / 8);
    }
    }
}

// N(h) lists of at most this many entries are sorted by (|g|, g) when the
// oriented centre kernel runs (larger ones are met through their table)
constexpr int kSortMax = 4096;

struct SmemNH {
    unsigned long long skey[kSortMax];  // sort keys |g| << 43 | g << 12 | list index
    int32_t keys[NH_S];
    uint32_t vals[NH_S];
    int32_t aux[NH_S];
    int32_t list[NH_S / 2];
    int64_t seg_off[NT_NH];
    int32_t seg_v[NT_NH];
    int32_t seg_pre[NT_NH + 1];
    int warp_tmp[32];
    long long red[NT_NH / 32];
    long long item;
    long long r_at;
    int n_list;
    unsigned long long acc[128];      // open-at-h class counts of this block
    uint32_t hx[2][kHistSmem + 1];    // x histograms of N'(h), split by [g inside h]
    unsigned long long q3[3];
};

// Class of an open triad {h, g1, g2} centred at h (g1, g2 in N(h), g1 and
// g2 disjoint): regions h-only |h| - x1 - x2, g1-only |g1| - x1, g2-only
// |g2| - x2, h&g1 and h&g2 non-empty, the rest empty.
__device__ __forceinline__ int open_at_h_mask(int kh, int x1, int x2, int k1, int k2) {
    return (kh != x1 + x2 ? 1 : 0) | (k1 != x1 ? 2 : 0) | (k2 != x2 ? 4 : 0) | (1 << 3) | (1 << 5);
}

// Restricted incidence lists of a large N(h): R(u) = {f in N(h) : u in f}
// for every vertex u of h's graph, as a dense index idx[0..nv] and the lists
// ent[idx[u] .. idx[u+1]).  k_center walks R(u) for the members u of a
// candidate g1 instead of all of N(g1): N(g1) and N(h) then meet in
// sum over u in g1 of |R(u)| steps rather than sum of member degrees.
// Entries are counted per vertex, prefix-summed (idx[u] = end of R(u)) and
// scattered downwards (idx[u] ends at the start of R(u)).
__device__ void build_rlist(const CountArgs& A, SmemNH& s, int64_t i, int g, int64_t base, int nn) {
    const Store& S = A.S;
    const CountScratch& cs = A.cs;
    const int tid = threadIdx.x, lane = lane_id(), wid = warp_id();
    constexpr int NW = NT_NH / 32;
    __syncthreads();
    long long eh = 0;
    for (int q = tid; q < nn; q += NT_NH) eh += S.h_card[cs.nh_g[base + q]];
    eh = block_sum<NT_NH>(eh, s.red);
    const int64_t nvg = S.nv[g];
    if (tid == 0) {
        s.r_at = -1;
        const unsigned long long need = (unsigned long long)((nvg + 1 + eh + 3) & ~3ll);
        if (nvg <= 4 * eh) {
            const unsigned long long at = atomicAdd(&A.sc->r_used[A.side], need);
            if (at + need <= (unsigned long long)cs.r_cap) s.r_at = (long long)at;
        }
        cs.r_off[i] = s.r_at;
    }
    __syncthreads();
    const long long at = s.r_at;
    if (at < 0) return;
    int32_t* idx = cs.r_pool + at;
    int32_t* ent = idx + nvg + 1;
    const int64_t vb = S.vbase[g];
    const int32_t* h2v = S.hp.arena;
    for (int64_t t = tid; t < nvg; t += NT_NH) idx[t] = 0;
    if (tid == 0) idx[nvg] = int32_t(eh);
    __syncthreads();
    for (int q = wid; q < nn; q += NW) {
        const int32_t f = cs.nh_g[base + q];
        const int32_t* fm = h2v + S.h_off[f];
        const int kf = S.h_card[f];
        for (int m = lane; m < kf; m += 32) atomicAdd(&idx[fm[m] - vb], 1);
    }
    __syncthreads();
    // inclusive prefix over idx[0..nvg), in tiles of 4 entries per thread
    int carry = 0;
    for (int64_t t0 = 0; t0 < nvg; t0 += NT_NH * 4) {
        int v[4], loc = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t j = t0 + tid * 4 + k;
            v[k] = j < nvg ? idx[j] : 0;
            loc += v[k];
        }
        int tot;
        int pre = block_exclusive_scan<NT_NH>(loc, &tot, s.warp_tmp) + carry;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t j = t0 + tid * 4 + k;
            pre += v[k];
            if (j < nvg) idx[j] = pre;
        }
        carry += tot;
    }
    __syncthreads();
    for (int q = wid; q < nn; q += NW) {
        const int32_t f = cs.nh_g[base + q];
        const int32_t* fm = h2v + S.h_off[f];
        const int kf = S.h_card[f];
        for (int m = lane; m < kf; m += 32) ent[atomicSub(&idx[fm[m] - vb], 1) - 1] = f;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NT_NH) k_nh_build(CountArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemNH& s = *reinterpret_cast<SmemNH*>(smem_raw);
    const Store& S = A.S;
    if (A.sc->gate) return;
    const int tid = threadIdx.x;
    const uint32_t fam = S.fam;
    const CountScratch& cs = A.cs;
    for (int i = tid; i < NH_S; i += NT_NH) {
        s.keys[i] = EMPTY;
        s.vals[i] = 0;
        s.aux[i] = INT_MAX;
    }
    for (int i = tid; i < 128; i += NT_NH) s.acc[i] = 0;
    for (int i = tid; i < 2 * (kHistSmem + 1); i += NT_NH) s.hx[i / (kHistSmem + 1)][i % (kHistSmem + 1)] = 0;
    if (tid == 0) s.n_list = 0;
    // open-at-h triads are counted in aggregate (static classes); with the
    // temporal family only for the oriented centre kernel (k_open_h counts
    // their temporal classes), the earlier one classifies each of them
    const bool agg = (fam & kFamH) && (!(fam & kFamT) || A.orient);
    // without the temporal family k_center may meet N(g1) and a large N(h)
    // through restricted lists
    const bool use_r = !(fam & kFamT) && cs.r_cap > 0;
    const RunRange R = run_of(A);
    uint32_t* ghx = cs.onh_hist + int64_t(blockIdx.x) * 2 * (kMaxCard + 1);
    __syncthreads();
    const int64_t gs = cs.gs_nh;
    Tab gNH{cs.onh_keys + blockIdx.x * gs, cs.onh_vals + blockIdx.x * gs, cs.onh_aux + blockIdx.x * gs,
            cs.onh_list + blockIdx.x * (gs / 2), &s.n_list, uint32_t(gs - 1), int(gs / 2)};
    Accum acc = {0, 0, 0, 0, 0, 0, 0, 0, {0, 0, 0, 0, 0, 0}, 0, 0, 0, 0, 0};
    int cur_g = -1;
    const int32_t* v2h = S.vp.arena;
    for (;;) {
        __syncthreads();
        if (tid == 0) s.item = (long long)atomicAdd(&A.sc->qnh[A.side], 1ull);
        __syncthreads();
        if (s.item >= R.n) break;
        const int64_t i = cs.order[s.item];  // index in the side
        const int32_t h = A.changed[A.lo + i];
        const int g = A.changed_g ? A.changed_g[A.lo + i] : 0;
        if (g != cur_g) {
            if (cur_g >= 0) flush<NT_NH>(A, s.acc, nullptr, 0, cur_g, acc, s.red);
            cur_g = g;
        }
        const int kh = S.h_card[h];
        const int32_t* hmem = S.hp.arena + S.h_off[h];
        long long uh = 0;
        for (int t = tid; t < kh; t += NT_NH) uh += S.v_deg[hmem[t]];
        uh = block_sum<NT_NH>(uh, s.red);
        Tab NH;
        const uint32_t cap = pow2_at_least(2 * uh);
        const int64_t base = cs.nh_off[i] - R.base;
        // a neighbourhood too large for the block's tables is built in place,
        // in the table part of its own list region (see k_nh_size)
        const bool huge = cap > A.nh_smem_cap && (int64_t)cap > gs;
        const bool big = uh > cs.big_nh;
        // the list region k_nh_size reserved must hold what is written below
        // (it reserves nothing for a hyperedge over the size limit, which it
        // reports); a hyperedge that does not fit is skipped, never written
        if (uh + ((big || huge) ? (long long)cap + cap / 8 : 0) > cs.nh_off[i + 1] - cs.nh_off[i]) {
            if (tid == 0) {
                set_error(A.sc, kErrUnsupported, -12, h, uh);
                cs.nh_n[i] = 0;
                cs.nh_toff[i] = 0;
                cs.nh_tcap[i] = 0;
                cs.nh_flag[i] = 0;
                cs.r_off[i] = -1;
            }
            continue;
        }
        uint64_t* const xv_t = cs.nh_xv + base + uh;
        if (cap <= A.nh_smem_cap) {
            NH = Tab{s.keys, s.vals, s.aux, s.list, &s.n_list, cap - 1, NH_S / 2};
        } else if (!huge) {
            NH = gNH;
            NH.mask = cap - 1;
        } else {
            NH = Tab{cs.nh_g + base + uh, nullptr, nullptr, cs.nh_g + base, &s.n_list, cap - 1, int(uh)};
            for (uint32_t t = tid; t < cap; t += NT_NH) {
                NH.keys[t] = EMPTY;
                xv_t[t] = uint64_t(uint32_t(INT_MAX)) << 32;
            }
            __syncthreads();
        }
        uint32_t* const filt = reinterpret_cast<uint32_t*>(cs.nh_g + base + uh + cap);
        if (big)
            for (uint32_t t = tid; t < cap / 8; t += NT_NH) filt[t] = 0;
        acc.n_h2v += (tid < kh) ? (kh - tid + NT_NH - 1) / NT_NH : 0;
        if (tid == 0) {
            acc.n_alg += (unsigned long long)(uh + kh);
            acc.n_build += (unsigned long long)uh;
            acc.n_store += 2ull * (unsigned long long)kh + 4ull;
        }
        for (int m0 = 0; m0 < kh; m0 += NT_NH) {
            const int n = min(NT_NH, kh - m0);
            const int tot = load_segment<NT_NH>(S, hmem + m0, n, s.seg_off, s.seg_v, s.seg_pre, s.warp_tmp);
            for (int e = tid; e < tot; e += NT_NH) {
                const int m = seg_member(s.seg_pre, n, e);
                const int32_t f = v2h[s.seg_off[m] + (e - s.seg_pre[m])];
                if (f == h) continue;
                if (huge) tab_insert_packed(NH, xv_t, f, s.seg_v[m], A.sc);
                else tab_insert(NH, f, 1u, s.seg_v[m], A.sc);
            }
            acc.n_v2h += (tid < tot) ? (tot - tid + NT_NH - 1) / NT_NH : 0;
            __syncthreads();
        }
        // distinct neighbours never outnumber the region reserved for them
        // (sum of member degrees); the clamp only matters after an error
        const int nn = int(min((long long)min(s.n_list, NH.list_cap), uh));
        // for the oriented centre kernel the list goes out sorted by (|g|, g),
        // so that the neighbours of h above a given g1 are a suffix of it
        const bool sorted = A.orient && !huge && nn <= kSortMax;
        if (sorted) {
            int n2 = 2;
            while (n2 < nn) n2 <<= 1;
            for (int q = tid; q < n2; q += NT_NH) {
                unsigned long long key = ~0ull;
                if (q < nn) {
                    const int32_t gg = NH.keys[NH.list[q]];
                    key = (uint64_t(S.h_card[gg]) << 43) | (uint64_t(uint32_t(gg)) << 12) | uint64_t(q);
                }
                s.skey[q] = key;
            }
            __syncthreads();
            // bitonic sort of skey[0, n2)
            for (int k = 2; k <= n2; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int t = tid; t < (n2 >> 1); t += NT_NH) {
                        const int a = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                        const unsigned long long x0 = s.skey[a], x1 = s.skey[a + j];
                        if ((x0 > x1) == ((a & k) == 0)) {
                            s.skey[a] = x1;
                            s.skey[a + j] = x0;
                        }
                    }
                    __syncthreads();
                }
        }
        for (int p = tid; p < nn; p += NT_NH) {
            // in place, the list of taken slots is the list region itself:
            // each entry is read and then overwritten by the same thread
            const int q = sorted ? int(s.skey[p] & 0xfffu) : p;
            const int sl = NH.list[q];
            const int32_t gg = NH.keys[sl];
            const uint64_t xvt = huge ? xv_t[sl] : uint64_t(NH.vals[sl]) | (uint64_t(uint32_t(NH.aux[sl])) << 32);
            const uint32_t x = uint32_t(xvt) & kXMask;
            const int kg = sorted ? int(s.skey[p] >> 43) : S.h_card[gg];
            const bool chg_g = bit_test(A.chg, gg);
            // the list entry also carries |g| and whether g changed, read
            // in order by k_center instead of gathered per visit
            cs.nh_g[base + p] = gg;
            cs.nh_xv[base + p] = (xvt & 0xffffffff00000000ull) | x | (uint64_t(kg) << 16) | (chg_g ? 1ull << 31 : 0ull);
            if (cs.nh_ts) cs.nh_ts[base + p] = S.h_ts[gg];
            if (big) {
                uint32_t bits;
                const uint32_t w = filter_word(gg, cap, bits);
                atomicOr(&filt[w], bits);
            }
            if (gg < h && chg_g) continue;  // pair attributed elsewhere
            if (atomicAdd(&cs.lcnt[gg], 1) == 0) cs.d_list[atomicAdd(&A.sc->n_d[A.side], 1)] = gg;
            if ((fam & kFamV) && x >= 2)
                acc.v2 += (unsigned long long)(x * (x - 1) / 2) * (unsigned long long)(kh + kg - 4);
        }
        // a large N(h) also goes out as its hash table, probed by k_center
        if (big && !huge) {
            const int64_t toff = base + uh;
            for (uint32_t t = tid; t <= NH.mask; t += NT_NH) {
                const int32_t key = NH.keys[t];
                cs.nh_g[toff + t] = key;
                if (key != EMPTY)
                    cs.nh_xv[toff + t] = uint64_t(NH.vals[t]) | (uint64_t(uint32_t(NH.aux[t])) << 32);
            }
        }
        if (tid == 0) {
            cs.nh_n[i] = nn;
            cs.nh_flag[i] = sorted ? 1 : 0;
            cs.nh_toff[i] = big ? base + uh : 0;
            cs.nh_tcap[i] = big ? int32_t(NH.mask + 1) : 0;
            if ((fam & kFamV) && kh >= 3) acc.v1 += (unsigned long long)kh * (kh - 1) * (kh - 2) / 6;
        }
        if (use_r && big && uh >= cs.r_min) build_rlist(A, s, i, g, base, nn);
        else if (tid == 0) cs.r_off[i] = -1;
        // entry q of N(h): from the block's table, or from the list just
        // written when the table was built in place
        if (huge) __syncthreads();
        auto entry = [&](int q, int32_t& gg, int& x) {
            if (huge) {
                gg = cs.nh_g[base + q];
                x = int(uint32_t(cs.nh_xv[base + q]) & kXMask);
            } else {
                const int sl = NH.list[q];
                gg = NH.keys[sl];
                x = int(NH.vals[sl]);
            }
        };
        if (agg) {
            // open triads centred at h, in aggregate over the pairs of N'(h)
            // (N(h) without the neighbours attributed elsewhere): the class is
            // set by E = [x1 + x2 = |h|] and by which of g1, g2 lie inside h.
            // Closed pairs are counted here too and taken back by k_center.
            uint32_t* H = kh <= kHistSmem ? &s.hx[0][0] : ghx;
            const int hstride = kh <= kHistSmem ? kHistSmem + 1 : kMaxCard + 1;
            unsigned long long n1w = 0, n0w = 0;
            for (int q = tid; q < nn; q += NT_NH) {
                int32_t gg;
                int x;
                entry(q, gg, x);
                if (gg < h && bit_test(A.chg, gg)) continue;
                const int in = S.h_card[gg] == x ? 1 : 0;
                atomicAdd(&H[in * hstride + x], 1u);
                if (in) ++n1w; else ++n0w;
            }
            const long long n1 = block_sum<NT_NH>((long long)n1w, s.red);
            const long long n0 = block_sum<NT_NH>((long long)n0w, s.red);
            unsigned long long q00 = 0, q11 = 0, q01 = 0;
            for (int x = 1 + tid; x < kh; x += NT_NH) {
                const unsigned long long a0 = H[x], a1 = H[hstride + x];
                const unsigned long long b0 = H[kh - x], b1 = H[hstride + kh - x];
                q00 += a0 * b0;
                q11 += a1 * b1;
                q01 += a0 * b1;
            }
            q00 = (unsigned long long)block_sum<NT_NH>((long long)q00, s.red);
            q11 = (unsigned long long)block_sum<NT_NH>((long long)q11, s.red);
            q01 = (unsigned long long)block_sum<NT_NH>((long long)q01, s.red);
            if (tid == 0) {
                if ((kh & 1) == 0) {  // ordered pairs (g, g) with x = |h|/2
                    q00 -= H[kh / 2];
                    q11 -= H[hstride + kh / 2];
                }
                q00 /= 2;
                q11 /= 2;
                const unsigned long long p00 = (unsigned long long)n0 * (n0 - 1) / 2;
                const unsigned long long p11 = (unsigned long long)n1 * (n1 - 1) / 2;
                const unsigned long long p01 = (unsigned long long)n0 * n1;
                // mask with E, s1 = [g1 inside h], s2 = [g2 inside h]
                auto add = [&](int E, int s1, int s2, unsigned long long c) {
                    if (!c) return;
                    const int m = (E ? 0 : 1) | (s1 ? 0 : 2) | (s2 ? 0 : 4) | (1 << 3) | (1 << 5);
                    s.acc[c_tables.cls30[m]] += c;
                    acc.n_tri += c;
                };
                add(1, 0, 0, q00);
                add(0, 0, 0, p00 - q00);
                add(1, 1, 1, q11);
                add(0, 1, 1, p11 - q11);
                add(1, 0, 1, q01);
                add(0, 0, 1, p01 - q01);
            }
            __syncthreads();
            for (int q = tid; q < nn; q += NT_NH) {
                int32_t gg;
                int x;
                entry(q, gg, x);
                H[x] = 0;
                H[hstride + x] = 0;
            }
        }
        __syncthreads();
        if (!huge) tab_clear<NT_NH>(NH, nn);
        __syncthreads();
        if (tid == 0) s.n_list = 0;
    }
    __syncthreads();
    if (cur_g >= 0) flush<NT_NH>(A, s.acc, nullptr, 0, cur_g, acc, s.red);
    flush_stats<NT_NH>(A, acc, s.red);
}

// ---------------------------------------------------------------------------
// 2. invert candidate pairs into L(g1)
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// processing order: the persistent blocks take the longest work first, so
// that no block starts a large neighbourhood when the others run dry
// ---------------------------------------------------------------------------

constexpr int32_t kBigFirst = 4096;  // neighbour-region entries from which h goes first
constexpr int kOrderBuckets = 16;    // log2 buckets of |g1| for the centre items

__global__ void k_order_flags(CountArgs A) {
    const RunRange R = run_of(A);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < R.n; i += int64_t(gridDim.x) * blockDim.x)
        A.cs.oflag[i] = A.cs.sizes[R.lo + i] >= kBigFirst ? 1 : 0;
}

// stable partition of the run: the flagged hyperedges in order, then the
// others in order (as indices in the side)
__global__ void k_order_place(CountArgs A) {
    const RunRange R = run_of(A);
    const int32_t* flag = A.cs.oflag;
    const int64_t* pre = A.cs.opre;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < R.n; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t nb = pre[R.n];
        A.cs.order[flag[i] ? pre[i] : nb + (i - pre[i])] = int32_t(R.lo + i);
    }
}

__device__ __forceinline__ int g1_bucket(int k1) { return min(kOrderBuckets - 1, 31 - __clz(max(k1, 1))); }

// distinct candidate neighbours g1 by descending log2 |g1| (the cost of an
// item grows with the neighbourhood of g1 built for it)
__global__ void k_dsort_count(CountArgs A) {
    const CountScratch& cs = A.cs;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(cs.block_sums);
    const int nd = A.sc->n_d[A.side];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x)
        atomicAdd(&cnt[g1_bucket(A.S.h_card[cs.d_list[j]])], 1ull);
}

__global__ void k_dsort_scan(CountArgs A) {
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(A.cs.block_sums);
    if (threadIdx.x != 0) return;
    unsigned long long pos = 0;
    for (int b = kOrderBuckets - 1; b >= 0; --b) {
        const unsigned long long c = cnt[b];
        cnt[b] = pos;
        pos += c;
    }
}

__global__ void k_dsort_scatter(CountArgs A) {
    const CountScratch& cs = A.cs;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(cs.block_sums);
    const int nd = A.sc->n_d[A.side];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x) {
        const int32_t g1 = cs.d_list[j];
        cs.d_items[atomicAdd(&cnt[g1_bucket(A.S.h_card[g1])], 1ull)] = g1;
    }
}

__global__ void k_dsort_copy(CountArgs A) {
    const CountScratch& cs = A.cs;
    const int nd = A.sc->n_d[A.side];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x)
        cs.d_list[j] = cs.d_items[j];
}

__global__ void k_d_prep(CountArgs A) {
    const CountScratch& cs = A.cs;
    const int nd = A.sc->n_d[A.side];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x) {
        const int c = cs.lcnt[cs.d_list[j]];
        cs.d_cnt[j] = c;
        cs.d_items[j] = ((c + LCH - 1) / LCH + kSuper - 1) / kSuper;
    }
}

__global__ void k_set_loffg(CountArgs A) {
    const CountScratch& cs = A.cs;
    const int nd = A.sc->n_d[A.side];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x)
        cs.loffg[cs.d_list[j]] = cs.d_loff[j];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t items = cs.d_item_start[nd];
        // the item map holds every item (a bound the arena sizes guarantee)
        if (items > cs.items_cap) set_error(A.sc, kErrUnsupported, -13, items, cs.items_cap);
        A.sc->items[A.side] = (A.sc->gate || items > cs.items_cap) ? 0 : items;
        A.sc->queue[A.side] = 0;
    }
}

// Per distinct g1 (a warp each): |g1|, the sum of its members' degrees (the
// entries of N(g1) with repeats) and its h2v offset, read once here instead
// of at the start of every centre item; and the index j of every item of g1.
__global__ void k_item_prep(CountArgs A) {
    const CountScratch& cs = A.cs;
    const Store& S = A.S;
    if (A.sc->gate) return;
    const int nd = A.sc->n_d[A.side];
    const int lane = lane_id();
    for (int64_t j = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; j < nd;
         j += (int64_t(gridDim.x) * blockDim.x) >> 5) {
        const int32_t g1 = cs.d_list[j];
        const int k1 = S.h_card[g1];
        const int64_t off = S.h_off[g1];
        long long u = 0;
        for (int t = lane; t < k1; t += 32) u += S.v_deg[S.hp.arena[off + t]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (lane == 0) {
            cs.d_k1[j] = k1;
            cs.d_u1[j] = u;
            cs.d_hoff[j] = off;
        }
        const int64_t i0 = cs.d_item_start[j], i1 = cs.d_item_start[j + 1];
        for (int64_t it = i0 + lane; it < i1 && it < cs.items_cap; it += 32) cs.item_j[it] = int32_t(j);
    }
}

__global__ void k_scatter(CountArgs A) {
    const CountScratch& cs = A.cs;
    const int lane = lane_id();
    if (A.sc->gate) return;
    const RunRange R = run_of(A);
    for (int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < R.n;
         w += (int64_t(gridDim.x) * blockDim.x) >> 5) {
        const int64_t i = R.lo + w;  // index in the side
        const int32_t h = A.changed[A.lo + i];
        const int64_t base = cs.nh_off[i] - R.base;
        const int nn = cs.nh_n[i];
        for (int q = lane; q < nn; q += 32) {
            const int32_t gg = cs.nh_g[base + q];
            if (gg < h && bit_test(A.chg, gg)) continue;
            const int64_t pos = cs.loffg[gg] + atomicAdd(&cs.lfill[gg], 1);
            cs.l_i[pos] = int32_t(i);
            cs.l_xv[pos] = cs.nh_xv[base + q];
            cs.l_q[pos] = q;
        }
    }
}

__global__ void k_d_clean(CountArgs A) {
    const CountScratch& cs = A.cs;
    const int nd = A.sc->n_d[A.side];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x) {
        const int32_t g = cs.d_list[j];
        cs.lcnt[g] = 0;
        cs.lfill[g] = 0;
    }
}

// ---------------------------------------------------------------------------
// 3. centre kernel
// ---------------------------------------------------------------------------

template <int NT_C, int T1_S>
struct SmemC {
    static constexpr int NW_C = NT_C / 32;
    Tables tb;
    uint32_t hist[NW_C][128];
    uint32_t hneg[NW_C][32];   // open-at-h classes taken back for closed pairs
    unsigned long long acc[128];
    int32_t keys[T1_S];
    uint32_t vals[T1_S];
    uint32_t mark[T1_S];       // bit l: the entry is in N(h) of the item's l-th h
    int32_t list[T1_S / 2];
    int32_t lk[T1_S / 2];      // size of f, bit 31: f is changed
    int64_t lts[T1_S / 2];     // timestamp of f; in aggregate mode the changed f as (slot, size)
    int64_t seg_off[NT_C];
    int32_t seg_pre[NT_C + 1];
    int warp_tmp[32];
    long long red[NW_C];
    long long item;
    int n_list;
    // aggregated open-at-centre counts (no temporal family): over the f of
    // N(g1), totals by C = [f not inside g1] and a window of x = |g1 & f|
    // values near |g1|
    uint32_t tot[2];
    uint32_t win[kWin][2];
    int n_cl;
    // the changed hyperedges h of the item
    int32_t hh[LCH], hk[LCH], hx[LCH], hvf[LCH], hli[LCH], hnn[LCH], htcap[LCH];
    int64_t hts[LCH], hnb[LCH], htoff[LCH];
    const int32_t* hmem[LCH];
    int32_t hfrom[LCH];        // 0: visit N(h); 1: visit N(g1) probing N(h)'s table; 2: restricted lists
    int64_t hr[LCH];           // start of h's restricted lists in the pool, -1: none
    int32_t hpre[LCH + 1];     // prefix of the per-h work of pass (i)
    uint32_t sub[LCH][4];
    uint32_t xc[LCH][2];
    int32_t hI[LCH][kIC];      // h & g1 when 2 <= |h & g1| <= kIC
    int hIn[LCH];
    // one-hash filter of an N(g1) whose table is in global memory (words; a
    // power of two, smaller where the block's own table is larger)
    static constexpr int BLOOM_W = T1_S >= 4096 ? 2048 : 4096;
    uint32_t bloom[BLOOM_W];
};

// three blocks of the default centre shape fit one SM's shared memory
// (233,472 bytes, 1,024 of them reserved per block) and leave the rest to L1,
// which the gathers of the pair pass use: four blocks (with |h & g1| listed
// up to 16) were 8% slower on the 1M-vertex workload
static_assert(sizeof(SmemC<256, 2048>) + 1024 <= 233472 / 3, "three 256-thread centre blocks per SM");

// t = |h & g1 & g2| from the smallest shared vertices (see the file comment);
// when both |h & g1| and |h & g2| exceed 1, the listed h & g1 (hI, nI
// entries) is tested against g2, else every member of h.
__device__ __forceinline__ int triple_size(int xh1, int32_t vf1, int xh2, int32_t vf2, const int32_t* g1mem,
                                           int k1, const int32_t* g2mem, int k2, const int32_t* hmem, int kh,
                                           const int32_t* hI, int nI, unsigned long long& slow) {
    if (xh1 == 1 && xh2 == 1) return vf1 == vf2;
    if (xh1 == 1) return contains_sorted(g2mem, k2, vf1);
    if (xh2 == 1) return contains_sorted(g1mem, k1, vf2);
    int t = 0;
    if (nI == xh1) {
        slow += nI;
        for (int q = 0; q < nI; ++q) t += contains_sorted(g2mem, k2, hI[q]) ? 1 : 0;
        return t;
    }
    slow += kh;
    const int32_t lo = vf1 > vf2 ? vf1 : vf2;
    for (int q = 0; q < kh; ++q) {
        const int32_t u = hmem[q];
        if (u < lo) continue;
        if (contains_sorted(g1mem, k1, u) && contains_sorted(g2mem, k2, u)) ++t;
    }
    return t;
}

// slot of key k in a table stored in the neighbour lists (a large N(h)), or -1
__device__ __forceinline__ int probe_list_table(const int32_t* keys, uint32_t mask, int32_t k) {
    uint32_t ps = fmix32(uint32_t(k)) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t key = keys[ps];
        if (key == k) return int(ps);
        if (key == EMPTY) return -1;
        ps = (ps + 1) & mask;
    }
    return -1;
}

// add 1 to counter[key] for every lane holding key >= 0, one atomic per distinct key
__device__ __forceinline__ void warp_count(uint32_t* counter, int key) {
    const unsigned same = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && lane_id() == __ffs(same) - 1) atomicAdd(&counter[key], __popc(same));
}

template <int NT_C, int T1_S, int MINB>
__global__ void __launch_bounds__(NT_C, MINB) k_center(CountArgs A) {
    constexpr int NW_C = NT_C / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemC<NT_C, T1_S>& s = *reinterpret_cast<SmemC<NT_C, T1_S>*>(smem_raw);
    const Store& S = A.S;
    if (A.sc->gate) return;
    const int tid = threadIdx.x;
    const int lane = lane_id();
    const int wid = warp_id();
    const uint32_t fam = S.fam;
    const int64_t delta = S.delta;
    const bool want_open = (fam & (kFamH | kFamT)) != 0;
    const bool want_t = (fam & kFamT) != 0;
    // without the temporal family, open triads are counted in aggregate: those
    // centred at h by k_nh_build, those centred at g1 here from totals
    const bool agg = want_open && !want_t;
    const CountScratch& cs = A.cs;
    const RunRange R = run_of(A);
    const int32_t* v2h = S.vp.arena;
    const int32_t* h2v = S.hp.arena;
    load_tables(s.tb, NT_C);
    for (int i = tid; i < 128; i += NT_C) {
        s.acc[i] = 0;
        for (int w = 0; w < NW_C; ++w) s.hist[w][i] = 0;
    }
    for (int i = tid; i < NW_C * 32; i += NT_C) s.hneg[i / 32][i % 32] = 0;
    for (int i = tid; i < T1_S; i += NT_C) {
        s.keys[i] = EMPTY;
        s.vals[i] = 0;
        s.mark[i] = 0;
    }
    for (int i = tid; i < LCH * 4; i += NT_C) s.sub[i >> 2][i & 3] = 0;
    for (int i = tid; i < LCH * 2; i += NT_C) s.xc[i >> 1][i & 1] = 0;
    if (tid < 2) s.tot[tid] = 0;
    for (int i = tid; i < kWin * 2; i += NT_C) s.win[i >> 1][i & 1] = 0;
    if (tid == 0) {
        s.n_list = 0;
        s.n_cl = 0;
    }
    __syncthreads();
    const int64_t gs = cs.gs_c;
    int32_t* g_keys = cs.oc_keys + blockIdx.x * gs;
    uint32_t* g_vals = cs.oc_vals + blockIdx.x * gs;
    uint32_t* g_mark = cs.oc_mark + blockIdx.x * gs;
    int32_t* g_list = cs.oc_list + blockIdx.x * (gs / 2);
    int32_t* g_lk = cs.oc_lk + blockIdx.x * (gs / 2);
    int64_t* g_lts = cs.oc_lts + blockIdx.x * (gs / 2);
    int32_t* g_lkey = cs.oc_lkey + blockIdx.x * (gs / 2);
    uint32_t* hist = s.hist[wid];
    Accum acc = {0, 0, 0, 0, 0, 0, 0, 0, {0, 0, 0, 0, 0, 0}, 0, 0, 0, 0, 0};
    const int64_t n_items = A.sc->items[A.side];
    const int nd = A.sc->n_d[A.side];
    int cur_g = -1;

    for (;;) {
        __syncthreads();
        if (tid == 0) s.item = (long long)atomicAdd(&A.sc->queue[A.side], 1ull);
        __syncthreads();
        const int64_t item = s.item;
        if (item >= n_items) break;
        const int64_t j = upper_bound_dev(cs.d_item_start, int64_t(nd) + 1, item) - 1;
        // this item: chunks [c_beg, c_end) of L(g1), LCH changed hyperedges
        // each, all served by one build of N(g1)
        const int64_t sup = item - cs.d_item_start[j];
        const int32_t g1 = cs.d_list[j];
        const int64_t l_lo = cs.d_loff[j], l_hi = cs.d_loff[j + 1];
        const int64_t n_chunks = (l_hi - l_lo + LCH - 1) / LCH;
        const int64_t c_beg = sup * kSuper, c_end = min(c_beg + kSuper, n_chunks);
        const int64_t nh_all = min(l_lo + c_end * LCH, l_hi) - (l_lo + c_beg * LCH);
        const int g = A.changed_g ? A.changed_g[A.lo + cs.l_i[l_lo + c_beg * LCH]] : 0;
        if (g != cur_g) {
            if (cur_g >= 0) flush<NT_C>(A, s.acc, s.hist, NW_C, cur_g, acc, s.red);
            cur_g = g;
        }
        const int k1 = S.h_card[g1];
        const int32_t* g1mem = h2v + S.h_off[g1];
        const int64_t ts1 = S.h_ts[g1];
        // size of N(g1) with repeats, to choose the table
        long long u1 = 0;
        for (int t = tid; t < k1; t += NT_C) u1 += S.v_deg[g1mem[t]];
        u1 = block_sum<NT_C>(u1, s.red);
        acc.n_h2v += (tid < k1) ? (k1 - tid + NT_C - 1) / NT_C : 0;
        // the method reads N(g1) (sum of member degrees) once per pair (h, g1)
        if (tid == 0) {
            acc.n_alg += (unsigned long long)(u1 + k1) * (unsigned long long)nh_all;
            acc.n_alg_c += (unsigned long long)(u1 + k1) * (unsigned long long)nh_all;
            acc.n_open += (unsigned long long)u1 * (unsigned long long)nh_all;
            ++acc.w[0];
            acc.w[1] += (unsigned long long)u1;
        }
        Tab T1;
        uint32_t* mark;
        int32_t* lk;
        int64_t* lts;
        // an N(g1) too large for the block's shared table lives in global
        // memory; then its keys are also kept in list order (lkey) and a
        // shared-memory filter answers most "is g2 in N(g1)" questions
        bool gbl = false;
        int P = 1;
        const uint32_t t1_cap = pow2_at_least(2 * u1);
        if (t1_cap <= min(A.c_smem_cap, uint32_t(T1_S))) {  // the block's table holds T1_S slots
            T1 = Tab{s.keys, s.vals, nullptr, s.list, &s.n_list, t1_cap - 1, T1_S / 2};
            mark = s.mark;
            lk = s.lk;
            lts = s.lts;
        } else {
            T1 = Tab{g_keys, g_vals, nullptr, g_list, &s.n_list, uint32_t(gs - 1), int(gs / 2)};
            mark = g_mark;
            lk = g_lk;
            lts = g_lts;
            gbl = true;
            if ((int64_t)t1_cap <= gs) T1.mask = t1_cap - 1;
            else P = int((4 * u1 + gs - 1) / gs);
        }
        for (int p = 0; p < P; ++p) {
            if (gbl)
                for (int i = tid; i < s.BLOOM_W; i += NT_C) s.bloom[i] = 0;
            // ---- N(g1): x = |g1 & f| per distinct f != g1 (of partition p)
            for (int m0 = 0; m0 < k1; m0 += NT_C) {
                const int n = min(NT_C, k1 - m0);
                const int tot = load_segment<NT_C>(S, g1mem + m0, n, s.seg_off, nullptr, s.seg_pre, s.warp_tmp);
                for (int e = tid; e < tot; e += NT_C) {
                    const int m = seg_member(s.seg_pre, n, e);
                    const int32_t f = v2h[s.seg_off[m] + (e - s.seg_pre[m])];
                    if (f == g1) continue;
                    if (P > 1 && part_of(f, P) != p) continue;
                    tab_insert(T1, f, 1u, 0, A.sc);
                }
                acc.n_v2h += (tid < tot) ? (tot - tid + NT_C - 1) / NT_C : 0;
                __syncthreads();
            }
            const int n1 = min(s.n_list, T1.list_cap);
            // ---- what the per-h passes need of every f: size, changed flag,
            //      time; in aggregate mode the totals, the x window and the
            //      list of changed f
            const int wlo = k1 - kWin;
            for (int q0 = 0; q0 < n1; q0 += NT_C) {
                const int q = q0 + tid;
                int wkey = -1, C = 0;
                if (q < n1) {
                    const int sl = T1.list[q];
                    const int32_t f = T1.keys[sl];
                    const int kf = S.h_card[f];
                    const bool changed_f = bit_test(A.chg, f);
                    lk[q] = kf | (changed_f ? int32_t(0x80000000u) : 0);
                    if (gbl) {
                        g_lkey[q] = f;
                        const uint32_t bb = bloom_bit(f, s.BLOOM_W);
                        atomicOr(&s.bloom[bb >> 5], 1u << (bb & 31));
                    }
                    if (want_t) lts[q] = S.h_ts[f];
                    if (agg) {
                        const int x = int(T1.vals[sl]);
                        C = kf > x ? 1 : 0;
                        if (x >= wlo && x < k1) wkey = (x - wlo) * 2 + C;
                        if (changed_f) {
                            const int c = atomicAdd(&s.n_cl, 1);
                            lts[c] = int64_t(uint32_t(sl)) | (int64_t(kf) << 32);
                        }
                    }
                }
                if (agg) {
                    const unsigned in = __ballot_sync(0xffffffffu, q < n1);
                    const unsigned c1 = __ballot_sync(0xffffffffu, q < n1 && C == 1);
                    if (lane == 0) {
                        if (__popc(in & ~c1)) atomicAdd(&s.tot[0], __popc(in & ~c1));
                        if (__popc(c1)) atomicAdd(&s.tot[1], __popc(c1));
                    }
                    warp_count(&s.win[0][0], wkey);
                }
            }
            acc.n_meta += (tid < n1) ? (n1 - tid + NT_C - 1) / NT_C : 0;
            for (int64_t ch = c_beg; ch < c_end; ++ch) {
                const int64_t lbeg = l_lo + ch * LCH;
                const int nh = int(min(lbeg + LCH, l_hi) - lbeg);
                __syncthreads();
                // the chunk's changed hyperedges
                if (tid < nh) {
                    const int64_t e = lbeg + tid;
                    const int32_t li = cs.l_i[e];
                    const uint64_t xv1 = cs.l_xv[e];
                    const int32_t h = A.changed[A.lo + li];
                    s.hh[tid] = h;
                    s.hk[tid] = S.h_card[h];
                    s.hx[tid] = int(xv1 & kXMask);
                    s.hvf[tid] = int32_t(uint32_t(xv1 >> 32));
                    s.hli[tid] = li;
                    s.hts[tid] = S.h_ts[h];
                    s.hmem[tid] = h2v + S.h_off[h];
                    s.hnb[tid] = cs.nh_off[li] - R.base;
                    s.hnn[tid] = cs.nh_n[li];
                    s.htcap[tid] = cs.nh_tcap[li];
                    s.htoff[tid] = cs.nh_toff[li];
                    s.hr[tid] = cs.r_off[li];
                    s.hIn[tid] = 0;
                }
                __syncthreads();
                // h & g1 for the h sharing 2..kIC vertices with g1: the smaller list is
                // searched in the larger
                for (int l = 0; l < nh; ++l) {
                    const int xh1 = s.hx[l];
                    if (xh1 < 2 || xh1 > kIC) continue;
                    const int kh = s.hk[l];
                    const bool from_h = kh <= k1;
                    const int32_t* a = from_h ? s.hmem[l] : g1mem;
                    const int32_t* b = from_h ? g1mem : s.hmem[l];
                    const int na = from_h ? kh : k1, nb = from_h ? k1 : kh;
                    for (int i = tid; i < na; i += NT_C) {
                        const int32_t u = a[i];
                        if (contains_sorted(b, nb, u)) {
                            const int c = atomicAdd(&s.hIn[l], 1);
                            if (c < kIC) s.hI[l][c] = u;
                        }
                    }
                }
                if (tid == 0) {
                    // work of pass (i) per h: the smaller of N(h) and N(g1) when N(h)
                    // has a table to probe (aggregate mode), else all of N(h)
                    int run = 0;
                    for (int l = 0; l < nh; ++l) {
                        s.hpre[l] = run;
                        // a visit of N(g1) (mode 1: shared-memory list, one filter
                        // load) costs less than a visit of N(h) (mode 0: list from
                        // global memory, a hash probe); m1_pct weighs the two
                        int mode = 0, work = s.hnn[l];
                        if (!want_t && s.htcap[l] > 0) {
                            if (s.hr[l] >= 0 && k1 < min(s.hnn[l], n1)) {
                                mode = 2;
                                work = k1;
                            } else if (int64_t(n1) * 100 < int64_t(s.hnn[l]) * cs.m1_pct) {
                                mode = 1;
                                work = n1;
                            }
                        }
                        s.hfrom[l] = mode;
                        run += work;
                    }
                    s.hpre[nh] = run;
                }
                __syncthreads();
                const int n_cl = s.n_cl;

                // ---- (i) the pairs {g1, g2}, g2 in N(h), for every h of the item.
                // Every g2 also in N(g1) (a closed pair) is marked for that h and
                // counted at g1 < g2 unless g2 is a changed hyperedge of smaller
                // ID than h.  With the temporal family every g2 of N(h) is visited
                // (the open pairs centred at h are enumerated); otherwise the
                // closed pairs are found from the smaller of N(h) and N(g1),
                // probing the other's hash table, or, for an h with restricted
                // lists, from R(u) for the members u of g1.
                const int wtot = s.hpre[nh];
                if (tid == 0) acc.w[2] += (unsigned long long)wtot;
                // a closed pair {g1, g2} for the item's l-th h
                // a closed pair {g1, g2} for the item's l-th h; its bins go to
                // bh / bt / bn (class, temporal class, open-at-h class taken
                // back) for one warp-aggregated update, or, when direct, to
                // the histograms at once
                auto closed = [&](int l, int32_t h, int32_t g2, int sl, int xh2, int32_t vf2, int k2, bool chg2,
                                  int64_t ts2, int& skey, int& bh, int& bt, int& bn, bool direct) {
                    const int kh = s.hk[l], xh1 = s.hx[l];
                    const int x12 = int(T1.vals[sl]);
                    if (want_open && !direct) atomicOr(&mark[sl], 1u << l);
                    if (agg) {
                        const int b = (x12 != k1 - xh1 ? 2 : 0) | (k2 > x12 ? 1 : 0);
                        if (direct) atomicAdd(&s.sub[l][b], 1u);
                        else skey = l * 4 + b;
                    }
                    if (g2 > g1 && !(g2 < h && chg2)) {
                        ++acc.n_meta;
                        ++acc.w[3];
                        acc.n_closed += (unsigned long long)min(k1, k2);
                        const int t = triple_size(xh1, s.hvf[l], xh2, vf2, g1mem, k1, h2v + S.h_off[g2], k2, s.hmem[l],
                                                  kh, s.hI[l], s.hIn[l], acc.w[4]);
                        if (want_open)
                            classify_bins(s.tb, fam, delta, h, g1, g2, kh, k1, k2, xh1, x12, xh2, t, s.hts[l], ts1, ts2,
                                          bh, bt, acc);
                        if (agg) bn = s.tb.cls30[open_at_h_mask(kh, xh1, xh2, k1, k2)];
                        if (direct) {
                            if (bh >= 0) atomicAdd(&hist[bh], 1u);
                            if (bt >= 0) atomicAdd(&hist[kHistT + bt], 1u);
                            if (bn >= 0) atomicAdd(&s.hneg[wid][bn], 1u);
                            bh = bt = bn = -1;
                        }
                        if (fam & kFamV)
                            acc.v3 += (unsigned long long)xh1 * x12 * xh2 - (unsigned long long)t * (xh1 + x12 + xh2) +
                                      2ull * t;
                    }
                };
                for (int idx0 = 0; idx0 < wtot; idx0 += NT_C) {
                    const int idx = idx0 + tid;
                    int skey = -1, bh = -1, bt = -1, bn = -1;
                    if (idx < wtot) {
                        int l = 0, hi_l = nh - 1;  // the h of this work index: last l with hpre[l] <= idx
                        while (l < hi_l) {
                            const int mid = (l + hi_l + 1) >> 1;
                            if (s.hpre[mid] <= idx) l = mid;
                            else hi_l = mid - 1;
                        }
                        const int q = idx - s.hpre[l];
                        const int32_t h = s.hh[l];
                        const int mode = s.hfrom[l];
                        if (mode == 2) {
                            // the neighbours f of h holding the q-th member u of g1:
                            // each is in N(g1); one met through several shared
                            // vertices is taken once (its mark bit)
                            const int32_t* ridx = cs.r_pool + s.hr[l];
                            const int32_t* ent = ridx + S.nv[g] + 1;
                            const int64_t lu = int64_t(g1mem[q]) - S.vbase[g];
                            const int e1 = ridx[lu + 1];
                            for (int e = ridx[lu]; e < e1; ++e) {
                                ++acc.w[2];
                                const int32_t f = ent[e];
                                if (f == g1 || (P > 1 && part_of(f, P) != p)) continue;
                                const int sl = tab_find(T1, f);
                                if (sl < 0) continue;
                                if ((atomicOr(&mark[sl], 1u << l) >> l) & 1u) continue;
                                const int ps = probe_list_table(cs.nh_g + s.htoff[l], uint32_t(s.htcap[l] - 1), f);
                                if (ps < 0) continue;
                                const uint64_t xv2 = cs.nh_xv[s.htoff[l] + ps];
                                int unused, dh = -1, dt = -1, dn = -1;
                                closed(l, h, f, sl, int(xv2 & kXMask), int32_t(uint32_t(xv2 >> 32)), S.h_card[f],
                                       bit_test(A.chg, f), want_t ? S.h_ts[f] : 0, unused, dh, dt, dn, true);
                            }
                        } else if (mode == 1) {
                            const int32_t g2 = gbl ? g_lkey[q] : T1.keys[T1.list[q]];
                            // most g2 are not in N(h): the filter answers them
                            // with one load; the rest probe the table
                            const uint32_t tcap = uint32_t(s.htcap[l]);
                            uint32_t bits;
                            const uint32_t fw = reinterpret_cast<const uint32_t*>(
                                cs.nh_g + s.htoff[l] + tcap)[filter_word(g2, tcap, bits)];
                            const int ps = (fw & bits) == bits
                                               ? probe_list_table(cs.nh_g + s.htoff[l], tcap - 1, g2)
                                               : -1;
                            if (ps >= 0) {
                                const int sl = T1.list[q];
                                const uint64_t xv2 = cs.nh_xv[s.htoff[l] + ps];
                                const int32_t meta = lk[q];
                                closed(l, h, g2, sl, int(xv2 & kXMask), int32_t(uint32_t(xv2 >> 32)), meta & 0x7fffffff,
                                       meta < 0, want_t ? lts[q] : 0, skey, bh, bt, bn, false);
                            }
                        } else {
                            const int32_t g2 = cs.nh_g[s.hnb[l] + q];
                            if (P == 1 || part_of(g2, P) == p) {
                                int sl = -1;
                                if (gbl) {
                                    const uint32_t bb = bloom_bit(g2, s.BLOOM_W);
                                    if ((s.bloom[bb >> 5] >> (bb & 31)) & 1u) sl = tab_find(T1, g2);
                                } else {
                                    sl = tab_find(T1, g2);
                                }
                                if (sl >= 0 || (!agg && want_open)) {
                                    const uint64_t xv2 = cs.nh_xv[s.hnb[l] + q];
                                    const int xh2 = int(xv2 & kXMask);
                                    const int k2 = int((xv2 >> 16) & 0x7fffu);
                                    const bool chg2 = ((xv2 >> 31) & 1u) != 0;
                                    const int32_t vf2 = int32_t(uint32_t(xv2 >> 32));
                                    const int64_t ts2 = want_t ? cs.nh_ts[s.hnb[l] + q] : 0;
                                    if (sl >= 0) {
                                        closed(l, h, g2, sl, xh2, vf2, k2, chg2, ts2, skey, bh, bt, bn, false);
                                    } else if (g2 > g1 && !(g2 < h && chg2)) {
                                        // open pair centred at h, enumerated (temporal family kept)
                                        ++acc.n_meta;
                                        classify_bins(s.tb, fam, delta, h, g1, g2, s.hk[l], k1, k2, s.hx[l], 0, xh2, 0,
                                                      s.hts[l], ts1, ts2, bh, bt, acc);
                                    }
                                }
                            }
                        }
                    }
                    if (agg && __any_sync(0xffffffffu, skey >= 0)) warp_count(&s.sub[0][0], skey);
                    // one shared-memory atomic per distinct bin of the warp
                    // (most iterations of the hyperedge family classify nothing)
                    if (__any_sync(0xffffffffu, bh >= 0)) warp_count(hist, bh);
                    if (__any_sync(0xffffffffu, bt >= 0)) warp_count(hist + kHistT, bt);
                    if (agg && __any_sync(0xffffffffu, bn >= 0)) warp_count(s.hneg[wid], bn);
                }
                __syncthreads();
                if (agg) {
                    // (ii) in aggregate.  An open triad {h, g1, f} (f in N(g1),
                    // f outside N(h), f != h) has regions h-only |h| - |h&g1|,
                    // g1-only |g1| - |h&g1| - |g1&f|, f-only |f| - |g1&f|, h&g1
                    // and g1&f non-empty, the rest empty: its class is set by
                    // A = [h not inside g1] and the bucket b = 2B + C of f, with
                    // B = [|g1&f| != |g1| - |h&g1|], C = [f not inside g1].  The
                    // buckets over all of N(g1) come from the totals and the x
                    // window; subtracted are the f in N(h) (marked in (i)), f = h,
                    // and the changed f < h (attributed to f).
                    const int wc = nh * n_cl;
                    if (tid == 0) acc.w[5] += (unsigned long long)wc;
                    for (int idx0 = 0; idx0 < wc; idx0 += NT_C) {
                        const int idx = idx0 + tid;
                        int skey = -1;
                        if (idx < wc) {
                            const int l = idx / n_cl, c = idx - l * n_cl;
                            const int64_t v = lts[c];
                            const int sl = int(uint32_t(v));
                            const int32_t f = T1.keys[sl];
                            if (f < s.hh[l] && !((mark[sl] >> l) & 1u)) {
                                const int x = int(T1.vals[sl]);
                                skey = l * 4 + ((x != k1 - s.hx[l] ? 2 : 0) | (int(v >> 32) > x ? 1 : 0));
                            }
                        }
                        warp_count(&s.sub[0][0], skey);
                    }
                    if (tid < nh && (P == 1 || part_of(s.hh[tid], P) == p)) {
                        const int xh1 = s.hx[tid];
                        atomicAdd(&s.sub[tid][(xh1 != k1 - xh1 ? 2 : 0) | (s.hk[tid] > xh1 ? 1 : 0)], 1u);
                    }
                    for (int l = 0; l < nh; ++l) {  // x = |g1| - |h&g1| outside the window
                        if (s.hx[l] <= kWin) continue;
                        const int xstar = k1 - s.hx[l];
                        for (int q = tid; q < n1; q += NT_C)
                            if (int(T1.vals[T1.list[q]]) == xstar)
                                atomicAdd(&s.xc[l][(lk[q] & 0x7fffffff) > xstar ? 1 : 0], 1u);
                    }
                    __syncthreads();
                    if (tid < nh) {
                        const int xh1 = s.hx[tid], kh = s.hk[tid];
                        const int A_bit = kh > xh1 ? 1 : 0;
                        for (int b = 0; b < 4; ++b) {
                            const int B = b >> 1, C = b & 1;
                            const uint32_t h0 = xh1 <= kWin ? s.win[kWin - xh1][C] : s.xc[tid][C];
                            const uint32_t total = B == 0 ? h0 : s.tot[C] - h0;
                            const uint32_t n = total - s.sub[tid][b];
                            if (n) {
                                const int m = A_bit | (B << 1) | (C << 2) | (1 << 3) | (1 << 4);
                                atomicAdd(&hist[s.tb.cls30[m]], n);
                                acc.n_tri += n;
                            }
                            s.sub[tid][b] = 0;
                        }
                        s.xc[tid][0] = s.xc[tid][1] = 0;
                    }
                } else if (want_open) {
                    // (ii) open triads {h, g1, f} centred at g1: f in N(g1),
                    // outside N(h) (unmarked), f != h, f not a changed
                    // hyperedge of smaller ID than h.  Their class is set by
                    // A = [h not inside g1], the bucket 2B + C of f (as in
                    // aggregate mode) and, for the temporal family, by where f
                    // falls in time against h and g1 (before both, between,
                    // after both) and whether that triple fits the window; so
                    // one warp per h counts its f by (position, bucket) and
                    // classifies each count once.
                    for (int l = wid; l < nh; l += NW_C) {
                        const int32_t h = s.hh[l];
                        const int xh1 = s.hx[l], xstar = k1 - xh1;
                        const int64_t th = s.hts[l];
                        const bool h_first = th < ts1 || (th == ts1 && h < g1);
                        const int64_t tp = h_first ? th : ts1, tq = h_first ? ts1 : th;
                        const int32_t ip = h_first ? h : g1, iq = h_first ? g1 : h;
                        uint32_t cst[4] = {0, 0, 0, 0};
                        uint32_t ctm[3][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
                        for (int q = lane; q < n1; q += 32) {
                            const int sl = T1.list[q];
                            const int32_t f = T1.keys[sl];
                            if (f == h) continue;
                            const int32_t meta = lk[q];
                            if (meta < 0 && f < h) continue;  // changed, smaller ID: attributed to f
                            if ((mark[sl] >> l) & 1u) continue;
                            const int x = int(T1.vals[sl]);
                            const int b = (x != xstar ? 2 : 0) | ((meta & 0x7fffffff) > x ? 1 : 0);
                            int r = -1;  // position in time, -1: outside the window
                            if (want_t) {
                                const int64_t tf = lts[q];
                                if (tf < tp || (tf == tp && f < ip)) r = tq - tf <= delta ? 0 : -1;
                                else if (tf < tq || (tf == tq && f < iq)) r = tq - tp <= delta ? 1 : -1;
                                else r = tf - tp <= delta ? 2 : -1;
                            }
                            // constant indices keep the counters in registers
#pragma unroll
                            for (int bb = 0; bb < 4; ++bb) {
                                cst[bb] += b == bb ? 1u : 0u;
#pragma unroll
                                for (int rr = 0; rr < 3; ++rr) ctm[rr][bb] += (b == bb && r == rr) ? 1u : 0u;
                            }
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                            for (int b = 0; b < 4; ++b) {
                                cst[b] += __shfl_xor_sync(0xffffffffu, cst[b], o);
#pragma unroll
                                for (int r = 0; r < 3; ++r) ctm[r][b] += __shfl_xor_sync(0xffffffffu, ctm[r][b], o);
                            }
                        }
                        if (lane == 0) {
                            const int A_bit = s.hk[l] > xh1 ? 1 : 0;
                            // labels 0 = h, 1 = g1, 2 = f; p and q are h and g1 in time order
                            const int lp = h_first ? 0 : 1, lq = h_first ? 1 : 0;
                            for (int b = 0; b < 4; ++b) {
                                const int m = A_bit | ((b >> 1) << 1) | ((b & 1) << 2) | (1 << 3) | (1 << 4);
                                acc.n_tri += cst[b];
                                if ((fam & kFamH) && cst[b] && s.tb.cls30[m] >= 0)
                                    atomicAdd(&hist[s.tb.cls30[m]], cst[b]);
                                if (!want_t) continue;
                                for (int r = 0; r < 3; ++r) {
                                    if (!ctm[r][b]) continue;
                                    const int o0 = r == 0 ? 2 : lp, o1 = r == 0 ? lp : (r == 1 ? 2 : lq);
                                    const int c = s.tb.cls96[s.tb.perm[perm_index(o0, o1)][m]];
                                    if (c >= 0) atomicAdd(&hist[kHistT + c], ctm[r][b]);
                                }
                            }
                        }
                    }
                }
                __syncthreads();
                for (int i = tid; i < n1; i += NT_C) mark[T1.list[i]] = 0;
                // fold the warp histograms of this chunk
                for (int b = tid; b < kHistN; b += NT_C) {
                    unsigned long long v = 0;
                    for (int w = 0; w < NW_C; ++w) {
                        v += s.hist[w][b];
                        s.hist[w][b] = 0;
                        if (b < 32) {
                            v -= s.hneg[w][b];
                            s.hneg[w][b] = 0;
                        }
                    }
                    s.acc[b] += v;
                }
                __syncthreads();
            }  // chunks
            tab_clear<NT_C>(T1, n1);
            if (agg) {
                if (tid < 2) s.tot[tid] = 0;
                for (int i = tid; i < kWin * 2; i += NT_C) s.win[i >> 1][i & 1] = 0;
            }
            __syncthreads();
            if (tid == 0) {
                s.n_list = 0;
                s.n_cl = 0;
            }
        }
    }
    __syncthreads();
    if (cur_g >= 0) flush<NT_C>(A, s.acc, s.hist, NW_C, cur_g, acc, s.red);
    flush_stats<NT_C>(A, acc, s.red);
}

// a + b and a - b for b >= 0, held within the int64 range
__device__ __forceinline__ int64_t sat_add(int64_t a, int64_t b) { return a > INT64_MAX - b ? INT64_MAX : a + b; }
__device__ __forceinline__ int64_t sat_sub(int64_t a, int64_t b) { return a < INT64_MIN + b ? INT64_MIN : a - b; }

// ---------------------------------------------------------------------------
// 3a. open triads centred at h, temporal classes (oriented counter)
// ---------------------------------------------------------------------------
//
// Every unordered pair {a, b} of N'(h) (N(h) without the changed g < h) is
// an open triad {h, a, b} centred at h unless a meets b; the centre kernel
// finds the closed ones and takes back the class counted here.  With the
// labels h, a (earlier in (t, ID) order), b (later), the class depends on
// the mask bits [|h| != x_a + x_b], C_a = [a not inside h], C_b, and on
// where h falls in time.  With N'(h) sorted by (t, ID) and h's place s:
//   h last:   a, b both before h, within [t_h - delta, t_h]: one range;
//   h first:  a, b both after h, within [t_h, t_h + delta]: one range;
//   h middle: a before h, b after h with t_b - t_a <= delta: a range of b per a.
// Pairs inside a range are counted per later member from prefix counts of C;
// those with x_a + x_b = |h| from a second order by (x, place): the members
// with x = |h| - x_b and places in [L, b) are one stretch of it.  Work per h
// is O(n log^2 n) (two bitonic sorts) instead of one visit per pair.  A list
// of at most kOhMax entries (cs.oh_smem) is sorted in shared memory, a longer
// one of at most cs.oh_cap in the block's global scratch (the same code on
// L2-resident arrays); one longer still (or than cs.oh_max) is left to the
// centre kernel, which then classifies every pair of it (flag bit 1 of
// nh_flag).
constexpr int kOhNT = 1024;
constexpr int kOhMax = 8192;   // entries of N'(h) sorted in shared memory, at most
constexpr int kOhBig = 65536;  // entries sorted in the block's global scratch, at most
// short lists (at most kOsMax entries, most of them on sparse graphs) go to
// kOsNT-thread blocks with shared arrays for kOsMax entries, several per SM:
// a sort over a few hundred entries then waits at barriers of 8 warps, not 32
constexpr int kOsNT = 256;
constexpr int kOsMax = 1024;

template <int NT, int MAXN>
struct SmemOHT {
    Tables tb;
    int64_t t[MAXN];           // timestamp of each entry (sorted with id and pay)
    int32_t id[MAXN];
    int32_t pay[MAXN];         // x | C << 15
    uint32_t key[MAXN];        // x << ksh | place << 1 | C, sorted
    uint16_t p1[MAXN + 1];     // entries with C = 1 among the first i, in (t, ID) order
    uint16_t pc[MAXN + 1];     // the same in key order
    unsigned long long cnt[24];
    int wsum[NT / 32];
    long long item;
    int n, s_pos, l0, r1;
};
using SmemOH = SmemOHT<kOhNT, kOhMax>;
using SmemOS = SmemOHT<kOsNT, kOsMax>;

// out[i] = number of the first i of n entries with bit(i) set, and out[n]
template <int NT, typename PT, typename F>
__device__ __forceinline__ void oh_prefix(F bit, PT* out, int n, int* wsum) {
    const int tid = threadIdx.x, lane = lane_id(), w = warp_id();
    const int per = (n + NT - 1) / NT;
    const int q0 = tid * per, q1 = min(q0 + per, n);
    int c = 0;
    for (int q = q0; q < q1; ++q) c += bit(q);
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int x = lane < NT / 32 ? wsum[lane] : 0;
        const int own = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += v;
        }
        if (lane < NT / 32) wsum[lane] = x - own;
        if (lane == 31) out[n] = PT(x);
    }
    __syncthreads();
    int run = wsum[w] + inc - c;
    for (int q = q0; q < q1; ++q) {
        out[q] = PT(run);
        run += bit(q);
    }
    __syncthreads();
}

// The counts of one later member (or, in the middle case, of one earlier
// member against a range of later ones): CE is that member's C bit.
// Counter index: case * 8 + E * 4 + C_a * 2 + C_b.
template <int CE>
__device__ __forceinline__ void oh_add(unsigned (&c)[24], int cas, bool later, int tot, int t1, int e, int e1) {
    // tot members in the range, t1 of them with C = 1; e with x_a + x_b = |h|,
    // e1 of those with C = 1
    const int k = cas * 8;
    if (later) {  // the range holds the earlier members a; b is this one
        c[k + 4 + 2 + CE] += unsigned(e1);
        c[k + 4 + 0 + CE] += unsigned(e - e1);
        c[k + 0 + 2 + CE] += unsigned(t1 - e1);
        c[k + 0 + 0 + CE] += unsigned((tot - t1) - (e - e1));
    } else {      // this one is a; the range holds the later members b
        c[k + 4 + CE * 2 + 1] += unsigned(e1);
        c[k + 4 + CE * 2 + 0] += unsigned(e - e1);
        c[k + 0 + CE * 2 + 1] += unsigned(t1 - e1);
        c[k + 0 + CE * 2 + 0] += unsigned((tot - t1) - (e - e1));
    }
}

// The open triads centred at h over the n entries of N'(h) loaded into
// (T, I, P), in shared memory or the block's global scratch: sorted, ranked
// and counted into s.cnt, then added to graph g's temporal bins.  ksh: the
// key shift (places < 1 << (ksh - 1)).
template <int NT, int MAXN, typename PT>
__device__ void oh_count(SmemOHT<NT, MAXN>& s, const CountArgs& A, int n, int64_t* T, int32_t* I, int32_t* P,
                         uint32_t* K, PT* P1, PT* PC, int ksh, int kh, int64_t th, int32_t h, int g) {
    const int tid = threadIdx.x, lane = lane_id();
    const int64_t delta = A.S.delta;
    int n2 = 2;
    while (n2 < n) n2 <<= 1;
    for (int q = n + tid; q < n2; q += NT) {
        T[q] = INT64_MAX;
        I[q] = INT_MAX;
        P[q] = 0;
    }
    __syncthreads();
    // bitonic sort by (t, ID)
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int u = tid; u < (n2 >> 1); u += NT) {
                const int a = ((u & ~(j - 1)) << 1) | (u & (j - 1)), b = a + j;
                const int64_t ta = T[a], tb = T[b];
                const int32_t ia = I[a], ib = I[b];
                if ((ta > tb || (ta == tb && ia > ib)) == ((a & k) == 0)) {
                    T[a] = tb;
                    T[b] = ta;
                    I[a] = ib;
                    I[b] = ia;
                    const int32_t pa = P[a];
                    P[a] = P[b];
                    P[b] = pa;
                }
            }
            __syncthreads();
        }
    for (int q = tid; q < n2; q += NT)
        K[q] = q < n ? (uint32_t(P[q] & 0x7fff) << ksh) | (uint32_t(q) << 1) | uint32_t((P[q] >> 15) & 1) : UINT32_MAX;
    oh_prefix<NT, PT>([&](int q) { return (P[q] >> 15) & 1; }, P1, n, s.wsum);
    // bitonic sort of the keys
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int u = tid; u < (n2 >> 1); u += NT) {
                const int a = ((u & ~(j - 1)) << 1) | (u & (j - 1)), b = a + j;
                const uint32_t ka = K[a], kb = K[b];
                if ((ka > kb) == ((a & k) == 0)) {
                    K[a] = kb;
                    K[b] = ka;
                }
            }
            __syncthreads();
        }
    oh_prefix<NT, PT>([&](int q) { return int(K[q] & 1u); }, PC, n, s.wsum);
    if (tid == 0) {
        // h's place, the first member within delta before it, the end of
        // the members within delta after it
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (T[mid] < th || (T[mid] == th && I[mid] < h)) lo = mid + 1;
            else hi = mid;
        }
        const int sp = lo;
        lo = 0;
        hi = sp;
        const int64_t tlo = sat_sub(th, delta), thi = sat_add(th, delta);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (T[mid] < tlo) lo = mid + 1;
            else hi = mid;
        }
        s.l0 = lo;
        lo = sp;
        hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (T[mid] <= thi) lo = mid + 1;
            else hi = mid;
        }
        s.r1 = lo;
        s.s_pos = sp;
    }
    __syncthreads();
    const int sp = s.s_pos, l0 = s.l0, r1 = s.r1;
    // the first key at or above v (targets are formed in 64 bits: with the
    // place n << 1 they reach the first key of the next x)
    auto key_lb = [&](uint64_t v) {
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (uint64_t(K[mid]) < v) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    unsigned c[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) c[k] = 0;
    for (int e = tid; e < n; e += NT) {
        const int xe = P[e] & 0x7fff;
        const int ce = (P[e] >> 15) & 1;
        const int xs = kh - xe;  // the x of a partner that completes h
        // members in places [L, R) with x = xs: how many, and with C = 1
        auto match = [&](int L, int Rr, int& m, int& m1) {
            m = m1 = 0;
            if (xs < 1 || L >= Rr) return;
            const int i0 = key_lb((uint64_t(xs) << ksh) + (uint64_t(L) << 1));
            const int i1 = key_lb((uint64_t(xs) << ksh) + (uint64_t(Rr) << 1));
            m = i1 - i0;
            m1 = int(PC[i1]) - int(PC[i0]);
        };
        auto range = [&](int cas, bool later, int L, int Rr) {
            if (L >= Rr) return;
            int m, m1;
            match(L, Rr, m, m1);
            const int tot = Rr - L, t1 = int(P1[Rr]) - int(P1[L]);
            if (ce) oh_add<1>(c, cas, later, tot, t1, m, m1);
            else oh_add<0>(c, cas, later, tot, t1, m, m1);
        };
        if (e >= l0 && e < sp) range(0, true, l0, e);   // h last: a in [l0, e)
        if (e >= sp && e < r1) range(1, true, sp, e);   // h first: a in [sp, e)
        if (e < sp) {                                   // h middle: b after h within delta of e
            const int64_t tb = sat_add(T[e], delta);
            int lo = sp, hi = n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (T[mid] <= tb) lo = mid + 1;
                else hi = mid;
            }
            range(2, false, sp, lo);
        }
    }
#pragma unroll
    for (int k = 0; k < 24; ++k) {
        unsigned v = c[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(&s.cnt[k], (unsigned long long)v);
    }
    __syncthreads();
    if (tid < 24 && s.cnt[tid]) {
        const int cas = tid >> 3, E = (tid >> 2) & 1, ca = (tid >> 1) & 1, cb = tid & 1;
        // labels 0 = h, 1 = a, 2 = b; order: h last (a, b, h), first (h, a, b), middle (a, h, b)
        const int m = (E ? 0 : 1) | (ca ? 2 : 0) | (cb ? 4 : 0) | (1 << 3) | (1 << 5);
        const int pi = cas == 0 ? perm_index(1, 2) : cas == 1 ? perm_index(0, 1) : perm_index(1, 0);
        const int cl = s.tb.cls96[s.tb.perm[pi][m]];
        if (cl >= 0)
            atomicAdd(reinterpret_cast<unsigned long long*>(&A.dc[int64_t(g) * kCStride + kOffT + cl]), s.cnt[tid]);
    }
}

// SHORT: the kOsNT-thread variant, for lists of at most short_cap entries
// (before the changed g < h are dropped); the other takes the longer ones.
// Both walk all of the run's changed h, each through its own queue.
template <int NT, int MAXN, int MINB, bool SHORT>
__global__ void __launch_bounds__(NT, MINB) k_open_h(CountArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemOHT<NT, MAXN>& s = *reinterpret_cast<SmemOHT<NT, MAXN>*>(smem_raw);
    const Store& S = A.S;
    if (A.sc->gate) return;
    const CountScratch& cs = A.cs;
    const int tid = threadIdx.x;
    const RunRange R = run_of(A);
    const int short_cap = min(kOsMax, cs.oh_smem);
    const int smem_max = min(MAXN, cs.oh_smem);
    const int64_t gstride = cs.oh_cap + 1;
    int64_t* gT = cs.oh_t + blockIdx.x * gstride;
    int32_t* gI = cs.oh_i + blockIdx.x * gstride;
    int32_t* gP = cs.oh_p + blockIdx.x * gstride;
    uint32_t* gK = cs.oh_k + blockIdx.x * gstride;
    uint32_t* gP1 = cs.oh_p1 + blockIdx.x * gstride;
    uint32_t* gPC = cs.oh_pc + blockIdx.x * gstride;
    unsigned long long* queue = SHORT ? &A.sc->qos[A.side] : &A.sc->qoh[A.side];
    load_tables(s.tb, NT);
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            s.item = (long long)atomicAdd(queue, 1ull);
            s.n = 0;
        }
        if (tid < 24) s.cnt[tid] = 0;
        __syncthreads();
        if (s.item >= R.n) break;
        const int64_t i = cs.order[s.item];
        const int nn = cs.nh_n[i];
        if (nn < 2) continue;
        if (SHORT != (nn <= short_cap)) continue;  // the other variant's
        const int32_t h = A.changed[A.lo + i];
        const int g = A.changed_g ? A.changed_g[A.lo + i] : 0;
        const int kh = S.h_card[h];
        const int64_t th = S.h_ts[h];
        const int64_t base = cs.nh_off[i] - R.base;
        // N'(h), into shared memory while it fits, else into the block's
        // global scratch while that fits
        auto load = [&](int64_t* T, int32_t* I, int32_t* P, int cap) {
            for (int q = tid; q < nn; q += NT) {
                const int32_t gg = cs.nh_g[base + q];
                const uint64_t xv = cs.nh_xv[base + q];
                if (gg < h && ((xv >> 31) & 1u)) continue;  // changed below h: its triads belong to gg
                const int p = atomicAdd(&s.n, 1);
                if (p < cap) {
                    const int x = int(xv & kXMask), kg = int((xv >> 16) & 0x7fffu);
                    T[p] = cs.nh_ts[base + q];
                    I[p] = gg;
                    P[p] = x | (kg > x ? 1 << 15 : 0);
                }
            }
            __syncthreads();
        };
        load(s.t, s.id, s.pay, smem_max);
        const int n = s.n;
        if (n < 2) continue;
        if (n > cs.oh_max) {
            if (tid == 0) cs.nh_flag[i] |= 2;  // left to the centre kernel
        } else if (n <= smem_max) {
            oh_count<NT, MAXN, uint16_t>(s, A, n, s.t, s.id, s.pay, s.key, s.p1, s.pc, 14, kh, th, h, g);
        } else if (!SHORT && n <= cs.oh_cap) {
            __syncthreads();
            if (tid == 0) s.n = 0;
            __syncthreads();
            load(gT, gI, gP, int(cs.oh_cap));
            oh_count<NT, MAXN, uint32_t>(s, A, n, gT, gI, gP, gK, gP1, gPC, 17, kh, th, h, g);
        } else if (tid == 0) {
            cs.nh_flag[i] |= 2;  // left to the centre kernel
        }
    }
}

// ---------------------------------------------------------------------------
// 3b. oriented centre kernel (all neighbourhood families)
// ---------------------------------------------------------------------------
//
// Without the temporal family every open triad is counted in aggregate, so
// the pair pass only has to find the closed pairs {g1, g2} of N(h).  Each is
// searched from one side only: from the smaller of g1, g2 in the order
// (|g|, g).  For a pair (h, g1) that is either the part of N(h) above g1 (a
// suffix of h's list, sorted by k_nh_build), each probing N(g1)'s table
// (mode 0), or the part of N(g1) above g1 (the "plus list" built here), each
// probing N(h)'s filter and table (mode 1), whichever is shorter; an N(h) too
// long to sort is met through its table, or, when it has none, visited whole
// with the order tested per entry (mode 3).
//
// The aggregates count every pair of N'(h) (open at h, k_nh_build) and every
// f of N(g1) (open at g1, below) as open.  A closed triad {h, g1, g2} found
// here takes back the three open classes the aggregates gave it -- centred
// at h, at g1 (with f = g2) and at g2 (with f = g1) -- and adds its closed
// class.  The changed f < h of N(g1) are left out of h's aggregate at g1
// whether or not they lie in N(h): their triads belong to f.  So no mark of
// N(h) inside N(g1) is kept, and every closed triad is classified once.
//
// With the temporal family (TEMP) an open triad's class also depends on the
// time order of its three hyperedges and on the window, which no aggregate
// over N(g1) or N'(h) keeps.  The pair pass then visits every g2 of N'(h)
// above g1 (modes 0 and 3; the plus list is not used): a g2 outside N(g1)
// is an open triad centred at h, classified on the spot, a g2 inside it a
// closed pair, queued as before.  Open triads centred at g1 are counted per
// h by a warp over N(g1), bucketed by the static class bits and by where f
// falls in time against h and g1 (a constant number of counters per h).  A
// closed triad takes back the two open classes the warp pass gave it (at g1
// with f = g2, at g2 with f = g1), static and temporal, and adds its closed
// class; open triads at h need no taking back, since only open pairs were
// classified as such.

constexpr int kG1M = 1024;  // members of g1 kept in shared memory, at most

// t = |h & g1 & g2| for the oriented kernel (as triple_size).  When one of
// |h & g1|, |h & g2| is 1, its vertex v lies in h, so v is in the other
// intersection only if it is not below that one's smallest vertex: the order
// of the two smallest shared vertices settles most cases without a search.
// g1m holds g1's members (shared memory when they fit).
__device__ __forceinline__ int triple_size_o(int xh1, int32_t vf1, int xh2, int32_t vf2, const int32_t* g1m, int k1,
                                             const int32_t* g2mem, int k2, const int32_t* hmem, int kh,
                                             const int32_t* hI, int nI, unsigned long long& slow) {
    if (xh1 == 1 && xh2 == 1) return vf1 == vf2;
    if (xh1 == 1) {  // t = [vf1 in g2]
        if (vf1 <= vf2) return vf1 == vf2;
        return contains_sorted(g2mem, k2, vf1);
    }
    if (xh2 == 1) {  // t = [vf2 in g1]
        if (vf2 <= vf1) return vf2 == vf1;
        return contains_sorted(g1m, k1, vf2);
    }
    return triple_size(xh1, vf1, xh2, vf2, g1m, k1, g2mem, k2, hmem, kh, hI, nI, slow);
}

constexpr int kXG = 64;  // |h & g1| values whose place in the sweep's x order is tabulated

template <int NT_C, int T1_S>
struct SmemCO {
    static constexpr int NW_C = NT_C / 32;
    static constexpr int BLOOM_W = 2048;
    Tables tb;
    uint32_t hist[NW_C][32];
    uint32_t hneg[NW_C][32];     // open classes taken back for closed triads
    unsigned long long acc[32];
    int32_t keys[T1_S];
    uint32_t vals[T1_S];
    int32_t list[T1_S / 2];
    int32_t lk[T1_S / 2];        // |f|, bit 31: f is changed
    union {
        struct {
            int32_t pf[T1_S / 2];    // plus list: f above g1 ...
            uint32_t pm[T1_S / 2];   // ... and |g1 & f| | |f| << 16 | changed << 31
        } p;
        int64_t lts[T1_S / 2];       // with the temporal family: the timestamp of every f
    } u1;
    union {
        long long cl[T1_S / 2];      // changed f: f | |g1 & f| << 31 | |f| << 46
        struct {                     // with the temporal family:
            uint32_t th[NW_C][kNT];  //   temporal class bins per warp
            uint32_t tn[kNT];        //   temporal classes taken back for closed triads
            unsigned long long tacc[kNT];
            int64_t hts[LCH];        //   timestamps of the chunk's h
            // the sweep over N(g1): the chunk's h in (t, ID) order and in
            // (|h & g1|, t, ID) order, the place of each h in both, and the
            // range counts by (time position r, C) of each order (r = 3:
            // every h, for the static classes)
            int64_t ot_t[LCH], ox_t[LCH];
            int32_t ot_i[LCH], ox_i[LCH], ox_x[LCH];
            int32_t pt[LCH], px[LCH];
            int32_t dT[8][LCH + 1], dX[8][LCH + 1];
            uint8_t xg[2][kXG];      //   the h with |h & g1| = x (x < kXG): [xg[0][x], xg[1][x]) of the x order
            int n_before;            //   the chunk's h before g1 in (t, ID) order
        } t;
    } u2;
    int64_t seg_off[NT_C];
    int32_t seg_pre[NT_C + 1];
    int warp_tmp[32];
    long long red[NW_C];
    long long item;
    int n_list, n_plus, n_cl, n_c, n_li, n_lx, any_big;
    int32_t li_I[LCH], li_X[LCH];  // the h of a chunk with 2 <= |h&g1| <= kIC, and with |h&g1| > kWin
    uint32_t tot[2];
    uint32_t win[kWin][2];
    // the changed hyperedges h of a chunk
    int32_t hh[LCH], hk[LCH], hx[LCH], hvf[LCH], hnn[LCH], htcap[LCH], hpos[LCH], hmode[LCH];
    int64_t hnb[LCH], htoff[LCH];
    const int32_t* hmem[LCH];
    int32_t hord[LCH];           // the h with work in the pair pass, and the prefix of their work
    int32_t hpre[LCH + 1];
    uint32_t sub[LCH][4];
    uint32_t xc[LCH][2];
    int32_t hI[LCH][kIC];
    int hIn[LCH];
    // per warp, the closed pairs found and not yet classified: g2 | vf2 << 32,
    // and |g1 & g2| | |h & g2| << 16 | |g2| << 32 | l << 48
    unsigned long long cq0[NW_C][64], cq1[NW_C][64];
    uint32_t bloom[BLOOM_W];     // one-hash filter of N(g1)
    int32_t g1m[kG1M];           // g1's members, when |g1| <= kG1M
};

static_assert(sizeof(SmemCO<256, 2048>) + 1024 <= 233472 / 3, "three 256-thread oriented centre blocks per SM");

constexpr int kSweepMin = 4;  // chunks with fewer h count the open triads at g1 per h

__device__ __forceinline__ unsigned long long order_key(int k, int32_t g) {
    return (uint64_t(uint32_t(k)) << 32) | uint64_t(uint32_t(g));
}

// Temporal class of the triple with labels a, b, c (7-bit mask m under those
// labels), timestamps ta, tb, tc and IDs ia, ib, ic: the labels ordered by
// (timestamp, ID), the mask read in that order; -1 outside the window.
__device__ __forceinline__ int temporal_class(const Tables& tbl, int m, int64_t ta, int64_t tb, int64_t tc,
                                              int32_t ia, int32_t ib, int32_t ic, int64_t delta) {
    const int64_t T[3] = {ta, tb, tc};
    const int32_t I[3] = {ia, ib, ic};
    int o0 = 0, o1 = 1, o2 = 2, tmp;
#define ESC_BEFORE(x, y) (T[x] < T[y] || (T[x] == T[y] && I[x] < I[y]))
    if (ESC_BEFORE(o1, o0)) { tmp = o0; o0 = o1; o1 = tmp; }
    if (ESC_BEFORE(o2, o1)) { tmp = o1; o1 = o2; o2 = tmp; }
    if (ESC_BEFORE(o1, o0)) { tmp = o0; o0 = o1; o1 = tmp; }
#undef ESC_BEFORE
    return T[o2] - T[o0] <= delta ? tbl.cls96[tbl.perm[perm_index(o0, o1)][m]] : -1;
}

template <int NT_C, int T1_S, int MINB, bool TEMP>
__global__ void __launch_bounds__(NT_C, MINB) k_center_o(CountArgs A) {
    constexpr int NW_C = NT_C / 32;
    using Sm = SmemCO<NT_C, T1_S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm& s = *reinterpret_cast<Sm*>(smem_raw);
    const Store& S = A.S;
    if (A.sc->gate) return;
    const int tid = threadIdx.x;
    const int lane = lane_id();
    const int wid = warp_id();
    const uint32_t fam = S.fam;
    const bool want_h = (fam & kFamH) != 0;
    // without the temporal family the open triads are counted in aggregate;
    // with it (TEMP) the open triads centred at h are enumerated from the
    // suffixes of N(h) and those centred at g1 counted per h by time position
    const bool agg = want_h && !TEMP;
    const int64_t delta = S.delta;
    const CountScratch& cs = A.cs;
    const RunRange R = run_of(A);
    const int32_t* v2h = S.vp.arena;
    const int32_t* h2v = S.hp.arena;
    load_tables(s.tb, NT_C);
    for (int i = tid; i < NW_C * 32; i += NT_C) {
        s.hist[i / 32][i % 32] = 0;
        s.hneg[i / 32][i % 32] = 0;
    }
    for (int i = tid; i < 32; i += NT_C) s.acc[i] = 0;
    if constexpr (TEMP) {
        for (int i = tid; i < NW_C * kNT; i += NT_C) s.u2.t.th[i / kNT][i % kNT] = 0;
        for (int i = tid; i < kNT; i += NT_C) {
            s.u2.t.tn[i] = 0;
            s.u2.t.tacc[i] = 0;
        }
    }
    for (int i = tid; i < T1_S; i += NT_C) {
        s.keys[i] = EMPTY;
        s.vals[i] = 0;
    }
    for (int i = tid; i < Sm::BLOOM_W; i += NT_C) s.bloom[i] = 0;
    for (int i = tid; i < LCH * 4; i += NT_C) s.sub[i >> 2][i & 3] = 0;
    for (int i = tid; i < LCH * 2; i += NT_C) s.xc[i >> 1][i & 1] = 0;
    if (tid < 2) s.tot[tid] = 0;
    for (int i = tid; i < kWin * 2; i += NT_C) s.win[i >> 1][i & 1] = 0;
    if (tid == 0) {
        s.n_list = 0;
        s.n_plus = 0;
        s.n_cl = 0;
    }
    __syncthreads();
    const int64_t gs = cs.gs_c;
    int32_t* g_keys = cs.oc_keys + blockIdx.x * gs;
    uint32_t* g_vals = cs.oc_vals + blockIdx.x * gs;
    int32_t* g_list = cs.oc_list + blockIdx.x * (gs / 2);
    int32_t* g_lk = cs.oc_lk + blockIdx.x * (gs / 2);
    int32_t* g_pf = cs.oc_pf + blockIdx.x * (gs / 2);
    uint32_t* g_pm = cs.oc_pm + blockIdx.x * (gs / 2);
    long long* g_cl = reinterpret_cast<long long*>(cs.oc_lts) + blockIdx.x * (gs / 2);
    int64_t* g_lts = cs.oc_lts + blockIdx.x * (gs / 2);
    uint32_t* hist = s.hist[wid];
    uint32_t* hneg = s.hneg[wid];
    Accum acc = {0, 0, 0, 0, 0, 0, 0, 0, {0, 0, 0, 0, 0, 0}, 0, 0, 0, 0, 0};
    const int64_t n_items = A.sc->items[A.side];
    const int nd = A.sc->n_d[A.side];
    int cur_g = -1;

    for (;;) {
        __syncthreads();
        if (tid == 0) s.item = (long long)atomicAdd(&A.sc->queue[A.side], 1ull);
        __syncthreads();
        const int64_t item = s.item;
        if (item >= n_items) break;
        const int64_t j = cs.item_j[item];
        const int64_t sup = item - cs.d_item_start[j];
        const int32_t g1 = cs.d_list[j];
        const int64_t l_lo = cs.d_loff[j], l_hi = cs.d_loff[j + 1];
        const int64_t n_chunks = (l_hi - l_lo + LCH - 1) / LCH;
        const int64_t c_beg = sup * kSuper, c_end = min(c_beg + kSuper, n_chunks);
        const int64_t nh_all = min(l_lo + c_end * LCH, l_hi) - (l_lo + c_beg * LCH);
        const int g = A.changed_g ? A.changed_g[A.lo + cs.l_i[l_lo + c_beg * LCH]] : 0;
        if (g != cur_g) {
            if (cur_g >= 0) {
                __syncthreads();
                for (int b = tid; b < kNH; b += NT_C) {
                    unsigned long long v = s.acc[b];
                    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&A.dc[int64_t(cur_g) * kCStride + b]), v);
                    s.acc[b] = 0;
                }
                if constexpr (TEMP)
                    for (int b = tid; b < kNT; b += NT_C) {
                        unsigned long long v = s.u2.t.tacc[b];
                        if (v)
                            atomicAdd(reinterpret_cast<unsigned long long*>(
                                          &A.dc[int64_t(cur_g) * kCStride + kOffT + b]), v);
                        s.u2.t.tacc[b] = 0;
                    }
                flush<NT_C>(A, nullptr, nullptr, 0, cur_g, acc, s.red);
            }
            cur_g = g;
        }
        const int k1 = cs.d_k1[j];
        const int32_t* g1mem = h2v + cs.d_hoff[j];
        // g1's members in shared memory for the triple sizes (read after the
        // build's barriers)
        if (k1 <= kG1M)
            for (int t = tid; t < k1; t += NT_C) s.g1m[t] = g1mem[t];
        const int32_t* g1s = k1 <= kG1M ? s.g1m : g1mem;
        const unsigned long long key1 = order_key(k1, g1);
        const int64_t ts1 = TEMP ? S.h_ts[g1] : 0;
        const long long u1 = cs.d_u1[j];
        acc.n_h2v += (tid < k1) ? (k1 - tid + NT_C - 1) / NT_C : 0;
        if (tid == 0) {
            // open paths: N(g1) (sum of member degrees) per pair (h, g1)
            acc.n_open += (unsigned long long)u1 * (unsigned long long)nh_all;
            ++acc.w[0];
            acc.w[1] += (unsigned long long)u1;
        }
        Tab T1;
        int32_t* lk;
        int32_t* pf;
        uint32_t* pm;
        long long* cl;
        int64_t* lts;
        int P = 1;
        // with the temporal family the plus list lives in the block's global
        // scratch (its shared-memory place holds the timestamps of N(g1))
        bool plus_ok = true;
        const uint32_t t1_cap = pow2_at_least(2 * u1);
        if (t1_cap <= min(A.c_smem_cap, uint32_t(T1_S))) {
            T1 = Tab{s.keys, s.vals, nullptr, s.list, &s.n_list, t1_cap - 1, T1_S / 2};
            lk = s.lk;
            pf = TEMP ? g_pf : s.u1.p.pf;
            pm = TEMP ? g_pm : s.u1.p.pm;
            plus_ok = !TEMP || gs / 2 >= int64_t(T1.list_cap);
            cl = s.u2.cl;
            lts = s.u1.lts;
        } else {
            T1 = Tab{g_keys, g_vals, nullptr, g_list, &s.n_list, uint32_t(gs - 1), int(gs / 2)};
            lk = g_lk;
            pf = g_pf;
            pm = g_pm;
            cl = g_cl;
            lts = g_lts;
            if ((int64_t)t1_cap <= gs) T1.mask = t1_cap - 1;
            else P = int((4 * u1 + gs - 1) / gs);
        }
        // filter of N(g1): about 8 bits per entry, at most the array
        int bw = 32;
        while (bw < Sm::BLOOM_W && (long long)bw * 4 < u1 / P) bw <<= 1;
        for (int p = 0; p < P; ++p) {
            // ---- N(g1): x = |g1 & f| per distinct f != g1 (of partition p):
            //      one warp per member, its lanes over the member's hyperedges;
            //      a member of degree >= kBigDeg is left to the whole block
            constexpr int kBigDeg = 256;
            if (tid == 0) s.any_big = 0;
            for (int m0 = 0; m0 < k1; m0 += NT_C) {
                // the segment's members' degrees and v2h offsets, loaded at once
                const int n = min(NT_C, k1 - m0);
                if (tid < n) {
                    const int32_t v = g1mem[m0 + tid];
                    s.seg_pre[tid] = S.v_deg[v];
                    s.seg_off[tid] = S.v_off[v];
                }
                __syncthreads();
                for (int m = wid; m < n; m += NW_C) {
                    const int d = s.seg_pre[m];
                    if (d >= kBigDeg) {
                        if (lane == 0) s.any_big = 1;
                        continue;
                    }
                    const int32_t* lst = v2h + s.seg_off[m];
                    for (int e = lane; e < d; e += 32) {
                        const int32_t f = lst[e];
                        if (f == g1 || (P > 1 && part_of(f, P) != p)) continue;
                        tab_insert(T1, f, 1u, 0, A.sc);
                    }
                    acc.n_v2h += (lane < d) ? (d - lane + 31) / 32 : 0;
                }
                __syncthreads();
            }
            if (s.any_big) {
                for (int m = 0; m < k1; ++m) {
                    const int32_t v = g1mem[m];
                    const int d = S.v_deg[v];
                    if (d < kBigDeg) continue;
                    const int32_t* lst = v2h + S.v_off[v];
                    for (int e = tid; e < d; e += NT_C) {
                        const int32_t f = lst[e];
                        if (f == g1 || (P > 1 && part_of(f, P) != p)) continue;
                        tab_insert(T1, f, 1u, 0, A.sc);
                    }
                    acc.n_v2h += (tid < d) ? (d - tid + NT_C - 1) / NT_C : 0;
                }
                __syncthreads();
            }
            const int n1 = min(s.n_list, T1.list_cap);
            // ---- per f: size and changed flag, the filter, the plus list; in
            //      aggregate mode the totals, the x window and the changed f
            const int wlo = k1 - kWin;
            for (int q0 = 0; q0 < n1; q0 += NT_C) {
                const int q = q0 + tid;
                int wkey = -1, C = 0;
                if (q < n1) {
                    const int sl = T1.list[q];
                    const int32_t f = T1.keys[sl];
                    const int kf = S.h_card[f];
                    const bool changed_f = bit_test(A.chg, f);
                    const int x = int(T1.vals[sl]);
                    lk[q] = kf | (changed_f ? int32_t(0x80000000u) : 0);
                    const uint32_t bb = bloom_bit(f, bw);
                    atomicOr(&s.bloom[bb >> 5], 1u << (bb & 31));
                    if (TEMP) lts[q] = S.h_ts[f];
                    if (plus_ok && order_key(kf, f) > key1) {
                        const int c = atomicAdd(&s.n_plus, 1);
                        pf[c] = f;
                        pm[c] = uint32_t(x) | (uint32_t(kf) << 16) | (changed_f ? 0x80000000u : 0u);
                    }
                    if (agg) {
                        C = kf > x ? 1 : 0;
                        if (x >= wlo && x < k1) wkey = (x - wlo) * 2 + C;
                        if (changed_f) {
                            const int c = atomicAdd(&s.n_cl, 1);
                            cl[c] = (long long)f | ((long long)x << 31) | ((long long)kf << 46);
                        }
                    }
                }
                if (agg) {
                    const unsigned in = __ballot_sync(0xffffffffu, q < n1);
                    const unsigned c1 = __ballot_sync(0xffffffffu, q < n1 && C == 1);
                    if (lane == 0) {
                        if (__popc(in & ~c1)) atomicAdd(&s.tot[0], __popc(in & ~c1));
                        if (__popc(c1)) atomicAdd(&s.tot[1], __popc(c1));
                    }
                    warp_count(&s.win[0][0], wkey);
                }
            }
            acc.n_meta += (tid < n1) ? (n1 - tid + NT_C - 1) / NT_C : 0;
            __syncthreads();
            const int n_plus = s.n_plus;
            const int n_cl = s.n_cl;
            for (int64_t ch = c_beg; ch < c_end; ++ch) {
                const int64_t lbeg = l_lo + ch * LCH;
                const int nh = int(min(lbeg + LCH, l_hi) - lbeg);
                __syncthreads();
                if (wid == 0) {
                    // lane l: the chunk's l-th h, its pass mode and work; the
                    // h with work listed in hord with the prefix of their work
                    // in hpre; the h needing h & g1 listed, and those whose
                    // |h & g1| lies outside the x window
                    const int l = lane;
                    int work = 0, xh1 = 0;
                    if (l < nh) {
                        const int64_t e = lbeg + l;
                        const int32_t li = cs.l_i[e];
                        const uint64_t xv1 = cs.l_xv[e];
                        const int32_t h = A.changed[A.lo + li];
                        xh1 = int(xv1 & kXMask);
                        const int hnn = cs.nh_n[li], htcap = cs.nh_tcap[li];
                        // sorted list: the neighbours above g1 start after g1's place
                        const int hpos = (cs.nh_flag[li] & 1) ? cs.l_q[e] : -1;
                        s.hh[l] = h;
                        s.hk[l] = S.h_card[h];
                        s.hx[l] = xh1;
                        s.hvf[l] = int32_t(uint32_t(xv1 >> 32));
                        s.hmem[l] = h2v + S.h_off[h];
                        s.hnb[l] = cs.nh_off[li] - R.base;
                        s.hnn[l] = hnn;
                        s.htcap[l] = htcap;
                        s.htoff[l] = cs.nh_toff[li];
                        s.hpos[l] = hpos;
                        s.hIn[l] = 0;
                        if (TEMP) s.u2.t.hts[l] = S.h_ts[h];
                        // with the temporal family an N'(h) too long for
                        // k_open_h (flag bit 1) has every pair above g1
                        // visited here, the open ones classified (bit 4 of
                        // the mode)
                        const bool en = TEMP && (cs.nh_flag[li] & 2) != 0;
                        const bool m1ok = plus_ok && !en;
                        int mode;
                        if (hpos >= 0) {
                            const int sfx = hnn - hpos - 1;
                            if (m1ok && htcap > 0 && int64_t(n_plus) * 100 < int64_t(sfx) * cs.m1_pct) {
                                mode = 1;
                                work = n_plus;
                            } else {
                                mode = 0;
                                work = sfx;
                            }
                        } else if (m1ok && htcap > 0) {
                            mode = 1;
                            work = n_plus;
                        } else {
                            mode = 3;
                            work = hnn;
                        }
                        s.hmode[l] = mode | (en ? 16 : 0);
                    }
                    int inc = work;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += v;
                    }
                    const unsigned lt = (1u << lane) - 1u;
                    const unsigned has = __ballot_sync(0xffffffffu, work > 0);
                    if (work > 0) {
                        const int c = __popc(has & lt);
                        s.hord[c] = l;
                        s.hpre[c] = inc - work;
                    }
                    const bool needI = l < nh && xh1 >= 2 && xh1 <= kIC;
                    const bool needX = l < nh && xh1 > kWin;
                    const unsigned bI = __ballot_sync(0xffffffffu, needI);
                    const unsigned bX = __ballot_sync(0xffffffffu, needX);
                    if (needI) s.li_I[__popc(bI & lt)] = l;
                    if (needX) s.li_X[__popc(bX & lt)] = l;
                    if (lane == 31) {
                        s.hpre[__popc(has)] = inc;
                        s.n_c = __popc(has);
                        s.n_li = __popc(bI);
                        s.n_lx = __popc(bX);
                    }
                }
                __syncthreads();
                for (int li = 0; li < s.n_li; ++li) {
                    const int l = s.li_I[li];
                    const int kh = s.hk[l];
                    const bool from_h = kh <= k1;
                    const int32_t* a = from_h ? s.hmem[l] : g1mem;
                    const int32_t* b = from_h ? g1mem : s.hmem[l];
                    const int na = from_h ? kh : k1, nb = from_h ? k1 : kh;
                    for (int i = tid; i < na; i += NT_C) {
                        const int32_t u = a[i];
                        if (contains_sorted(b, nb, u)) {
                            const int c = atomicAdd(&s.hIn[l], 1);
                            if (c < kIC) s.hI[l][c] = u;
                        }
                    }
                }
                if (s.n_li > 0) __syncthreads();
                const int nc = s.n_c;
                const int wtot = s.hpre[nc];
                if (tid == 0) acc.w[2] += (unsigned long long)wtot;
                // each lane holds one h of the pass: its start and index
                const int my_pre = lane < nc ? s.hpre[lane] : INT_MAX;
                const int my_l = lane < nc ? s.hord[lane] : 0;

                // ---- the pair pass: a warp takes 32 consecutive work indices.
                // Closed pairs found go to the warp's queue and are classified
                // 32 at a time, so that every lane of the classifying code is
                // busy (about one visit in ten finds one).
                unsigned long long* const q0 = s.cq0[wid];
                unsigned long long* const q1 = s.cq1[wid];
                auto classify = [&](int e) {
                    const unsigned long long a = q0[e], b = q1[e];
                    const int32_t g2 = int32_t(uint32_t(a));
                    const int32_t vf2 = int32_t(uint32_t(a >> 32));
                    const int x12 = int(b & 0xffffu), xh2 = int((b >> 16) & 0xffffu);
                    const int k2 = int((b >> 32) & 0x7fffu), l = int(b >> 48);
                    const int kh = s.hk[l], xh1 = s.hx[l];
                    ++acc.w[3];
                    const int t = triple_size_o(xh1, s.hvf[l], xh2, vf2, g1s, k1, h2v + S.h_off[g2], k2, s.hmem[l],
                                                kh, s.hI[l], s.hIn[l], acc.w[4]);
                    acc.n_meta += 1;
                    acc.n_closed += (unsigned long long)min(k1, k2);  // closed pairs: min(|g1|, |g2|) entries
                    const int ra = kh - xh1 - xh2 + t, rb = k1 - xh1 - x12 + t, rc = k2 - x12 - xh2 + t;
                    const int mk = (ra > 0) | ((rb > 0) << 1) | ((rc > 0) << 2) | ((xh1 - t > 0) << 3) |
                                   ((x12 - t > 0) << 4) | ((xh2 - t > 0) << 5) | ((t > 0) << 6);
                    // the open classes the open-triad counts gave this triple:
                    // centred at g1 (f = g2) and at g2 (f = g1), and, when
                    // those at h are counted in aggregate, centred at h
                    const int m1 = (kh > xh1 ? 1 : 0) | (x12 != k1 - xh1 ? 2 : 0) | (k2 > x12 ? 4 : 0) | 8 | 16;
                    const int m2 = (kh > xh2 ? 1 : 0) | (x12 != k2 - xh2 ? 2 : 0) | (k1 > x12 ? 4 : 0) | 8 | 16;
                    ++acc.n_tri;
                    if (want_h) {
                        // every mask formed here is a valid triad (its pairwise
                        // intersections are non-empty), so each class is >= 0
                        const int cc = s.tb.cls30[mk];
                        const int c1 = s.tb.cls30[m1], c2 = s.tb.cls30[m2];
                        if (cc >= 0) atomicAdd(&hist[cc], 1u);
                        const int ch = s.tb.cls30[open_at_h_mask(kh, xh1, xh2, k1, k2)];
                        if (ch >= 0) atomicAdd(&hneg[ch], 1u);
                        if (c1 >= 0) atomicAdd(&hneg[c1], 1u);
                        if (c2 >= 0) atomicAdd(&hneg[c2], 1u);
                    }
                    if constexpr (TEMP) {
                        const int32_t h = s.hh[l];
                        const int64_t th = s.u2.t.hts[l], t2 = S.h_ts[g2];
                        const int cc = temporal_class(s.tb, mk, th, ts1, t2, h, g1, g2, delta);
                        const int p1 = temporal_class(s.tb, m1, th, ts1, t2, h, g1, g2, delta);
                        const int p2 = temporal_class(s.tb, m2, th, t2, ts1, h, g2, g1, delta);
                        if (cc >= 0) atomicAdd(&s.u2.t.th[wid][cc], 1u);
                        if (p1 >= 0) atomicAdd(&s.u2.t.tn[p1], 1u);
                        if (p2 >= 0) atomicAdd(&s.u2.t.tn[p2], 1u);
                        if (!(s.hmode[l] & 16)) {  // the open class k_open_h gave it at h
                            const int p0 = temporal_class(s.tb, open_at_h_mask(kh, xh1, xh2, k1, k2), th, ts1, t2, h,
                                                          g1, g2, delta);
                            if (p0 >= 0) atomicAdd(&s.u2.t.tn[p0], 1u);
                        }
                    }
                    if (fam & kFamV)
                        acc.v3 += (unsigned long long)xh1 * x12 * xh2 - (unsigned long long)t * (xh1 + x12 + xh2) +
                                  2ull * t;
                };
                int qn = 0;  // the warp's queue length (the same in every lane)
                const unsigned lt = (1u << lane) - 1u;
                for (int w0 = wid * 32; w0 < wtot; w0 += NT_C) {
                    const int idx = w0 + lane;
                    // the h of each index: the last one starting at or before it
                    const unsigned le = __ballot_sync(0xffffffffu, my_pre <= w0);
                    const int c0 = 31 - __clz(le);
                    const unsigned bnd = (my_pre > w0 && my_pre < w0 + 32) ? 1u << (my_pre - w0) : 0u;
                    const unsigned B = __reduce_or_sync(0xffffffffu, bnd);
                    const int c = c0 + __popc(B & ((2u << lane) - 1u));
                    const int l = __shfl_sync(0xffffffffu, my_l, c & 31);
                    const int q = idx - __shfl_sync(0xffffffffu, my_pre, c & 31);
                    bool found = false;
                    unsigned long long e0 = 0, e1 = 0;
                    do {
                    if (idx >= wtot) break;
                    const int mode = s.hmode[l] & 15;
                    int32_t g2;
                    int x12, xh2, k2;
                    int32_t vf2;
                    bool chg2;
                    if (mode == 1) {
                        g2 = pf[q];
                        const uint32_t tcap = uint32_t(s.htcap[l]);
                        uint32_t bits;
                        const uint32_t fw = reinterpret_cast<const uint32_t*>(
                            cs.nh_g + s.htoff[l] + tcap)[filter_word(g2, tcap, bits)];
                        if ((fw & bits) != bits) break;
                        const int ps = probe_list_table(cs.nh_g + s.htoff[l], tcap - 1, g2);
                        if (ps < 0) break;
                        const uint64_t xv2 = cs.nh_xv[s.htoff[l] + ps];
                        const uint32_t m = pm[q];
                        x12 = int(m & 0xffffu);
                        k2 = int((m >> 16) & 0x7fffu);
                        chg2 = (m >> 31) != 0;
                        xh2 = int(uint32_t(xv2) & kXMask);
                        vf2 = int32_t(uint32_t(xv2 >> 32));
                    } else if (TEMP && (s.hmode[l] & 16)) {
                        // every g2 of N'(h) above g1: closed pairs queued, open
                        // ones (centred at h) get their temporal class here (the
                        // static one is counted in aggregate by k_nh_build)
                        const int64_t at = s.hnb[l] + (mode == 0 ? s.hpos[l] + 1 + q : q);
                        g2 = cs.nh_g[at];
                        const uint64_t xv2 = cs.nh_xv[at];
                        k2 = int((xv2 >> 16) & 0x7fffu);
                        if (mode == 3 && order_key(k2, g2) <= key1) break;
                        chg2 = ((xv2 >> 31) & 1u) != 0;
                        const int32_t h = s.hh[l];
                        if (g2 < h && chg2) break;  // the triple belongs to g2 (or a smaller changed member)
                        if (P > 1 && part_of(g2, P) != p) break;
                        xh2 = int(xv2 & kXMask);
                        vf2 = int32_t(uint32_t(xv2 >> 32));
                        const uint32_t bb = bloom_bit(g2, bw);
                        const int sl = ((s.bloom[bb >> 5] >> (bb & 31)) & 1u) ? tab_find(T1, g2) : -1;
                        if (sl < 0) {
                            const int m = open_at_h_mask(s.hk[l], s.hx[l], xh2, k1, k2);
                            ++acc.n_tri;
                            const int c96 = temporal_class(s.tb, m, s.u2.t.hts[l], ts1, cs.nh_ts[at], h, g1, g2, delta);
                            if (c96 >= 0) atomicAdd(&s.u2.t.th[wid][c96], 1u);
                            break;
                        }
                        x12 = int(T1.vals[sl]);
                    } else {
                        const int64_t at = s.hnb[l] + (mode == 0 ? s.hpos[l] + 1 + q : q);
                        g2 = cs.nh_g[at];
                        uint64_t xv2 = 0;
                        if (mode == 3) {
                            xv2 = cs.nh_xv[at];
                            if (order_key(int((xv2 >> 16) & 0x7fffu), g2) <= key1) break;
                        }
                        if (P > 1 && part_of(g2, P) != p) break;
                        const uint32_t bb = bloom_bit(g2, bw);
                        if (!((s.bloom[bb >> 5] >> (bb & 31)) & 1u)) break;
                        const int sl = tab_find(T1, g2);
                        if (sl < 0) break;
                        if (mode != 3) xv2 = cs.nh_xv[at];
                        x12 = int(T1.vals[sl]);
                        xh2 = int(xv2 & kXMask);
                        k2 = int((xv2 >> 16) & 0x7fffu);
                        chg2 = ((xv2 >> 31) & 1u) != 0;
                        vf2 = int32_t(uint32_t(xv2 >> 32));
                    }
                    // a closed triad {h, g1, g2}, g1 below g2, unless it
                    // belongs to g2 (or a smaller changed member)
                    if (g2 < s.hh[l] && chg2) break;
                    found = true;
                    e0 = uint64_t(uint32_t(g2)) | (uint64_t(uint32_t(vf2)) << 32);
                    e1 = uint64_t(x12) | (uint64_t(xh2) << 16) | (uint64_t(k2) << 32) | (uint64_t(l) << 48);
                    } while (0);
                    const unsigned fm = __ballot_sync(0xffffffffu, found);
                    if (fm) {
                        if (found) {
                            const int at = qn + __popc(fm & lt);
                            q0[at] = e0;
                            q1[at] = e1;
                        }
                        qn += __popc(fm);
                        if (qn >= 32) {
                            __syncwarp();
                            classify(qn - 32 + lane);
                            qn -= 32;
                            __syncwarp();
                        }
                    }
                }
                __syncwarp();
                if (lane < qn) classify(lane);
                __syncthreads();
                if constexpr (TEMP) {
                    // open triads {h, g1, f} centred at g1: f in N(g1), f != h,
                    // f not a changed hyperedge of smaller ID than h (its triads
                    // belong to f).  Their class is set by A = [h not inside g1],
                    // the bucket 2B + C of f (B = [|g1&f| != |g1| - |h&g1|],
                    // C = [f not inside g1]) and, for the temporal family, by
                    // where f falls in time against h and g1 and whether the
                    // triple fits the window; a warp per h counts its f by
                    // (position, bucket).  Those f that meet h (closed triples)
                    // are taken back when their closed pair is classified.
                    if (nh < kSweepMin) {
                        if (tid == 0) acc.w[5] += (unsigned long long)nh * n1;
                        for (int l = wid; l < nh; l += NW_C) {
                            const int32_t h = s.hh[l];
                            const int xh1 = s.hx[l], xstar = k1 - xh1;
                            const int64_t th = s.u2.t.hts[l];
                            const bool h_first = th < ts1 || (th == ts1 && h < g1);
                            const int64_t tp = h_first ? th : ts1, tq = h_first ? ts1 : th;
                            const int32_t ip = h_first ? h : g1, iq = h_first ? g1 : h;
                            uint32_t cst[4] = {0, 0, 0, 0};
                            uint32_t ctm[3][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
                            for (int q = lane; q < n1; q += 32) {
                                const int sl = T1.list[q];
                                const int32_t f = T1.keys[sl];
                                if (f == h) continue;
                                const int32_t meta = lk[q];
                                if (meta < 0 && f < h) continue;
                                const int x = int(T1.vals[sl]);
                                const int b = (x != xstar ? 2 : 0) | ((meta & 0x7fffffff) > x ? 1 : 0);
                                const int64_t tf = lts[q];
                                int r;  // position in time, -1: outside the window
                                if (tf < tp || (tf == tp && f < ip)) r = tq - tf <= delta ? 0 : -1;
                                else if (tf < tq || (tf == tq && f < iq)) r = tq - tp <= delta ? 1 : -1;
                                else r = tf - tp <= delta ? 2 : -1;
                                // constant indices keep the counters in registers
    #pragma unroll
                                for (int bb = 0; bb < 4; ++bb) {
                                    cst[bb] += b == bb ? 1u : 0u;
    #pragma unroll
                                    for (int rr = 0; rr < 3; ++rr) ctm[rr][bb] += (b == bb && r == rr) ? 1u : 0u;
                                }
                            }
    #pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
    #pragma unroll
                                for (int b = 0; b < 4; ++b) {
                                    cst[b] += __shfl_xor_sync(0xffffffffu, cst[b], o);
    #pragma unroll
                                    for (int r = 0; r < 3; ++r) ctm[r][b] += __shfl_xor_sync(0xffffffffu, ctm[r][b], o);
                                }
                            }
                            if (lane == 0) {
                                const int A_bit = s.hk[l] > xh1 ? 1 : 0;
                                // labels 0 = h, 1 = g1, 2 = f; p and q are h and g1 in time order
                                const int lp = h_first ? 0 : 1, lq = h_first ? 1 : 0;
                                for (int b = 0; b < 4; ++b) {
                                    const int m = A_bit | ((b >> 1) << 1) | ((b & 1) << 2) | (1 << 3) | (1 << 4);
                                    acc.n_tri += cst[b];
                                    if (want_h && cst[b] && s.tb.cls30[m] >= 0) atomicAdd(&hist[s.tb.cls30[m]], cst[b]);
                                    for (int r = 0; r < 3; ++r) {
                                        if (!ctm[r][b]) continue;
                                        const int o0 = r == 0 ? 2 : lp, o1 = r == 0 ? lp : (r == 1 ? 2 : lq);
                                        const int c = s.tb.cls96[s.tb.perm[perm_index(o0, o1)][m]];
                                        if (c >= 0) atomicAdd(&s.u2.t.th[wid][c], ctm[r][b]);
                                    }
                                }
                            }
                        }
                    } else {
                        // The chunk's h sorted by (t, ID) and by (|h & g1|, t,
                        // ID); each f of N(g1) then adds one to a few
                        // contiguous ranges of h in those orders (difference
                        // arrays by time position r and C): where f falls
                        // against h and g1 and whether the window holds are
                        // monotone in th.  The ranges of the x-order cover the
                        // h with |h & g1| = |g1| - |g1 & f|, for which B = 0.
                        // A changed f is taken per h (it counts only for h < f).
                        if (tid == 0) acc.w[5] += (unsigned long long)n1;
                        auto& T = s.u2.t;
                        if (wid == 0) {
                            const bool in = lane < nh;
                            const int64_t tl = in ? T.hts[lane] : 0;
                            const int32_t il = in ? s.hh[lane] : 0;
                            const int xl = in ? s.hx[lane] : 0;
                            int rt = 0, rx = 0;
                            for (int m = 0; m < nh; ++m) {
                                const int64_t tm = T.hts[m];
                                const int32_t im = s.hh[m];
                                const int xm = s.hx[m];
                                const bool lt = tm < tl || (tm == tl && im < il);
                                rt += lt ? 1 : 0;
                                rx += (xm < xl || (xm == xl && lt)) ? 1 : 0;
                            }
                            if (in) {
                                T.ot_t[rt] = tl;
                                T.ot_i[rt] = il;
                                T.pt[lane] = rt;
                                T.ox_t[rx] = tl;
                                T.ox_i[rx] = il;
                                T.ox_x[rx] = xl;
                                T.px[lane] = rx;
                            }
                            const unsigned bef = __ballot_sync(0xffffffffu, in && (tl < ts1 || (tl == ts1 && il < g1)));
                            if (lane == 0) T.n_before = __popc(bef);
                            // where each small x starts and ends in the x order
                            for (int x = lane; x < kXG; x += 32) {
                                int lo = 0, hi = 0;
                                for (int m = 0; m < nh; ++m) {
                                    lo += s.hx[m] < x ? 1 : 0;
                                    hi += s.hx[m] <= x ? 1 : 0;
                                }
                                T.xg[0][x] = uint8_t(lo);
                                T.xg[1][x] = uint8_t(hi);
                            }
                        }
                        for (int i = tid; i < 8 * (LCH + 1); i += NT_C) {
                            (&T.dT[0][0])[i] = 0;
                            (&T.dX[0][0])[i] = 0;
                        }
                        __syncthreads();
                        const int s1 = T.n_before;
                        // counts at the places every f meets in the (t, ID)
                        // order -- 0 and s1 -- are kept per thread and added
                        // once (the end nh needs nothing: no prefix reads it)
                        int at0[8] = {0, 0, 0, 0, 0, 0, 0, 0}, ats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                        // a warp takes 32 consecutive f; a changed f is taken by the
                        // whole warp at once, a lane per h (a lane looping over
                        // the chunk's h alone would hold its warp)
                        for (int q0 = wid * 32; q0 < n1; q0 += NT_C) {
                            const int q = q0 + lane;
                            const bool act = q < n1;
                            int32_t f = 0, meta = 0;
                            int x = 0, C = 0;
                            int64_t tf = 0;
                            if (act) {
                                const int sl = T1.list[q];
                                f = T1.keys[sl];
                                meta = lk[q];
                                x = int(T1.vals[sl]);
                                C = (meta & 0x7fffffff) > x ? 1 : 0;
                                tf = lts[q];
                            }
                            for (unsigned chm = __ballot_sync(0xffffffffu, act && meta < 0); chm; chm &= chm - 1) {
                                const int b = __ffs(chm) - 1;
                                const int32_t fc = __shfl_sync(0xffffffffu, f, b);
                                const int xc = __shfl_sync(0xffffffffu, x, b), cc = __shfl_sync(0xffffffffu, C, b);
                                const int64_t tc = __shfl_sync(0xffffffffu, tf, b);
                                if (lane < nh) {
                                    const int32_t h = s.hh[lane];
                                    // f = h, or a changed f < h: its triads belong to f
                                    if (fc > h) {
                                        const int xh1 = s.hx[lane];
                                        const int m = (s.hk[lane] > xh1 ? 1 : 0) | (xc != k1 - xh1 ? 2 : 0) | (cc << 2) |
                                                      8 | 16;
                                        ++acc.n_tri;
                                        if (want_h) {
                                            const int c = s.tb.cls30[m];
                                            if (c >= 0) atomicAdd(&hist[c], 1u);
                                        }
                                        const int c96 = temporal_class(s.tb, m, T.hts[lane], ts1, tc, h, g1, fc, delta);
                                        if (c96 >= 0) atomicAdd(&T.th[wid][c96], 1u);
                                    }
                                }
                            }
                            if (!act || meta < 0) continue;
                            const bool fb = tf < ts1 || (tf == ts1 && f < g1);
                            // places in [lo, hi) of an order: the first not before
                            // (t, id); the first at time >= t; the first at time > t
                            auto first_not_before = [](const int64_t* ta, const int32_t* ia, int lo, int hi, int64_t t,
                                                       int32_t id) {
                                while (lo < hi) {
                                    const int mid = (lo + hi) >> 1;
                                    if (ta[mid] < t || (ta[mid] == t && ia[mid] < id)) lo = mid + 1;
                                    else hi = mid;
                                }
                                return lo;
                            };
                            auto first_ge = [](const int64_t* ta, int lo, int hi, int64_t t) {
                                while (lo < hi) {
                                    const int mid = (lo + hi) >> 1;
                                    if (ta[mid] < t) lo = mid + 1;
                                    else hi = mid;
                                }
                                return lo;
                            };
                            auto first_gt = [](const int64_t* ta, int lo, int hi, int64_t t) {
                                while (lo < hi) {
                                    const int mid = (lo + hi) >> 1;
                                    if (ta[mid] <= t) lo = mid + 1;
                                    else hi = mid;
                                }
                                return lo;
                            };
                            // the h of [lo, hi) (split: the first after g1) that f
                            // meets at each time position r within the window
                            auto ranges = [&](int32_t (*d)[LCH + 1], const int64_t* ta, const int32_t* ia, int lo, int hi,
                                              int split) {
                                const bool t_order = d == T.dT;
                                auto add = [&](int r, int a, int b) {
                                    if (a >= b) return;
                                    const int k = r * 2 + C;
#pragma unroll
                                    for (int kk = 0; kk < 8; ++kk)
                                        if (kk == k) {
                                            if (t_order && a == 0) ++at0[kk];
                                            else if (t_order && a == s1) ++ats[kk];
                                            else atomicAdd(&d[kk][a], 1);
                                            if (t_order && b == s1) --ats[kk];
                                            else if (!(t_order && b == nh)) atomicAdd(&d[kk][b], -1);
                                        }
                                };
                                const int pos = first_not_before(ta, ia, lo, hi, tf, f);
                                if (fb) {  // f before g1
                                    if (ts1 - tf <= delta) add(0, pos, split);               // h before g1, after f
                                    add(1, first_ge(ta, lo, hi, sat_sub(ts1, delta)), pos);   // h before f, th >= ts1 - delta
                                    add(0, split, max(split, first_gt(ta, lo, hi, sat_add(tf, delta))));  // h after g1, th <= tf + delta
                                } else {   // f after g1
                                    add(2, first_ge(ta, lo, hi, sat_sub(tf, delta)), split);  // h before g1, th >= tf - delta
                                    add(1, pos, max(pos, first_gt(ta, lo, hi, sat_add(ts1, delta))));  // h after f, th <= ts1 + delta
                                    if (tf - ts1 <= delta) add(2, split, pos);               // h after g1, before f
                                }
                                add(3, lo, hi);  // static classes: every h
                            };
                            ranges(T.dT, T.ot_t, T.ot_i, 0, nh, s1);
                            const int xs = k1 - x;
                            int ga = 0, gb = nh;  // the h with |h & g1| = xs
                            if (xs >= 0 && xs < kXG) {
                                ga = T.xg[0][xs];
                                gb = T.xg[1][xs];
                            } else {
                                int lo = 0, hi = nh;
                                while (lo < hi) {
                                    const int mid = (lo + hi) >> 1;
                                    if (T.ox_x[mid] < xs) lo = mid + 1;
                                    else hi = mid;
                                }
                                ga = lo;
                                hi = nh;
                                while (lo < hi) {
                                    const int mid = (lo + hi) >> 1;
                                    if (T.ox_x[mid] <= xs) lo = mid + 1;
                                    else hi = mid;
                                }
                                gb = lo;
                            }
                            if (ga < gb)
                                ranges(T.dX, T.ox_t, T.ox_i, ga, gb, first_not_before(T.ox_t, T.ox_i, ga, gb, ts1, g1));
                        }
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            int a = at0[k], b = ats[k];
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                a += __shfl_xor_sync(0xffffffffu, a, o);
                                b += __shfl_xor_sync(0xffffffffu, b, o);
                            }
                            if (lane == 0) {
                                if (a) atomicAdd(&T.dT[k][0], a);
                                if (b) atomicAdd(&T.dT[k][s1], b);
                            }
                        }
                        __syncthreads();
                        if (tid < 16) {  // inclusive prefix sums: the ranges holding each place
                            int32_t* d = tid < 8 ? T.dT[tid] : T.dX[tid - 8];
                            int run = 0;
                            for (int i = 0; i < nh; ++i) {
                                run += d[i];
                                d[i] = run;
                            }
                        }
                        __syncthreads();
                        if (wid == 0 && lane < nh) {
                            const int l = lane;
                            const int xh1 = s.hx[l];
                            const int A_bit = s.hk[l] > xh1 ? 1 : 0;
                            const bool h_first = T.hts[l] < ts1 || (T.hts[l] == ts1 && s.hh[l] < g1);
                            // labels 0 = h, 1 = g1, 2 = f; p and q are h and g1 in time order
                            const int lp = h_first ? 0 : 1, lq = h_first ? 1 : 0;
                            const int ptl = T.pt[l], pxl = T.px[l];
                            for (int r = 0; r < 4; ++r)
                                for (int C = 0; C < 2; ++C) {
                                    const int n_all = T.dT[r * 2 + C][ptl], n_b0 = T.dX[r * 2 + C][pxl];
                                    for (int B = 0; B < 2; ++B) {
                                        const int n = B ? n_all - n_b0 : n_b0;
                                        if (n <= 0) continue;
                                        const int m = A_bit | (B << 1) | (C << 2) | (1 << 3) | (1 << 4);
                                        if (r == 3) {
                                            acc.n_tri += (unsigned long long)n;
                                            const int c = s.tb.cls30[m];
                                            if (want_h && c >= 0) atomicAdd(&hist[c], uint32_t(n));
                                        } else {
                                            const int o0 = r == 0 ? 2 : lp, o1 = r == 0 ? lp : (r == 1 ? 2 : lq);
                                            const int c = s.tb.cls96[s.tb.perm[perm_index(o0, o1)][m]];
                                            if (c >= 0) atomicAdd(&T.th[wid][c], uint32_t(n));
                                        }
                                    }
                                }
                        }
                    }
                }
                if (agg) {
                    // open triads {h, g1, f} centred at g1, in aggregate: the
                    // class is set by A = [h not inside g1] and the bucket
                    // b = 2B + C of f, B = [|g1&f| != |g1| - |h&g1|],
                    // C = [f not inside g1]; from the totals over N(g1) are
                    // taken f = h and the changed f < h
                    if (tid == 0) acc.w[5] += (unsigned long long)nh * n_cl;
                    for (int l = wid; l < nh; l += NW_C) {  // a warp per h, its lanes over the changed f
                        const int32_t h = s.hh[l];
                        const int xs = k1 - s.hx[l];
                        uint32_t nb[4] = {0, 0, 0, 0};
                        for (int c0 = 0; c0 < n_cl; c0 += 32) {
                            int b = -1;
                            if (c0 + lane < n_cl) {
                                const long long v = cl[c0 + lane];
                                if (int32_t(v & 0x7fffffffll) < h) {
                                    const int x = int((v >> 31) & 0x7fffll), kf = int(v >> 46);
                                    b = (x != xs ? 2 : 0) | (kf > x ? 1 : 0);
                                }
                            }
#pragma unroll
                            for (int bb = 0; bb < 4; ++bb) nb[bb] += __popc(__ballot_sync(0xffffffffu, b == bb));
                        }
                        if (lane == 0)
                            for (int bb = 0; bb < 4; ++bb)
                                if (nb[bb]) atomicAdd(&s.sub[l][bb], nb[bb]);
                    }
                    if (tid < nh && (P == 1 || part_of(s.hh[tid], P) == p)) {
                        const int xh1 = s.hx[tid];
                        atomicAdd(&s.sub[tid][(xh1 != k1 - xh1 ? 2 : 0) | (s.hk[tid] > xh1 ? 1 : 0)], 1u);
                    }
                    for (int lx = 0; lx < s.n_lx; ++lx) {  // x = |g1| - |h&g1| outside the window
                        const int l = s.li_X[lx];
                        const int xstar = k1 - s.hx[l];
                        for (int q = tid; q < n1; q += NT_C)
                            if (int(T1.vals[T1.list[q]]) == xstar)
                                atomicAdd(&s.xc[l][(lk[q] & 0x7fffffff) > xstar ? 1 : 0], 1u);
                    }
                    __syncthreads();
                    if (tid < nh) {
                        const int xh1 = s.hx[tid], kh = s.hk[tid];
                        const int A_bit = kh > xh1 ? 1 : 0;
                        for (int b = 0; b < 4; ++b) {
                            const int B = b >> 1, C = b & 1;
                            const uint32_t h0 = xh1 <= kWin ? s.win[kWin - xh1][C] : s.xc[tid][C];
                            const uint32_t total = B == 0 ? h0 : s.tot[C] - h0;
                            const uint32_t n = total - s.sub[tid][b];
                            if (n) {
                                const int m = A_bit | (B << 1) | (C << 2) | (1 << 3) | (1 << 4);
                                atomicAdd(&hist[s.tb.cls30[m]], n);
                                acc.n_tri += n;
                            }
                            s.sub[tid][b] = 0;
                        }
                        s.xc[tid][0] = s.xc[tid][1] = 0;
                    }
                }
            }  // chunks
            __syncthreads();
            tab_clear<NT_C>(T1, n1);
            for (int i = tid; i < bw; i += NT_C) s.bloom[i] = 0;
            if (agg) {
                if (tid < 2) s.tot[tid] = 0;
                for (int i = tid; i < kWin * 2; i += NT_C) s.win[i >> 1][i & 1] = 0;
            }
            __syncthreads();
            if (tid == 0) {
                s.n_list = 0;
                s.n_plus = 0;
                s.n_cl = 0;
            }
        }
        // fold the warp histograms of this item
        for (int b = tid; b < kNH; b += NT_C) {
            unsigned long long v = 0;
            for (int w = 0; w < NW_C; ++w) {
                v += s.hist[w][b];
                v -= s.hneg[w][b];
                s.hist[w][b] = 0;
                s.hneg[w][b] = 0;
            }
            s.acc[b] += v;
        }
        if constexpr (TEMP)
            for (int b = tid; b < kNT; b += NT_C) {
                unsigned long long v = 0;
                for (int w = 0; w < NW_C; ++w) {
                    v += s.u2.t.th[w][b];
                    s.u2.t.th[w][b] = 0;
                }
                v -= s.u2.t.tn[b];
                s.u2.t.tn[b] = 0;
                s.u2.t.tacc[b] += v;
            }
    }
    __syncthreads();
    if (cur_g >= 0) {
        for (int b = tid; b < kNH; b += NT_C) {
            unsigned long long v = s.acc[b];
            if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&A.dc[int64_t(cur_g) * kCStride + b]), v);
            s.acc[b] = 0;
        }
        if constexpr (TEMP)
            for (int b = tid; b < kNT; b += NT_C) {
                unsigned long long v = s.u2.t.tacc[b];
                if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&A.dc[int64_t(cur_g) * kCStride + kOffT + b]), v);
                s.u2.t.tacc[b] = 0;
            }
        flush<NT_C>(A, nullptr, nullptr, 0, cur_g, acc, s.red);
    }
    flush_stats<NT_C>(A, acc, s.red);
}

// ---------------------------------------------------------------------------
// scans: host-known length, and device-known length (read from a counter)
// ---------------------------------------------------------------------------

constexpr int kScanNT = 1024, kScanPer = 4, kScanBlock = kScanNT * kScanPer;

template <typename In>
__global__ void k_scan_sums(const In* in, int64_t n_host, const int32_t* n_dev, int64_t* sums) {
    __shared__ int64_t red[kScanNT / 32];
    const int64_t n = n_dev ? *n_dev : n_host;
    const int64_t base = int64_t(blockIdx.x) * kScanBlock;
    if (base >= n && blockIdx.x > 0) return;
    int64_t v = 0;
    for (int k = 0; k < kScanPer; ++k) {
        int64_t i = base + int64_t(threadIdx.x) * kScanPer + k;
        if (i < n) v += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kScanNT / 32; ++w) t += red[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void k_scan_top(int64_t* sums, int64_t nb_host, const int32_t* n_dev) {
    if (threadIdx.x != 0) return;
    int64_t nb = nb_host;
    if (n_dev) {
        nb = (int64_t(*n_dev) + kScanBlock - 1) / kScanBlock;
        if (nb < 1) nb = 1;
    }
    int64_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t v = sums[b];
        sums[b] = run;
        run += v;
    }
}

template <typename In>
__global__ void k_scan_apply(const In* in, int64_t n_host, const int32_t* n_dev, const int64_t* sums, int64_t* out) {
    __shared__ int64_t wsum[kScanNT / 32];
    const int64_t n = n_dev ? *n_dev : n_host;
    const int64_t base = int64_t(blockIdx.x) * kScanBlock;
    if (n == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
        return;
    }
    if (base >= n) return;
    int64_t loc[kScanPer];
    int64_t v = 0;
    for (int k = 0; k < kScanPer; ++k) {
        int64_t i = base + int64_t(threadIdx.x) * kScanPer + k;
        loc[k] = v;
        if (i < n) v += in[i];
    }
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane_id() >= o) x += y;
    }
    if (lane_id() == 31) wsum[warp_id()] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t w = threadIdx.x < kScanNT / 32 ? wsum[threadIdx.x] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane_id() >= o) w += y;
        }
        if (threadIdx.x < kScanNT / 32) wsum[threadIdx.x] = w;
    }
    __syncthreads();
    int64_t pre = sums[blockIdx.x] + (warp_id() > 0 ? wsum[warp_id() - 1] : 0) + x - v;
    for (int k = 0; k < kScanPer; ++k) {
        int64_t i = base + int64_t(threadIdx.x) * kScanPer + k;
        if (i < n) out[i] = pre + loc[k];
        if (i == n - 1) out[n] = pre + loc[k] + in[i];
    }
}

__global__ void k_run_begin(Scalars* sc, int side) {
    sc->r_used[side] = 0;
    sc->qnh[side] = 0;
    sc->qoh[side] = 0;
    sc->qos[side] = 0;
    sc->queue[side] = 0;
    sc->n_d[side] = 0;
    sc->items[side] = 0;
}

inline unsigned blocks_for(int64_t n, int per) {
    int64_t b = (n + per - 1) / per;
    return unsigned(b < 1 ? 1 : b);
}

inline unsigned capped(unsigned b) { return b < 4096u ? b : 4096u; }

}  // namespace

size_t count_scratch_bytes(const CountShape& sh) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t b = 0;
    const int64_t nbs = (std::max(sh.cap, sh.e_cap) + kScanBlock - 1) / kScanBlock + 2;
    b += al(sizeof(int32_t) * sh.cap) + al(sizeof(int64_t) * (sh.cap + 1)) + al(sizeof(int32_t) * sh.cap);
    b += al(sizeof(int64_t) * sh.cap) + al(sizeof(int32_t) * sh.cap);
    b += al(sizeof(uint32_t) * sh.n_cta_nh * 2 * (kMaxCard + 1));
    b += 2 * (al(sizeof(int32_t) * sh.list_cap) + al(sizeof(uint64_t) * sh.list_cap));
    b += al(sizeof(int32_t) * sh.list_cap) + al(sizeof(int32_t) * sh.cap);
    b += sh.with_ts ? al(sizeof(int64_t) * sh.list_cap) : 0;
    b += 2 * al(sizeof(int32_t) * sh.e_cap) + al(sizeof(int64_t) * sh.e_cap);
    b += 3 * al(sizeof(int32_t) * sh.e_cap) + 2 * al(sizeof(int64_t) * (sh.e_cap + 1));
    b += al(sizeof(int64_t) * nbs);
    b += al(sizeof(int32_t) * sh.e_cap) + 2 * al(sizeof(int64_t) * sh.e_cap) +
         al(sizeof(int32_t) * (sh.e_cap + sh.list_cap / (LCH * kSuper) + 1));
    b += al(sizeof(int32_t) * sh.r_cap) + al(sizeof(int64_t) * sh.cap);
    b += 2 * al(sizeof(int32_t) * sh.cap) + al(sizeof(int64_t) * (sh.cap + 1));
    const int64_t rn = sh.n_cta_nh, rc = int64_t(sh.c_per_sm) * sh.n_cta_c;
    b += 3 * al(sizeof(int32_t) * rn * sh.gs_nh) + al(sizeof(int32_t) * rn * (sh.gs_nh / 2));
    b += 3 * al(sizeof(int32_t) * rc * sh.gs_c) + 5 * al(sizeof(int32_t) * rc * (sh.gs_c / 2)) +
         al(sizeof(int64_t) * rc * (sh.gs_c / 2));
    const int64_t oh = open_h_cap(sh);
    if (oh > 0) {
        const size_t nb = size_t(sh.n_cta_c) * size_t(oh + 1);
        b += al(sizeof(int64_t) * nb) + 5 * al(sizeof(int32_t) * nb);
    }
    return b + 4096;
}

cudaError_t count_scratch_init(CountScratch* cs, void* mem, const CountShape& sh, int64_t* pinned_word,
                               cudaStream_t st) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    char* p = static_cast<char*>(mem);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        void* r = p + o;
        o += al(bytes);
        return r;
    };
    const int64_t nbs = (std::max(sh.cap, sh.e_cap) + kScanBlock - 1) / kScanBlock + 2;
    cs->cap = sh.cap;
    cs->list_cap = sh.list_cap;
    cs->e_cap = sh.e_cap;
    cs->gs_nh = sh.gs_nh;
    cs->gs_c = sh.gs_c;
    cs->n_cta_nh = sh.n_cta_nh;
    cs->n_cta_c = sh.n_cta_c;
    cs->sizes = static_cast<int32_t*>(take(sizeof(int32_t) * sh.cap));
    cs->nh_off = static_cast<int64_t*>(take(sizeof(int64_t) * (sh.cap + 1)));
    cs->nh_n = static_cast<int32_t*>(take(sizeof(int32_t) * sh.cap));
    cs->nh_toff = static_cast<int64_t*>(take(sizeof(int64_t) * sh.cap));
    cs->nh_tcap = static_cast<int32_t*>(take(sizeof(int32_t) * sh.cap));
    cs->onh_hist = static_cast<uint32_t*>(take(sizeof(uint32_t) * sh.n_cta_nh * 2 * (kMaxCard + 1)));
    cs->nh_g = static_cast<int32_t*>(take(sizeof(int32_t) * sh.list_cap));
    cs->nh_xv = static_cast<uint64_t*>(take(sizeof(uint64_t) * sh.list_cap));
    cs->nh_ts = sh.with_ts ? static_cast<int64_t*>(take(sizeof(int64_t) * sh.list_cap)) : nullptr;
    cs->l_i = static_cast<int32_t*>(take(sizeof(int32_t) * sh.list_cap));
    cs->l_xv = static_cast<uint64_t*>(take(sizeof(uint64_t) * sh.list_cap));
    cs->l_q = static_cast<int32_t*>(take(sizeof(int32_t) * sh.list_cap));
    cs->nh_flag = static_cast<int32_t*>(take(sizeof(int32_t) * sh.cap));
    cs->lcnt = static_cast<int32_t*>(take(sizeof(int32_t) * sh.e_cap));
    cs->lfill = static_cast<int32_t*>(take(sizeof(int32_t) * sh.e_cap));
    cs->loffg = static_cast<int64_t*>(take(sizeof(int64_t) * sh.e_cap));
    cs->d_list = static_cast<int32_t*>(take(sizeof(int32_t) * sh.e_cap));
    cs->d_cnt = static_cast<int32_t*>(take(sizeof(int32_t) * sh.e_cap));
    cs->d_items = static_cast<int32_t*>(take(sizeof(int32_t) * sh.e_cap));
    cs->d_loff = static_cast<int64_t*>(take(sizeof(int64_t) * (sh.e_cap + 1)));
    cs->d_item_start = static_cast<int64_t*>(take(sizeof(int64_t) * (sh.e_cap + 1)));
    cs->block_sums = static_cast<int64_t*>(take(sizeof(int64_t) * nbs));
    cs->n_block_sums = nbs;
    cs->d_k1 = static_cast<int32_t*>(take(sizeof(int32_t) * sh.e_cap));
    cs->d_u1 = static_cast<int64_t*>(take(sizeof(int64_t) * sh.e_cap));
    cs->d_hoff = static_cast<int64_t*>(take(sizeof(int64_t) * sh.e_cap));
    cs->items_cap = sh.e_cap + sh.list_cap / (LCH * kSuper) + 1;
    cs->item_j = static_cast<int32_t*>(take(sizeof(int32_t) * cs->items_cap));
    cs->r_cap = sh.r_cap;
    cs->r_pool = static_cast<int32_t*>(take(sizeof(int32_t) * sh.r_cap));
    cs->r_off = static_cast<int64_t*>(take(sizeof(int64_t) * sh.cap));
    cs->order = static_cast<int32_t*>(take(sizeof(int32_t) * sh.cap));
    cs->oflag = static_cast<int32_t*>(take(sizeof(int32_t) * sh.cap));
    cs->opre = static_cast<int64_t*>(take(sizeof(int64_t) * (sh.cap + 1)));
    const int64_t rn = sh.n_cta_nh, rc = int64_t(sh.c_per_sm) * sh.n_cta_c;
    cs->c_per_sm = sh.c_per_sm;
    cs->onh_keys = static_cast<int32_t*>(take(sizeof(int32_t) * rn * sh.gs_nh));
    cs->onh_vals = static_cast<uint32_t*>(take(sizeof(uint32_t) * rn * sh.gs_nh));
    cs->onh_aux = static_cast<int32_t*>(take(sizeof(int32_t) * rn * sh.gs_nh));
    cs->onh_list = static_cast<int32_t*>(take(sizeof(int32_t) * rn * (sh.gs_nh / 2)));
    cs->oc_keys = static_cast<int32_t*>(take(sizeof(int32_t) * rc * sh.gs_c));
    cs->oc_vals = static_cast<uint32_t*>(take(sizeof(uint32_t) * rc * sh.gs_c));
    cs->oc_mark = static_cast<uint32_t*>(take(sizeof(uint32_t) * rc * sh.gs_c));
    cs->oc_list = static_cast<int32_t*>(take(sizeof(int32_t) * rc * (sh.gs_c / 2)));
    cs->oc_lk = static_cast<int32_t*>(take(sizeof(int32_t) * rc * (sh.gs_c / 2)));
    cs->oc_lts = static_cast<int64_t*>(take(sizeof(int64_t) * rc * (sh.gs_c / 2)));
    cs->oc_lkey = static_cast<int32_t*>(take(sizeof(int32_t) * rc * (sh.gs_c / 2)));
    cs->oc_pf = static_cast<int32_t*>(take(sizeof(int32_t) * rc * (sh.gs_c / 2)));
    cs->oc_pm = static_cast<uint32_t*>(take(sizeof(uint32_t) * rc * (sh.gs_c / 2)));
    cs->oh_cap = open_h_cap(sh);
    if (cs->oh_cap > 0) {
        const size_t nb = size_t(sh.n_cta_c) * size_t(cs->oh_cap + 1);
        cs->oh_t = static_cast<int64_t*>(take(sizeof(int64_t) * nb));
        cs->oh_i = static_cast<int32_t*>(take(sizeof(int32_t) * nb));
        cs->oh_p = static_cast<int32_t*>(take(sizeof(int32_t) * nb));
        cs->oh_k = static_cast<uint32_t*>(take(sizeof(uint32_t) * nb));
        cs->oh_p1 = static_cast<uint32_t*>(take(sizeof(uint32_t) * nb));
        cs->oh_pc = static_cast<uint32_t*>(take(sizeof(uint32_t) * nb));
    }
    cs->h_total = pinned_word;
    cudaError_t e;
    if ((e = cudaMemsetAsync(cs->lcnt, 0, sizeof(int32_t) * sh.e_cap, st))) return e;
    if ((e = cudaMemsetAsync(cs->lfill, 0, sizeof(int32_t) * sh.e_cap, st))) return e;
    if ((e = cudaMemsetAsync(cs->onh_hist, 0, sizeof(uint32_t) * sh.n_cta_nh * 2 * (kMaxCard + 1), st))) return e;
    if ((e = cudaMemsetAsync(cs->onh_keys, 0xff, sizeof(int32_t) * rn * sh.gs_nh, st))) return e;
    if ((e = cudaMemsetAsync(cs->onh_vals, 0, sizeof(uint32_t) * rn * sh.gs_nh, st))) return e;
    if ((e = cudaMemsetAsync(cs->onh_aux, 0x7f, sizeof(int32_t) * rn * sh.gs_nh, st))) return e;
    if ((e = cudaMemsetAsync(cs->oc_keys, 0xff, sizeof(int32_t) * rc * sh.gs_c, st))) return e;
    if ((e = cudaMemsetAsync(cs->oc_vals, 0, sizeof(uint32_t) * rc * sh.gs_c, st))) return e;
    if ((e = cudaMemsetAsync(cs->oc_mark, 0, sizeof(uint32_t) * rc * sh.gs_c, st))) return e;
    return cudaSuccess;
}

cudaError_t upload_tables(cudaStream_t st) {
    static ClassTables t;
    static std::once_flag built;
    std::call_once(built, [] { build_class_tables(&t); });
    return cudaMemcpyToSymbolAsync(c_tables, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
}

// The centre and neighbourhood kernels' shared-memory limits, raised once per
// device (function attributes belong to the device they are set on).
void count_prepare() {
    constexpr int kDev = 64;
    static std::once_flag once[kDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) dev = 0;
    std::call_once(once[dev], [] {
    cudaFuncSetAttribute(k_nh_build, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(SmemNH)));
    cudaFuncSetAttribute(k_center<512, 8192, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(SmemC<512, 8192>)));
    cudaFuncSetAttribute(k_center<256, 4096, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(SmemC<256, 4096>)));
    cudaFuncSetAttribute(k_center<512, 4096, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(SmemC<512, 4096>)));
    cudaFuncSetAttribute(k_center<256, 2048, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(SmemC<256, 2048>)));
    cudaFuncSetAttribute(k_open_h<kOhNT, kOhMax, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(SmemOH)));
    cudaFuncSetAttribute(k_open_h<kOsNT, kOsMax, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(SmemOS)));
#define ESC_CO_ATTR(NT, TS, MB)                                                                          \
    cudaFuncSetAttribute(k_center_o<NT, TS, MB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                         int(sizeof(SmemCO<NT, TS>)));                                                      \
    cudaFuncSetAttribute(k_center_o<NT, TS, MB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                         int(sizeof(SmemCO<NT, TS>)));
    ESC_CO_ATTR(512, 8192, 1)
    ESC_CO_ATTR(256, 4096, 2)
    ESC_CO_ATTR(512, 4096, 2)
    ESC_CO_ATTR(256, 2048, 3)
#undef ESC_CO_ATTR
    });
}

// One count run: the changed hyperedges [lo, lo + n) (host-planned), or the
// range k_run_plan left on the device (dev).
static cudaError_t count_run(const Store& S, Scalars* sc, const int32_t* changed, const int32_t* changed_g,
                             const uint32_t* chg_bits, int64_t lo, int64_t n, bool dev, int side,
                             uint64_t* dcounts_side, const CountScratch& cs, cudaStream_t st, LaunchCounter& lc) {
    // without restricted lists closed pairs are searched in (|g|, g) order by
    // k_center_o (its temporal variant when the temporal family is kept)
    const bool orient = cs.orient && cs.r_cap == 0;
    const bool temp = (S.fam & kFamT) != 0;
    CountArgs A{S, sc, changed, changed_g, chg_bits, lo, n, side, dcounts_side, cs,
                uint32_t(cs.smem_slots < NH_S ? cs.smem_slots : NH_S),
                uint32_t(std::min<int64_t>(cs.smem_slots, cs.center_small == 0 ? 8192 : 4096)), dev, orient};
    const unsigned gd = blocks_for(cs.e_cap, kScanBlock);
    const unsigned ge = capped(blocks_for(cs.e_cap, 256));
    const int64_t nmax = dev ? cs.cap : n;  // what the grids are made for
    const unsigned gn = blocks_for(nmax, kScanBlock);
    const int32_t* n_run = dev ? &sc->run_n32[side] : nullptr;
    k_run_begin<<<1, 1, 0, st>>>(sc, side);
    k_order_flags<<<capped(blocks_for(nmax, 256)), 256, 0, st>>>(A);
    k_scan_sums<int32_t><<<gn, kScanNT, 0, st>>>(cs.oflag, n, n_run, cs.block_sums);
    k_scan_top<<<1, 32, 0, st>>>(cs.block_sums, gn, n_run);
    k_scan_apply<int32_t><<<gn, kScanNT, 0, st>>>(cs.oflag, n, n_run, cs.block_sums, cs.opre);
    k_order_place<<<capped(blocks_for(nmax, 256)), 256, 0, st>>>(A);
    k_nh_build<<<cs.n_cta_nh, NT_NH, sizeof(SmemNH), st>>>(A);
    if (orient && temp) {
        k_open_h<kOsNT, kOsMax, 4, true><<<cs.n_cta_c * 4, kOsNT, sizeof(SmemOS), st>>>(A);
        k_open_h<kOhNT, kOhMax, 1, false><<<cs.n_cta_c, kOhNT, sizeof(SmemOH), st>>>(A);
    }
    cudaMemsetAsync(cs.block_sums, 0, sizeof(int64_t) * kOrderBuckets, st);
    k_dsort_count<<<ge, 256, 0, st>>>(A);
    k_dsort_scan<<<1, 32, 0, st>>>(A);
    k_dsort_scatter<<<ge, 256, 0, st>>>(A);
    k_dsort_copy<<<ge, 256, 0, st>>>(A);
    k_d_prep<<<ge, 256, 0, st>>>(A);
    k_scan_sums<int32_t><<<gd, kScanNT, 0, st>>>(cs.d_cnt, 0, &sc->n_d[side], cs.block_sums);
    k_scan_top<<<1, 32, 0, st>>>(cs.block_sums, 0, &sc->n_d[side]);
    k_scan_apply<int32_t><<<gd, kScanNT, 0, st>>>(cs.d_cnt, 0, &sc->n_d[side], cs.block_sums, cs.d_loff);
    k_scan_sums<int32_t><<<gd, kScanNT, 0, st>>>(cs.d_items, 0, &sc->n_d[side], cs.block_sums);
    k_scan_top<<<1, 32, 0, st>>>(cs.block_sums, 0, &sc->n_d[side]);
    k_scan_apply<int32_t><<<gd, kScanNT, 0, st>>>(cs.d_items, 0, &sc->n_d[side], cs.block_sums, cs.d_item_start);
    k_set_loffg<<<ge, 256, 0, st>>>(A);
    if (orient) k_item_prep<<<capped(blocks_for(int64_t(cs.e_cap) * 32, 256)), 256, 0, st>>>(A);
    k_scatter<<<capped(blocks_for(nmax * 32, 256)), 256, 0, st>>>(A);
    const bool timed = cs.cev && cs.n_cev && *cs.n_cev < cs.max_cev;
    if (timed) cudaEventRecord(cs.cev[2 * *cs.n_cev], st);
    // three blocks per SM need the tables sized for them
    const int shape = cs.center_small == 3 && cs.c_per_sm < 3 ? 1 : cs.center_small;
    if (orient) {
#define ESC_CO_LAUNCH(NT, TS, MB, GRID)                                                            \
    (temp ? k_center_o<NT, TS, MB, true><<<GRID, NT, sizeof(SmemCO<NT, TS>), st>>>(A)             \
          : k_center_o<NT, TS, MB, false><<<GRID, NT, sizeof(SmemCO<NT, TS>), st>>>(A))
        switch (shape) {
            case 0: ESC_CO_LAUNCH(512, 8192, 1, cs.n_cta_c); break;
            case 2: ESC_CO_LAUNCH(512, 4096, 2, cs.n_cta_c * 2); break;
            case 3: ESC_CO_LAUNCH(256, 2048, 3, cs.n_cta_c * 3); break;
            default: ESC_CO_LAUNCH(256, 4096, 2, cs.n_cta_c * 2); break;
        }
#undef ESC_CO_LAUNCH
    } else {
        switch (shape) {
            case 0: k_center<512, 8192, 1><<<cs.n_cta_c, 512, sizeof(SmemC<512, 8192>), st>>>(A); break;
            case 2: k_center<512, 4096, 2><<<cs.n_cta_c * 2, 512, sizeof(SmemC<512, 4096>), st>>>(A); break;
            case 3: k_center<256, 2048, 3><<<cs.n_cta_c * 3, 256, sizeof(SmemC<256, 2048>), st>>>(A); break;
            default: k_center<256, 4096, 2><<<cs.n_cta_c * 2, 256, sizeof(SmemC<256, 4096>), st>>>(A); break;
        }
    }
    if (timed) cudaEventRecord(cs.cev[2 * (*cs.n_cev)++ + 1], st);
    k_d_clean<<<ge, 256, 0, st>>>(A);
    lc.total += (orient ? 23 : 22) + (orient && temp ? 2 : 0);
    lc.count += 2;
    return cudaGetLastError();
}

cudaError_t count_launch(const Store& S, Scalars* sc, const int32_t* changed, const int32_t* changed_g,
                         const uint32_t* chg_bits, int64_t lo, int64_t hi, int side, uint64_t* dcounts_side,
                         const CountScratch& cs, int64_t max_u, cudaStream_t st, LaunchCounter& lc) {
    count_prepare();
    if (cs.split_world > 1 && hi > lo) {
        // this rank's share of the side, by the prefix of the neighbourhood
        // sizes (a side holds at most cs.cap changed hyperedges)
        const int64_t n = std::min<int64_t>(hi - lo, cs.cap);
        k_nh_size<<<blocks_for(n * 32, 256), 256, 0, st>>>(S, sc, changed, lo, n, nullptr, cs.sizes, max_u,
                                                           cs.big_nh);
        const unsigned gb = blocks_for(n, kScanBlock);
        k_scan_sums<int32_t><<<gb, kScanNT, 0, st>>>(cs.sizes, n, nullptr, cs.block_sums);
        k_scan_top<<<1, 32, 0, st>>>(cs.block_sums, gb, nullptr);
        k_scan_apply<int32_t><<<gb, kScanNT, 0, st>>>(cs.sizes, n, nullptr, cs.block_sums, cs.nh_off);
        lc.total += 4;
        std::vector<int64_t> pre(size_t(n) + 1);
        cudaError_t e = cudaMemcpyAsync(pre.data(), cs.nh_off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        const int64_t W = cs.split_world, r = cs.split_rank, T = pre[n] + n;
        // owner of i: floor((pre[i] + i) * W / T), non-decreasing in i
        auto owner = [&](int64_t i) { return int64_t((__int128(pre[i] + i) * W) / T); };
        int64_t a = 0, b = n;
        while (a < n && owner(a) < r) ++a;
        b = a;
        while (b < n && owner(b) == r) ++b;
        CountScratch one = cs;
        one.split_world = 1;
        if (b > a)
            if ((e = count_launch(S, sc, changed, changed_g, chg_bits, lo + a, lo + b, side, dcounts_side, one,
                                  max_u, st, lc)))
                return e;
        if (hi - lo > n)  // never with the engine's sizes; kept exact regardless
            return count_launch(S, sc, changed, changed_g, chg_bits, lo + n, hi, side, dcounts_side, cs, max_u, st,
                                lc);
        return cudaSuccess;
    }
    for (int64_t a = lo; a < hi; a += cs.cap) {
        const int64_t b = a + cs.cap < hi ? a + cs.cap : hi;
        const int64_t n = b - a;
        // sizes of N(h) and the prefix that places every list
        k_nh_size<<<blocks_for(n * 32, 256), 256, 0, st>>>(S, sc, changed, a, n, nullptr, cs.sizes, max_u,
                                                           cs.big_nh);
        const unsigned gb = blocks_for(n, kScanBlock);
        k_scan_sums<int32_t><<<gb, kScanNT, 0, st>>>(cs.sizes, n, nullptr, cs.block_sums);
        k_scan_top<<<1, 32, 0, st>>>(cs.block_sums, gb, nullptr);
        k_scan_apply<int32_t><<<gb, kScanNT, 0, st>>>(cs.sizes, n, nullptr, cs.block_sums, cs.nh_off);
        lc.total += 4;
        cudaError_t e = cudaMemcpyAsync(cs.h_total, cs.nh_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        if (*cs.h_total <= cs.list_cap) {
            if ((e = count_run(S, sc, changed, changed_g, chg_bits, a, n, false, side, dcounts_side, cs, st, lc)))
                return e;
            continue;
        }
        // the lists do not fit: split [a, b) by the prefix of the sizes
        std::vector<int64_t> pre(size_t(n) + 1);
        if ((e = cudaMemcpy(pre.data(), cs.nh_off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost))) return e;
        int64_t s0 = 0;
        while (s0 < n) {
            int64_t s1 = s0;
            while (s1 < n && pre[s1 + 1] - pre[s0] <= cs.list_cap) ++s1;
            if (s1 == s0) return cudaErrorInvalidValue;  // one list alone exceeds the capacity
            if ((e = count_launch(S, sc, changed, changed_g, chg_bits, a + s0, a + s1, side, dcounts_side, cs,
                                  max_u, st, lc)))
                return e;
            s0 = s1;
        }
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// count runs planned on the device: a fixed launch sequence (capturable in a
// CUDA graph) for a side whose size the kernels read from n_side
// ---------------------------------------------------------------------------

__global__ void k_side_n(Scalars* sc, int side, const int64_t* n_side) {
    sc->n_side[side] = int32_t(*n_side);
    sc->run_lo[side] = 0;
    sc->run_n[side] = 0;
}

// Run r of a side: from the end of run r - 1, the longest range of changed
// hyperedges whose lists fit the arena.
__global__ void k_run_plan(Scalars* sc, int side, const int64_t* nh_off, int64_t list_cap) {
    const int64_t n = sc->n_side[side];
    const int64_t lo = sc->run_lo[side] + sc->run_n[side];
    int64_t hi = lo;
    if (lo < n && !sc->gate) {
        const int64_t lim = nh_off[lo] + list_cap;
        int64_t a = lo, b = n;  // the last index whose prefix stays within lim
        while (a < b) {
            const int64_t mid = (a + b + 1) >> 1;
            if (nh_off[mid] <= lim) a = mid;
            else b = mid - 1;
        }
        hi = a;
        if (hi == lo) set_error(sc, kErrUnsupported, -9, lo, nh_off[lo + 1] - nh_off[lo]);
    }
    sc->run_lo[side] = lo;
    sc->run_n[side] = hi - lo;
    sc->run_n32[side] = int32_t(hi - lo);
    sc->run_base[side] = lo < n ? nh_off[lo] : 0;
}

__global__ void k_run_check(Scalars* sc, int side) {
    if (!sc->gate && sc->run_lo[side] + sc->run_n[side] < sc->n_side[side])
        set_error(sc, kErrRetry, -10, side, sc->run_lo[side] + sc->run_n[side]);
}

// Before the store changes: the neighbour-list sizes the inserted side will
// have (the sum of the members' new degrees, as k_nh_size will find after the
// insert) and whether the fixed sequence's runs hold them; if not, the call
// takes the retry status now, while nothing has changed.
__global__ void k_pre_sizes(Store S, Call C, int32_t* sizes, int64_t max_u, int64_t big_nh) {
    const int64_t n = C.dims[1];
    if (blockIdx.x == 0 && threadIdx.x == 0) C.sc->n_side[1] = int32_t(n);
    if (C.sc->gate) return;
    const int lane = lane_id();
    for (int64_t j = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; j < n;
         j += (int64_t(gridDim.x) * blockDim.x) >> 5) {
        const int64_t p0 = C.ins_off[j];
        const int k = C.card[j];
        long long u = 0;
        for (int t = lane; t < k; t += 32) {
            const int32_t v = C.sorted[p0 + t];
            u += S.v_deg[v] - S.v_ndel[v] + S.v_nins[v];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (lane == 0) {
            if (u > max_u) u = 0;  // the ingest check reports it
            const long long t = u > big_nh ? (long long)pow2_at_least(2 * u) : 0;
            sizes[j] = int32_t(u + t + t / 8);
        }
    }
}

__global__ void k_pre_plan(Scalars* sc, const int64_t* pre, int64_t list_cap, int runs) {
    if (sc->gate) return;
    const int64_t n = sc->n_side[1];
    int64_t lo = 0;
    for (int r = 0; r < runs && lo < n; ++r) {
        const int64_t lim = pre[lo] + list_cap;
        int64_t a = lo, b = n;
        while (a < b) {
            const int64_t mid = (a + b + 1) >> 1;
            if (pre[mid] <= lim) a = mid;
            else b = mid - 1;
        }
        if (a == lo) return;  // one list alone exceeds the arena: the count reports it
        lo = a;
    }
    if (lo < n) set_error(sc, kErrRetry, -11, 1, lo);
}

cudaError_t count_precheck_fixed(const Store& S, const Call& C, const CountScratch& cs, int64_t max_u, int runs,
                                 cudaStream_t st, LaunchCounter& lc) {
    const int32_t* n1 = &C.sc->n_side[1];
    k_pre_sizes<<<capped(blocks_for(cs.cap * 32, 256)), 256, 0, st>>>(S, C, cs.oflag, max_u, cs.big_nh);
    const unsigned gb = blocks_for(cs.cap, kScanBlock);
    k_scan_sums<int32_t><<<gb, kScanNT, 0, st>>>(cs.oflag, 0, n1, cs.block_sums);
    k_scan_top<<<1, 32, 0, st>>>(cs.block_sums, gb, n1);
    k_scan_apply<int32_t><<<gb, kScanNT, 0, st>>>(cs.oflag, 0, n1, cs.block_sums, cs.opre);
    k_pre_plan<<<1, 1, 0, st>>>(C.sc, cs.opre, cs.list_cap, runs);
    lc.total += 5;
    return cudaGetLastError();
}

cudaError_t count_launch_fixed(const Store& S, Scalars* sc, const int32_t* changed, const int32_t* changed_g,
                               const uint32_t* chg_bits, const int64_t* n_side, int side, uint64_t* dcounts_side,
                               const CountScratch& cs, int64_t max_u, int runs, cudaStream_t st,
                               LaunchCounter& lc) {
    count_prepare();
    const int32_t* nd = &sc->n_side[side];
    k_side_n<<<1, 1, 0, st>>>(sc, side, n_side);
    k_nh_size<<<capped(blocks_for(cs.cap * 32, 256)), 256, 0, st>>>(S, sc, changed, 0, 0, nd, cs.sizes, max_u,
                                                                    cs.big_nh);
    const unsigned gb = blocks_for(cs.cap, kScanBlock);
    k_scan_sums<int32_t><<<gb, kScanNT, 0, st>>>(cs.sizes, 0, nd, cs.block_sums);
    k_scan_top<<<1, 32, 0, st>>>(cs.block_sums, gb, nd);
    k_scan_apply<int32_t><<<gb, kScanNT, 0, st>>>(cs.sizes, 0, nd, cs.block_sums, cs.nh_off);
    lc.total += 5;
    cudaError_t e;
    for (int r = 0; r < runs; ++r) {
        k_run_plan<<<1, 1, 0, st>>>(sc, side, cs.nh_off, cs.list_cap);
        ++lc.total;
        if ((e = count_run(S, sc, changed, changed_g, chg_bits, 0, 0, true, side, dcounts_side, cs, st, lc)))
            return e;
    }
    k_run_check<<<1, 1, 0, st>>>(sc, side);
    ++lc.total;
    return cudaGetLastError();
}

}  // namespace esc

// pairs.cu -- incident-vertex triads of types 1 and 2 from vertex-pair
// statistics (the family ESC_FAMILY_VERTEX12).
//
// Types 1 and 2 (Sec. II; a vertex triple with one witnessing hyperedge per
// vertex pair, typed by the number of distinct witnesses) need no
// neighbourhoods.  Type 1 is the sum over hyperedges of C(|h|, 3).  For
// type 2, with m_uv the number of hyperedges holding the vertex pair {u, v}
// and S_uv the sum of their sizes,
//     T2 = sum over hyperedge pairs {h, g} of C(|h & g|, 2) (|h| + |g| - 4)
//        = sum over vertex pairs {u, v} of (m_uv - 1) S_uv - 4 C(m_uv, 2),
// since a hyperedge pair sharing x vertices is met once per pair of them.
// Adding a hyperedge of size k to the pair {u, v} holding (m, S) changes its
// term by S + m (k - 4); removing one of size k from (m, S) changes it by
// -((S - k) + (m - 1)(k - 4)).  Both are >= 0 in magnitude (every size is
// >= 2).
//
// A batch applies Alg. 3's two sides: the deleted hyperedges leave the pair
// statistics and the inserted ones arrive.  Each (pair, hyperedge) step is
// one 64-bit atomicAdd on the pair's packed word m << 40 | S, which returns
// the (m, S) the step started from; steps on one pair are thereby
// serialised, and the changes of all steps telescope to T2(after) -
// T2(before) exactly, whatever their order -- so both sides run in one pass.
// The work per batch is the sum over changed hyperedges of C(|h|, 2),
// independent of vertex degrees, which makes hub vertices (a vertex in most
// hyperedges) cheap.
//
// Load balance: the member pairs of all changed hyperedges (deleted first,
// then inserted) form one index range, split evenly over the grid by the
// exclusive prefix of C(|h|, 2); a hyperedge with a million member pairs is
// spread over every SM, and ten thousand 2-member hyperedges fill one warp
// pass each.  A warp walks its contiguous part 32 pairs at a time, finding
// the hyperedge of each lane among the next 32 prefix entries.
//
// The statistics live in one open-addressing table keyed by the vertex pair
// (u << 32 | v, u < v, so key 0 marks an unused slot), key and word side by
// side in 16 bytes: a probe and its atomic touch one sector.  A pair whose
// last hyperedge leaves keeps its slot with m = 0 (its term is 0).
// Admission: before anything changes, the table must hold every key the
// batch could add (its inserted pairs) within its load limit, else the
// batch fails with OUT_OF_MEMORY.
#include <algorithm>

#include "escher_internal.cuh"
#include "store_api.cuh"

namespace esc {

namespace {

constexpr int kPairNT = 256;
constexpr int kPairTile = kPairNT * 16;   // changed hyperedges per scan tile
constexpr int kTopNT = 1024;
constexpr uint64_t kMask40 = (uint64_t(1) << 40) - 1;

// MurmurHash3's 64-bit finaliser (Appleby, public domain), used as the slot hash.
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

// Slot of a pair key; absent keys are added when `add` (the inserted side),
// otherwise -1 is returned (the deleted side always finds its keys).  A key
// this call added counts one in `fresh` (added to the table's count once
// per warp: a single counter taking one atomic per new key would serialise).
__device__ __forceinline__ int64_t pair_slot(const PairTable& P, uint64_t key, bool add, Scalars* sc,
                                             unsigned long long& fresh) {
    uint64_t s = fmix64(key) & P.mask;
    volatile unsigned long long* kv = P.kv;
    for (uint64_t probe = 0; probe <= P.mask; ++probe) {
        const unsigned long long cur = kv[2 * s];
        if (cur == key) return int64_t(s);
        if (cur == kPairEmpty) {
            if (!add) break;
            const unsigned long long old = atomicCAS(&P.kv[2 * s], kPairEmpty, (unsigned long long)key);
            if (old == kPairEmpty) {
                ++fresh;
                return int64_t(s);
            }
            if (old == key) return int64_t(s);
        }
        s = (s + 1) & P.mask;
    }
    // the admission check keeps the table below its load limit, and a
    // deleted hyperedge's pairs were added when it was inserted
    set_error(sc, kErrUnsupported, -14, int64_t(key >> 32), int64_t(key & 0xffffffffu));
    return -1;
}

// The pair (a, b), a < b < k, at index q of the pairs listed row by row
// (row a holds (a, a+1) .. (a, k-1) and starts at a (2k - a - 1) / 2).  The
// row comes from the quadratic's root; its discriminant is formed exactly
// in integers, so the float root is within one row, which the two loops fix.
__device__ __forceinline__ void pair_of(int64_t q, int k, int& a, int& b) {
    const int64_t bb = 2 * int64_t(k) - 1;
    const int64_t disc = bb * bb - 8 * q;  // >= 9 for every q < C(k, 2)
    int r = int((float(bb) - sqrtf(float(disc))) * 0.5f);
    r = max(0, min(r, k - 2));
    auto row0 = [k](int64_t x) { return x * (2 * int64_t(k) - x - 1) / 2; };
    while (r > 0 && row0(r) > q) --r;
    while (r < k - 2 && row0(r + 1) <= q) ++r;
    a = r;
    b = int(r + 1 + (q - row0(r)));
}

// Changed hyperedge j of the call: deleted ones first (side 0, members read
// from the store before the delete), then inserted ones (side 1, sorted
// members from the call's staging).
struct Changed {
    int k, side, g;
    const int32_t* m;
};
__device__ __forceinline__ Changed changed_at(const Store& S, const Call& C, int64_t nd, int64_t j) {
    Changed c;
    if (j < nd) {
        const int32_t h = C.del[j];
        c.k = S.h_card[h];
        c.m = S.hp.arena + S.h_off[h];
        c.g = C.del_g[j];
        c.side = 0;
    } else {
        const int64_t i = j - nd;
        c.k = C.card[i];
        c.m = C.sorted + C.ins_off[i];
        c.g = C.ins_g[i];
        c.side = 1;
    }
    return c;
}

__device__ __forceinline__ unsigned long long n_pairs(int k) {
    return (unsigned long long)k * (unsigned long long)(k - 1) / 2;
}

__device__ __forceinline__ uint64_t* v_out(const Store& S, int key) {
    // key = side * n_graphs + g
    return S.dcounts + int64_t(key) * kCStride + kOffV;
}

// Add `v` to word `w` (0: type 1, 1: type 2) of the output `key`, reduced
// over the warp when all its lanes hold the same key (or nothing).
__device__ __forceinline__ void warp_flush(const Store& S, int key, unsigned long long v, int w) {
    const int k0 = __shfl_sync(0xffffffffu, key, 0);
    if (__all_sync(0xffffffffu, key == k0 || v == 0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane_id() == 0 && v && k0 >= 0)
            atomicAdd(reinterpret_cast<unsigned long long*>(&v_out(S, k0)[w]), v);
    } else if (v && key >= 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&v_out(S, key)[w]), v);
    }
}

// ---- the exclusive prefix of C(|h|, 2) over the changed hyperedges ----

// tile sums
__global__ void __launch_bounds__(kPairNT) k_pair_tiles(Store S, Call C, PairTable P) {
    __shared__ unsigned long long red[kPairNT / 32];
    if (C.sc->gate) return;
    const int64_t nd = C.dims[2], n = nd + C.dims[1];
    const int64_t base = int64_t(blockIdx.x) * kPairTile;
    if (base >= n) return;
    unsigned long long s = 0;
    for (int64_t j = base + threadIdx.x; j < min(base + kPairTile, n); j += kPairNT)
        s += n_pairs(changed_at(S, C, nd, j).k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane_id() == 0) red[warp_id()] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kPairNT / 32; ++w) t += red[w];
        P.tsum[blockIdx.x] = int64_t(t);
    }
}

// exclusive scan of the tile sums, in place; the total closes the prefix
__global__ void __launch_bounds__(kTopNT) k_pair_top(Call C, PairTable P) {
    __shared__ int64_t part[kTopNT];
    if (C.sc->gate) return;
    const int64_t n = C.dims[2] + C.dims[1];
    const int64_t nt = (n + kPairTile - 1) / kPairTile;
    const int64_t per = (nt + kTopNT - 1) / kTopNT;
    const int64_t lo = min(nt, int64_t(threadIdx.x) * per), hi = min(nt, lo + per);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += P.tsum[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < kTopNT; ++t) {
            const int64_t v = part[t];
            part[t] = run;
            run += v;
        }
        P.poff[n] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = lo; i < hi; ++i) {
        const int64_t v = P.tsum[i];
        P.tsum[i] = run;
        run += v;
    }
}

// each tile's entries, and the type-1 terms C(|h|, 3)
__global__ void __launch_bounds__(kPairNT) k_pair_down(Store S, Call C, PairTable P) {
    __shared__ int64_t wsum[kPairNT / 32];
    if (C.sc->gate) return;
    const int64_t nd = C.dims[2], n = nd + C.dims[1];
    const int64_t base = int64_t(blockIdx.x) * kPairTile;
    if (base >= n) return;
    constexpr int kPer = kPairTile / kPairNT;
    const int64_t j0 = base + int64_t(threadIdx.x) * kPer;
    int64_t cnt[kPer];
    int64_t s = 0;
    int key = -1;
    unsigned long long t1 = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        cnt[i] = 0;
        if (j0 + i < n) {
            const Changed c = changed_at(S, C, nd, j0 + i);
            cnt[i] = int64_t(n_pairs(c.k));
            const int kk = c.side * S.n_graphs + c.g;
            if (kk != key) {
                if (t1 && key >= 0) atomicAdd(reinterpret_cast<unsigned long long*>(&v_out(S, key)[0]), t1);
                key = kk;
                t1 = 0;
            }
            if (c.k >= 3) t1 += (unsigned long long)c.k * (c.k - 1) * (c.k - 2) / 6;
        }
        s += cnt[i];
    }
    warp_flush(S, key, t1, 0);
    // block exclusive scan of the per-thread sums
    int64_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane_id() >= o) inc += v;
    }
    if (lane_id() == 31) wsum[warp_id()] = inc;
    __syncthreads();
    int64_t off = P.tsum[blockIdx.x];
    for (int w = 0; w < warp_id(); ++w) off += wsum[w];
    off += inc - s;
#pragma unroll
    for (int i = 0; i < kPer; ++i)
        if (j0 + i < n) {
            P.poff[j0 + i] = off;
            off += cnt[i];
        }
}

// ---- the pair steps ----
__global__ void __launch_bounds__(kPairNT) k_pairs(Store S, Call C, PairTable P) {
    if (C.sc->gate) return;
    const int64_t nd = C.dims[2], n = nd + C.dims[1];
    const int64_t total = P.poff[n];
    if (total == 0) return;
    constexpr int NW = kPairNT / 32;
    const int lane = lane_id();
    const int64_t nw_all = int64_t(gridDim.x) * NW;
    const int64_t w = int64_t(blockIdx.x) * NW + warp_id();
    int64_t p0 = total * w / nw_all;
    const int64_t p_end = total * (w + 1) / nw_all;
    if (p0 >= p_end) return;
    // the hyperedge holding p0: the last j with poff[j] <= p0 (every lane
    // searches the same entries)
    int64_t lo = 0, hi = n;  // poff[lo] <= p0 < poff[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (P.poff[mid] <= p0) lo = mid;
        else hi = mid;
    }
    int64_t j0 = lo, start0 = P.poff[lo];
    int key = -1;
    unsigned long long t2 = 0, fresh = 0;
    for (; p0 < p_end; p0 += 32) {
        // lane i's pair p lies in hyperedge jl, which starts at sl: the
        // boundaries poff[jw + 1 ..] after the window base are read 32 at a
        // time (sorted across the lanes); a run of empty hyperedges (fewer
        // than two members) can take more than one window
        const int64_t p = p0 + lane;
        const int64_t pe = min(p, p_end - 1);
        int64_t jl = j0, sl = start0;
        for (int64_t jw = j0;; jw += 32) {
            const int64_t bnd = jw + 1 + lane <= n ? P.poff[jw + 1 + lane] : INT64_MAX;
            int c = 0;  // boundaries of the window at or below pe
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int64_t v = __shfl_sync(0xffffffffu, bnd, c + step - 1);
                if (v <= pe) c += step;
            }
            const int64_t last = __shfl_sync(0xffffffffu, bnd, 31);
            if (c == 31 && last <= pe) c = 32;
            const int64_t vc = __shfl_sync(0xffffffffu, bnd, max(c - 1, 0));
            if (c > 0) {
                jl = jw + c;
                sl = vc;
            }
            if (!__any_sync(0xffffffffu, last <= pe)) break;
        }
        if (p < p_end) {
            const Changed ch = changed_at(S, C, nd, jl);
            int a, b;
            pair_of(p - sl, ch.k, a, b);
            const uint64_t pk = (uint64_t(uint32_t(ch.m[a])) << 32) | uint64_t(uint32_t(ch.m[b]));
            const int64_t slot = pair_slot(P, pk, ch.side == 1, C.sc, fresh);
            if (slot >= 0) {
                const unsigned long long inc = (1ull << 40) + (unsigned long long)ch.k;
                const unsigned long long old = atomicAdd(&P.kv[2 * slot + 1], ch.side ? inc : 0ull - inc);
                const int64_t mo = int64_t(old >> 40), so = int64_t(old & kMask40);
                // the change of the pair's term (its magnitude for a removal)
                const int64_t d = ch.side ? so + mo * (ch.k - 4) : (so - ch.k) + (mo - 1) * (ch.k - 4);
                const int kk = ch.side * S.n_graphs + ch.g;
                if (kk != key) {
                    if (t2 && key >= 0) atomicAdd(reinterpret_cast<unsigned long long*>(&v_out(S, key)[1]), t2);
                    key = kk;
                    t2 = 0;
                }
                t2 += (unsigned long long)d;
            }
        }
        // the next group starts in (or after) the hyperedge of the last lane
        j0 = __shfl_sync(0xffffffffu, jl, 31);
        start0 = __shfl_sync(0xffffffffu, sl, 31);
    }
    warp_flush(S, key, t2, 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fresh += __shfl_xor_sync(0xffffffffu, fresh, o);
    if (lane == 0 && fresh) atomicAdd(P.used, fresh);
}

// Admission, before anything changes: the keys the inserted hyperedges
// could add (all their member pairs) must fit below the table's load limit.
__global__ void k_pairs_check(Call C, PairTable P) {
    __shared__ unsigned long long red[32];
    if (C.sc->gate) return;
    const int64_t n = C.dims[1];
    unsigned long long need = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) need += n_pairs(C.card[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) need += __shfl_xor_sync(0xffffffffu, need, o);
    if (lane_id() == 0) red[warp_id()] = need;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < int(blockDim.x / 32); ++w) tot += red[w];
        if (*P.used + tot > P.limit) set_error(C.sc, kErrNoMem, -15, int64_t(*P.used + tot), int64_t(P.limit));
    }
}

int64_t n_tiles(int64_t n) { return (n + kPairTile - 1) / kPairTile; }

}  // namespace

size_t pair_table_bytes(int64_t pairs, int64_t n_cap) {
    const uint64_t slots = pair_table_slots(pairs);
    return size_t(slots) * 16 + 256 + size_t(n_cap + 1) * 8 + size_t(n_tiles(n_cap) + 1) * 8;
}

cudaError_t pair_table_init(PairTable* P, void* mem, int64_t pairs, int64_t n_cap, cudaStream_t st) {
    const uint64_t slots = pair_table_slots(pairs);
    char* p = static_cast<char*>(mem);
    P->kv = reinterpret_cast<unsigned long long*>(p);
    P->used = reinterpret_cast<unsigned long long*>(p + slots * 16);
    P->poff = reinterpret_cast<int64_t*>(p + slots * 16 + 256);
    P->tsum = P->poff + (n_cap + 1);
    P->mask = slots - 1;
    P->limit = pairs;
    P->n_cap = n_cap;
    static_assert(kPairEmpty == 0, "unused slots are zero");
    return cudaMemsetAsync(P->kv, 0, slots * 16 + 256, st);
}

cudaError_t pairs_check(const PairTable& P, const Call& C, cudaStream_t st, LaunchCounter& lc) {
    k_pairs_check<<<1, 1024, 0, st>>>(C, P);
    ++lc.total;
    return cudaGetLastError();
}

cudaError_t pairs_update(const Store& S, const Call& C, const PairTable& P, int sm_count, cudaStream_t st,
                         LaunchCounter& lc) {
    // the grids are made for the call's changed hyperedges (or, for a fixed
    // sequence, the limit); every kernel reads the counts on the device
    const int64_t n_grid = C.fixed ? std::min<int64_t>(C.grid_ins, P.n_cap) : C.grid_ins + C.grid_del;
    if (!C.fixed && n_grid <= 0) return cudaSuccess;
    const unsigned tiles = unsigned(std::max<int64_t>(n_tiles(n_grid), 1));
    k_pair_tiles<<<tiles, kPairNT, 0, st>>>(S, C, P);
    k_pair_top<<<1, kTopNT, 0, st>>>(C, P);
    k_pair_down<<<tiles, kPairNT, 0, st>>>(S, C, P);
    // one wave of resident blocks: the pair range is split evenly over them
    static const int per_sm = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs, kPairNT, 0) != cudaSuccess || b < 1) b = 1;
        return b;
    }();
    k_pairs<<<unsigned(sm_count) * unsigned(per_sm), kPairNT, 0, st>>>(S, C, P);
    lc.total += 4;
    lc.count += 1;
    return cudaGetLastError();
}

}  // namespace esc

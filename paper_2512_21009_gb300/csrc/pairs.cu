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
// A batch applies Alg. 3's two sides in order: the deleted hyperedges are
// removed from the pair statistics, then the inserted ones added.  Each
// (pair, hyperedge) step is one 64-bit atomicAdd on the pair's packed word
// m << 40 | S, which returns the (m, S) the step started from; steps on one
// pair are thereby serialised, and the changes of all steps telescope to
// T2(after) - T2(before) exactly, whatever their order.  The work per batch
// is the sum over changed hyperedges of C(|h|, 2), independent of vertex
// degrees, which makes hub vertices (a vertex in most hyperedges) cheap.
//
// The statistics live in one open-addressing table keyed by the vertex pair
// (u << 32 | v, u < v); a pair whose last hyperedge leaves keeps its slot
// with m = 0 (its term is 0).  Admission: before anything changes, the
// table must hold every key the batch could add (its inserted pairs) within
// its load limit, else the batch fails with OUT_OF_MEMORY.
#include <algorithm>

#include "escher_internal.cuh"
#include "store_api.cuh"

namespace esc {

namespace {

constexpr int kPairNT = 256;
constexpr int kPairSmem = 4096;      // members of a hyperedge staged in shared memory
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
// otherwise -1 is returned (the deleted side always finds its keys).
__device__ __forceinline__ int64_t pair_slot(const PairTable& P, uint64_t key, bool add, Scalars* sc) {
    uint64_t s = fmix64(key) & P.mask;
    volatile unsigned long long* vk = P.keys;
    for (uint64_t probe = 0; probe <= P.mask; ++probe) {
        const unsigned long long cur = vk[s];
        if (cur == key) return int64_t(s);
        if (cur == kPairEmpty) {
            if (!add) break;
            const unsigned long long old = atomicCAS(&P.keys[s], kPairEmpty, (unsigned long long)key);
            if (old == kPairEmpty) {
                atomicAdd(P.used, 1ull);
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

// row of pair index p among the pairs (i, j), i < j < k, listed row by row
__device__ __forceinline__ void pair_of(int64_t p, int k, int& i, int& j) {
    const double b = 2.0 * k - 1.0;
    int r = int((b - sqrt(b * b - 8.0 * double(p))) * 0.5);
    auto row0 = [k](int64_t q) { return q * (2 * int64_t(k) - q - 1) / 2; };
    if (r < 0) r = 0;
    while (r > 0 && row0(r) > p) --r;
    while (r + 1 < k - 1 && row0(r + 1) <= p) ++r;
    i = r;
    j = int(r + 1 + (p - row0(r)));
}

// One side of a batch: side 0 removes the deleted hyperedges (members from
// the store, before the delete), side 1 adds the inserted ones (sorted
// members from the call's staging).  A block per hyperedge, its threads
// over the member pairs.
__global__ void __launch_bounds__(kPairNT) k_pairs(Store S, Call C, PairTable P, int side) {
    __shared__ int32_t mem_s[kPairSmem];
    __shared__ unsigned long long red[kPairNT / 32];
    if (C.sc->gate) return;
    const int64_t n = side ? C.dims[1] : C.dims[2];
    const int tid = threadIdx.x;
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        int k, g;
        const int32_t* m;
        if (side) {
            k = C.card[j];
            m = C.sorted + C.ins_off[j];
            g = C.ins_g[j];
        } else {
            const int32_t h = C.del[j];
            k = S.h_card[h];
            m = S.hp.arena + S.h_off[h];
            g = C.del_g[j];
        }
        const bool staged = k <= kPairSmem;
        __syncthreads();
        if (staged)
            for (int t = tid; t < k; t += kPairNT) mem_s[t] = m[t];
        __syncthreads();
        const int32_t* mm = staged ? mem_s : m;
        const int64_t np = int64_t(k) * (k - 1) / 2;
        const unsigned long long inc = (1ull << 40) + (unsigned long long)k;
        unsigned long long t2 = 0;
        for (int64_t p = tid; p < np; p += kPairNT) {
            int a, b;
            pair_of(p, k, a, b);
            const uint64_t key = (uint64_t(uint32_t(mm[a])) << 32) | uint64_t(uint32_t(mm[b]));
            const int64_t sl = pair_slot(P, key, side == 1, C.sc);
            if (sl < 0) continue;
            const unsigned long long old = atomicAdd(&P.vals[sl], side ? inc : 0ull - inc);
            const int64_t mo = int64_t(old >> 40), so = int64_t(old & kMask40);
            // the change of the pair's term (its magnitude for a removal)
            const int64_t d = side ? so + mo * (k - 4) : (so - k) + (mo - 1) * (k - 4);
            t2 += (unsigned long long)d;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
        if (lane_id() == 0) red[warp_id()] = t2;
        __syncthreads();
        if (tid == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < kPairNT / 32; ++w) tot += red[w];
            uint64_t* out = S.dcounts + (int64_t(side) * S.n_graphs + g) * kCStride + kOffV;
            const unsigned long long t1 =
                k >= 3 ? (unsigned long long)k * (k - 1) * (k - 2) / 6 : 0ull;
            if (t1) atomicAdd(reinterpret_cast<unsigned long long*>(&out[0]), t1);
            if (tot) atomicAdd(reinterpret_cast<unsigned long long*>(&out[1]), tot);
        }
    }
}

// Admission, before anything changes: the keys the inserted hyperedges
// could add (all their member pairs) must fit below the table's load limit.
__global__ void k_pairs_check(Call C, PairTable P) {
    __shared__ unsigned long long red[32];
    if (C.sc->gate) return;
    const int64_t n = C.dims[1];
    unsigned long long need = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const unsigned long long k = (unsigned long long)C.card[j];
        need += k * (k - 1) / 2;
    }
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

}  // namespace

size_t pair_table_bytes(int64_t pairs) {
    const uint64_t slots = pair_table_slots(pairs);
    return size_t(slots) * 16 + 256;
}

cudaError_t pair_table_init(PairTable* P, void* mem, int64_t pairs, cudaStream_t st) {
    const uint64_t slots = pair_table_slots(pairs);
    char* p = static_cast<char*>(mem);
    P->keys = reinterpret_cast<unsigned long long*>(p);
    P->vals = reinterpret_cast<unsigned long long*>(p + slots * 8);
    P->used = reinterpret_cast<unsigned long long*>(p + slots * 16);
    P->mask = slots - 1;
    P->limit = pairs;
    cudaError_t e;
    if ((e = cudaMemsetAsync(P->keys, 0xff, slots * 8, st))) return e;
    if ((e = cudaMemsetAsync(P->vals, 0, slots * 8, st))) return e;
    return cudaMemsetAsync(P->used, 0, sizeof(unsigned long long), st);
}

cudaError_t pairs_check(const PairTable& P, const Call& C, cudaStream_t st, LaunchCounter& lc) {
    k_pairs_check<<<1, 1024, 0, st>>>(C, P);
    ++lc.total;
    return cudaGetLastError();
}

cudaError_t pairs_update(const Store& S, const Call& C, const PairTable& P, int side, int sm_count, cudaStream_t st,
                         LaunchCounter& lc) {
    const int64_t n = side ? C.grid_ins : C.grid_del;
    if (!C.fixed && n <= 0) return cudaSuccess;
    const int64_t grid = std::min<int64_t>(std::max<int64_t>(n, 1), int64_t(sm_count) * 16);
    k_pairs<<<unsigned(grid), kPairNT, 0, st>>>(S, C, P, side);
    ++lc.total;
    ++lc.count;
    return cudaGetLastError();
}

}  // namespace esc

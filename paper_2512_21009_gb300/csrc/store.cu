// store.cu -- batch ingest, validation and the vertical update of the
// incidence store (paper Section III-B, "Deletion of hyperedges" and
// "Insertion of Hyperedges"; Algorithm 3, step 3).
//
// A call runs in three phases, all on one stream:
//   ingest     gather the batches into call arrays (translated to the store's
//              global IDs), sort and deduplicate every inserted member list,
//              validate every delete, count per-vertex deltas, and check every
//              capacity -- nothing of the store changes here;
//   (count of the deleted side on the old graph, count.cu)
//   mutate     free deleted hyperedges, assign IDs to inserts (j-th insert ->
//              j-th smallest free ID), allocate slabs, write h2v, rewrite the
//              v2h lists of touched vertices;
//   (count of the inserted side on the new graph, count.cu)
//   finish     fold the two count deltas into the counts, clear scratch.
// The first error found latches a "gate" word; every later kernel that would
// change the store reads the gate first and does nothing when it is set, so a
// failed call leaves the store unchanged.
#include <algorithm>

#include "escher_internal.cuh"
#include "store_api.cuh"

namespace esc {

namespace {

constexpr int kBlk = 256;  // threads per block of the element-wise kernels

__device__ __forceinline__ int64_t pool_alloc(const SlabPool& P, int c) {
    int i = atomicSub(&P.top[c], 1) - 1;
    if (i >= 0) return int64_t(P.stack[P.base[c] + i]) << kMinSlabLog;
    return int64_t(atomicAdd(reinterpret_cast<unsigned long long*>(P.tail),
                             static_cast<unsigned long long>(slab_size(c))));
}

__device__ __forceinline__ void pool_free(const SlabPool& P, int c, int64_t off) {
    int i = atomicAdd(&P.top[c], 1);
    P.stack[P.base[c] + i] = uint32_t(off >> kMinSlabLog);
}

__device__ __forceinline__ void pool_clamp(const SlabPool& P) {
    for (int c = 0; c < kNumClasses; ++c)
        if (P.top[c] < 0) P.top[c] = 0;
}

// Sizes of the call, read on the device (so one launch sequence serves calls
// of any size, e.g. replayed from a CUDA graph).
__device__ __forceinline__ int nbat(const Call& C) { return int(C.dims[0]); }
__device__ __forceinline__ int64_t nins(const Call& C) { return C.dims[1]; }
__device__ __forceinline__ int64_t ndel(const Call& C) { return C.dims[2]; }

// Grid-stride ranges: one thread, or one warp, per element.
#define ESC_FOR_THREADS(i, n) \
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < (n); i += int64_t(gridDim.x) * blockDim.x)
#define ESC_FOR_WARPS(i, n)                                                            \
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < (n); \
         i += (int64_t(gridDim.x) * blockDim.x) >> 5)

__device__ __forceinline__ void touch(const Store& S, const Call& C, int32_t v) {
    if (atomicExch(&S.v_touch[v], 1) == 0) {
        int t = atomicAdd(&C.sc->n_touched, 1);
        C.touched[t] = v;
    }
}

// ---------------------------------------------------------------------------
// ingest
// ---------------------------------------------------------------------------

// Member count of every batch (read from its device offsets) and the member
// offset of each batch in the call arrays.
__global__ void k_plan(Call C) {
    __shared__ int warp_tmp[32];
    __shared__ long long carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int nb = nbat(C);
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        int b = b0 + threadIdx.x;
        long long nnz = 0;
        if (b < nb) {
            const BatchIn& B = C.batches[b];
            if (B.n_ins > 0) {
                if (B.off[0] != 0) set_error(C.sc, kErrInvalid, b, 0, B.off[0]);
                nnz = B.off[B.n_ins] - B.off[0];
                if (nnz < 0) { set_error(C.sc, kErrInvalid, b, B.n_ins, nnz); nnz = 0; }
            }
        }
        // members of one call stay below 2^31
        int tot;
        int pre = block_exclusive_scan<1024>(int(nnz > 0x7fffffff ? 0x7fffffff : nnz), &tot, warp_tmp);
        if (b < nb) C.nnz_lo[b] = carry_s + pre;
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        C.nnz_lo[nb] = carry_s;
        C.sc->nnz = carry_s;
        if (carry_s > C.max_nnz) set_error(C.sc, kErrNoMem, -1, carry_s, C.max_nnz);
    }
}

__device__ __forceinline__ int batch_of(const int64_t* lo, int nb, int64_t j) {
    return int(upper_bound_dev(lo, int64_t(nb) + 1, j) - 1);
}

// Inserts and deletes: offsets, timestamps, graph of each element; delete
// IDs translated to global IDs.
__global__ void k_gather(Store S, Call C, const int64_t* b_ins_lo, const int64_t* b_del_lo) {
    const int64_t ni = nins(C), nd = ndel(C);
    const int nb = nbat(C);
    ESC_FOR_THREADS(j, ni + nd) {
    if (j < ni) {
        int b = batch_of(b_ins_lo, nb, j);
        const BatchIn& B = C.batches[b];
        int64_t i = j - b_ins_lo[b];
        int64_t o0 = B.off[i], o1 = B.off[i + 1];
        int64_t n = o1 - o0;
        if (n <= 0) set_error(C.sc, n < 0 ? kErrInvalid : kErrInvalid, b, i, n);
        else if (n > kMaxCard) set_error(C.sc, kErrUnsupported, b, i, n);
        C.ins_off[j] = C.nnz_lo[b] + o0;
        if (j == ni - 1) C.ins_off[ni] = C.nnz_lo[b] + o1;
        C.ts[j] = B.ts ? B.ts[i] : 0;
        C.ins_g[j] = B.graph;
        if (B.pin) {
            // a horizontal update: the hyperedge keeps its ID and, unless
            // given one, its timestamp (read before anything changes)
            const int32_t p = B.pin[i];
            if (p < 0 || p >= S.ecap[B.graph]) {
                set_error(C.sc, kErrNotFound, -6, i, p);
                C.ids[j] = -1;
            } else {
                const int64_t id = S.ebase[B.graph] + p;
                C.ids[j] = int32_t(id);
                if (!B.ts) C.ts[j] = S.h_ts[id];
            }
        }
    } else {
        int64_t d = j - ni;
        int b = batch_of(b_del_lo, nb, d);
        const BatchIn& B = C.batches[b];
        int64_t i = d - b_del_lo[b];
        int32_t h = B.del[i];
        int g = B.graph;
        if (h < 0 || h >= S.ecap[g]) {
            set_error(C.sc, kErrNotFound, b, i, h);
            C.del[d] = -1;
        } else {
            C.del[d] = int32_t(S.ebase[g] + h);
        }
        C.del_g[d] = g;
    }
    }
}

// Members, translated to global vertex IDs and range-checked.
__global__ void k_gather_mem(Store S, Call C) {
    int64_t n = C.sc->nnz;
    if (n > C.max_nnz) n = C.max_nnz;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n;
         p += int64_t(gridDim.x) * blockDim.x) {
        int b = batch_of(C.nnz_lo, nbat(C), p);
        const BatchIn& B = C.batches[b];
        int32_t v = B.mem[p - C.nnz_lo[b]];
        int g = B.graph;
        if (v < 0 || v >= S.nv[g]) {
            set_error(C.sc, kErrInvalid, b, p - C.nnz_lo[b], v);
            v = 0;
        }
        C.raw[p] = int32_t(S.vbase[g] + v);
    }
}

__global__ void k_latch(Scalars* sc, int first) {
    sc->gate = sc->status;
    if (first && sc->status == 0) sc->ran = 1;
}

// Sort and deduplicate one inserted member list per warp (at most 32
// members): a bitonic network over the 32 lanes, then keep every value that
// differs from its left neighbour.  Longer lists go to the block sorter.
__global__ void k_sort_small(Store S, Call C) {
    if (C.sc->gate) return;
    const int lane = lane_id();
    ESC_FOR_WARPS(j, nins(C)) {
    int64_t p0 = C.ins_off[j];
    int n = int(C.ins_off[j + 1] - p0);
    if (n > 32) {
        if (lane == 0) C.big[atomicAdd(&C.sc->n_big, 1)] = int32_t(j);
        continue;
    }
    int32_t x = lane < n ? C.raw[p0 + lane] : 0x7fffffff;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int m = k >> 1; m > 0; m >>= 1) {
            int32_t y = __shfl_xor_sync(0xffffffffu, x, m);
            bool up = (lane & k) == 0;
            bool lower = (lane & m) == 0;
            x = (lower == up) ? min(x, y) : max(x, y);
        }
    }
    int32_t prev = __shfl_up_sync(0xffffffffu, x, 1);
    bool keep = lane < n && (lane == 0 || x != prev);
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) C.sorted[p0 + __popc(bal & ((1u << lane) - 1))] = x;
    if (lane == 0) {
        int k = __popc(bal);
        C.card[j] = k;
        atomicAdd(&C.sc->need_h[slab_class(k)], 1);
    }
    }
}

// Block sorter for member lists of 33..kMaxCard entries: bitonic sort in
// shared memory (padded to a power of two), then deduplicate with a block
// scan of "differs from left neighbour" flags.
constexpr int kSortNT = 512;
__global__ void __launch_bounds__(kSortNT) k_sort_big(Store S, Call C) {
    extern __shared__ int32_t sbuf[];  // kMaxCard
    __shared__ int warp_tmp[32];
    __shared__ int base_s;
    if (C.sc->gate) return;
    int nbig = C.sc->n_big;
    for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
        int64_t j = C.big[q];
        int64_t p0 = C.ins_off[j];
        int n = int(C.ins_off[j + 1] - p0);
        int np = 64;
        while (np < n) np <<= 1;
        for (int i = threadIdx.x; i < np; i += kSortNT) sbuf[i] = i < n ? C.raw[p0 + i] : 0x7fffffff;
        __syncthreads();
        for (int k = 2; k <= np; k <<= 1) {
            for (int m = k >> 1; m > 0; m >>= 1) {
                for (int i = threadIdx.x; i < np; i += kSortNT) {
                    int l = i ^ m;
                    if (l > i) {
                        int32_t a = sbuf[i], b = sbuf[l];
                        bool up = (i & k) == 0;
                        if ((a > b) == up) { sbuf[i] = b; sbuf[l] = a; }
                    }
                }
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) base_s = 0;
        __syncthreads();
        for (int i0 = 0; i0 < n; i0 += kSortNT) {
            int i = i0 + threadIdx.x;
            int keep = (i < n) && (i == 0 || sbuf[i] != sbuf[i - 1]);
            int tot;
            int pre = block_exclusive_scan<kSortNT>(keep, &tot, warp_tmp);
            if (keep) C.sorted[p0 + base_s + pre] = sbuf[i];
            __syncthreads();
            if (threadIdx.x == 0) base_s += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            C.card[j] = base_s;
            atomicAdd(&C.sc->need_h[slab_class(base_s)], 1);
        }
        __syncthreads();
    }
}

// Deletes: live and distinct; mark them; count the slab classes they free.
__global__ void k_del_check(Store S, Call C) {
    if (C.sc->gate) return;
    ESC_FOR_THREADS(d, ndel(C)) {
        int32_t h = C.del[d];
        if (!bit_test(S.live, h)) {
            set_error(C.sc, kErrNotFound, -1, d, h - S.ebase[C.del_g[d]]);
            continue;
        }
        uint32_t old = atomicOr(&S.delb[h >> 5], 1u << (h & 31));
        if (old & (1u << (h & 31))) {
            set_error(C.sc, kErrInvalid, -1, d, h - S.ebase[C.del_g[d]]);
            continue;
        }
        atomicAdd(&C.sc->freed_h[slab_class(S.h_card[h])], 1);
    }
}

// Inserts with given IDs: the ID must not hold a live hyperedge, unless the
// same call deletes it (a horizontal update).
__global__ void k_pin_check(Store S, Call C) {
    if (C.sc->gate) return;
    for (int bi = blockIdx.x; bi < nbat(C); bi += gridDim.x) {
        const BatchIn& B = C.batches[bi];
        if (!B.pin) continue;
        const int64_t eb = S.ebase[B.graph];
        for (int64_t i = threadIdx.x; i < B.n_ins; i += blockDim.x) {
            const int32_t p = B.pin[i];
            if (p < 0 || p >= S.ecap[B.graph]) continue;  // k_gather reports it
            const int64_t id = eb + p;
            if (bit_test(S.live, id) && !bit_test(S.delb, id)) set_error(C.sc, kErrInvalid, -5, i, p);
        }
    }
}

// Per-vertex delete counts from the deleted hyperedges' member lists, and the
// largest neighbour-entry count sum(deg) of a deleted hyperedge.
__global__ void k_touch_del(Store S, Call C) {
    if (C.sc->gate) return;
    const int lane = lane_id();
    ESC_FOR_WARPS(d, ndel(C)) {
    int32_t h = C.del[d];
    int k = bit_test(S.live, h) ? S.h_card[h] : 0;
    const int32_t* m = S.hp.arena + S.h_off[h];
    long long u = 0;
    for (int t = lane; t < k; t += 32) {
        int32_t v = m[t];
        u += S.v_deg[v];
        atomicAdd(&S.v_ndel[v], 1);
        touch(S, C, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (lane == 0) atomicMax(&C.sc->max_u, int(u > 0x7fffffff ? 0x7fffffff : u));
    }
}

// Per-vertex insert counts; every inserted member gets its place in the run
// of IDs appended to its vertex's v2h list.
__global__ void k_touch_ins(Store S, Call C) {
    if (C.sc->gate) return;
    const int lane = lane_id();
    ESC_FOR_WARPS(j, nins(C)) {
        int64_t p0 = C.ins_off[j];
        int k = C.card[j];
        for (int t = lane; t < k; t += 32) {
            int32_t v = C.sorted[p0 + t];
            C.slot[p0 + t] = atomicAdd(&S.v_nins[v], 1);
            touch(S, C, v);
        }
    }
}

// New degree of every touched vertex; vertices that outgrow their slab get
// a larger class.
__global__ void k_vplan(Store S, Call C) {
    if (C.sc->gate) return;
    int nt = C.sc->n_touched;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        int32_t v = C.touched[t];
        int nd = S.v_deg[v] - S.v_ndel[v] + S.v_nins[v];
        if (nd > S.v_cap[v]) {
            int c = slab_class(nd);
            atomicAdd(&C.sc->need_v[c], 1);
            S.v_newcap[v] = int32_t(slab_size(c));
            S.realloc_v[atomicAdd(&C.sc->n_realloc, 1)] = v;
        }
    }
}

// Largest neighbour-entry count of an inserted hyperedge on the new graph.
__global__ void k_ins_u(Store S, Call C) {
    if (C.sc->gate) return;
    const int lane = lane_id();
    ESC_FOR_WARPS(j, nins(C)) {
    int64_t p0 = C.ins_off[j];
    int k = C.card[j];
    long long u = 0;
    for (int t = lane; t < k; t += 32) {
        int32_t v = C.sorted[p0 + t];
        u += S.v_deg[v] - S.v_ndel[v] + S.v_nins[v];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (lane == 0) atomicMax(&C.sc->max_u, int(u > 0x7fffffff ? 0x7fffffff : u));
    }
}

// Capacities: slab arenas (exact demand per class after reuse of free
// slabs), ID ranges of every graph, and the counter's table limit.
__global__ void k_check(Store S, Call C, int64_t max_u) {
    if (C.sc->gate || threadIdx.x != 0) return;
    Scalars* sc = C.sc;
    long long bump = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        long long short_by = (long long)sc->need_h[c] - S.hp.top[c] - sc->freed_h[c];
        if (short_by > 0) bump += short_by * slab_size(c);
    }
    if (*S.hp.tail + bump > S.hp.cap) set_error(sc, kErrNoMem, -2, *S.hp.tail + bump, S.hp.cap);
    bump = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        long long short_by = (long long)sc->need_v[c] - S.vp.top[c];
        if (short_by > 0) bump += short_by * slab_size(c);
    }
    if (*S.vp.tail + bump > S.vp.cap) set_error(sc, kErrNoMem, -3, *S.vp.tail + bump, S.vp.cap);
    for (int b = 0; b < nbat(C); ++b) {
        const BatchIn& B = C.batches[b];
        if (B.pin) continue;  // kept IDs need no free ones
        int g = B.graph;
        long long freeids = S.hw[g] - S.n_live[g] + B.n_del;
        long long extra = B.n_ins - freeids;
        if (extra > 0 && S.hw[g] + extra > S.ecap[g]) set_error(sc, kErrNoMem, b, S.hw[g] + extra, S.ecap[g]);
    }
    if (sc->max_u > max_u) set_error(sc, kErrUnsupported, -4, sc->max_u, max_u);
}

// ---------------------------------------------------------------------------
// mutate
// ---------------------------------------------------------------------------

__global__ void k_hdel(Store S, Call C) {
    if (C.sc->gate) return;
    ESC_FOR_THREADS(d, ndel(C)) {
        int32_t h = C.del[d];
        pool_free(S.hp, slab_class(S.h_card[h]), S.h_off[h]);
        atomicAnd(&S.live[h >> 5], ~(1u << (h & 31)));
        S.h_card[h] = 0;
        atomicAdd(reinterpret_cast<unsigned long long*>(&S.n_live[C.del_g[d]]), ~0ull);
    }
}

// ID rule: the j-th insert of a graph takes the j-th smallest free ID below
// the high-water mark (free = not live; the deleted IDs were just freed),
// then fresh IDs upward.  One block per batch scans the graph's live bitmap.
constexpr int kSelNT = 1024;
__global__ void __launch_bounds__(kSelNT) k_select(Store S, Call C) {
    __shared__ int warp_tmp[32];
    __shared__ long long carry_s;
    if (C.sc->gate) return;
    for (int bi = blockIdx.x; bi < nbat(C); bi += gridDim.x) {
    const BatchIn& B = C.batches[bi];
    int64_t n = B.n_ins;
    if (n == 0) continue;
    if (B.pin) {
        // IDs given by the caller (set by k_gather): the high-water mark
        // covers them, so later inserts never take one
        int m = -1;
        for (int64_t r = threadIdx.x; r < n; r += kSelNT) m = max(m, B.pin[r]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane_id() == 0) warp_tmp[warp_id()] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 0; w < kSelNT / 32; ++w) m = max(m, warp_tmp[w]);
            if (int64_t(m) + 1 > S.hw[B.graph]) S.hw[B.graph] = int64_t(m) + 1;
        }
        __syncthreads();
        continue;
    }
    int g = B.graph;
    int64_t eb = S.ebase[g], hwg = S.hw[g];
    int64_t nwords = (hwg + 31) >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t w0 = 0; w0 < nwords; w0 += kSelNT) {
        if (carry_s >= n) break;
        int64_t w = w0 + threadIdx.x;
        uint32_t fr = 0;
        if (w < nwords) {
            fr = ~S.live[(eb >> 5) + w];
            int64_t rem = hwg - (w << 5);
            if (rem < 32) fr &= (1u << rem) - 1u;
        }
        int tot;
        int pre = block_exclusive_scan<kSelNT>(__popc(fr), &tot, warp_tmp);
        int64_t r = carry_s + pre;
        while (fr && r < n) {
            int b = __ffs(fr) - 1;
            C.ids[B.ins_lo + r] = int32_t(eb + (w << 5) + b);
            fr &= fr - 1;
            ++r;
        }
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tot;
        __syncthreads();
    }
    int64_t F = carry_s < n ? carry_s : n;
    for (int64_t r = F + threadIdx.x; r < n; r += kSelNT) C.ids[B.ins_lo + r] = int32_t(eb + hwg + (r - F));
    if (threadIdx.x == 0) S.hw[g] = hwg + (n - F);
    __syncthreads();
    }
}

__global__ void k_hins(Store S, Call C) {
    if (C.sc->gate) return;
    ESC_FOR_THREADS(j, nins(C)) {
        int32_t id = C.ids[j];
        int k = C.card[j];
        S.h_off[id] = pool_alloc(S.hp, slab_class(k));
        S.h_card[id] = k;
        S.h_ts[id] = C.ts[j];
        atomicOr(&S.live[id >> 5], 1u << (id & 31));
        atomicOr(&S.insb[id >> 5], 1u << (id & 31));
        atomicAdd(reinterpret_cast<unsigned long long*>(&S.n_live[C.ins_g[j]]), 1ull);
    }
}

__global__ void k_valloc(Store S, Call C) {
    if (C.sc->gate) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) pool_clamp(S.hp);
    int nr = C.sc->n_realloc;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        int32_t v = S.realloc_v[r];
        S.v_newoff[v] = pool_alloc(S.vp, slab_class(S.v_newcap[v]));
    }
}

// Rewrite the v2h list of every touched vertex: drop the deleted IDs (kept
// order, compacted by warp ballot, in place when the slab still fits) and
// leave room for the appended IDs.  A vertex of degree >= kVBig (a hub under
// skewed popularity, in a large share of all hyperedges) is left to
// k_vfilter_big: one warp walking its list 32 entries at a time would take
// tens of thousands of dependent steps.
constexpr int kVBig = 2048;

// The new v2h metadata of v once `kept` entries remain at dst.
__device__ __forceinline__ void vfilter_finish(const Store& S, const Call& C, int32_t v, int kept, int deg, int nd,
                                               int newdeg, bool moved, int64_t off, int64_t dst, int cap) {
    if (kept != deg - nd) set_error(C.sc, kErrCuda, -5, v, kept);
    S.v_base[v] = kept;
    S.v_deg[v] = newdeg;
    if (moved) {
        S.v_off[v] = dst;
        int newcap = S.v_newcap[v];
        S.v_newoff[v] = off;       // old slab, freed by k_vfree
        S.v_newcap[v] = cap;
        S.v_cap[v] = newcap;
    }
}

__global__ void k_vfilter(Store S, Call C) {
    if (C.sc->gate) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) pool_clamp(S.vp);
    int nt = C.sc->n_touched;
    int lane = lane_id();
    int64_t wid = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t t = wid; t < nt; t += nw) {
        int32_t v = C.touched[t];
        int nd = S.v_ndel[v], ni = S.v_nins[v], deg = S.v_deg[v], cap = S.v_cap[v];
        if (deg >= kVBig) {
            if (lane == 0) S.vbig[atomicAdd(&C.sc->n_vbig, 1)] = v;
            continue;
        }
        int64_t off = S.v_off[v];
        int newdeg = deg - nd + ni;
        bool moved = newdeg > cap;
        int64_t dst = moved ? S.v_newoff[v] : off;
        int kept = deg;
        if (nd > 0 || moved) {
            kept = 0;
            for (int base = 0; base < deg; base += 32) {
                int e = base + lane;
                int32_t h = e < deg ? S.vp.arena[off + e] : 0;
                bool keep = e < deg && !bit_test(S.delb, h);
                unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (keep) S.vp.arena[dst + kept + __popc(bal & ((1u << lane) - 1))] = h;
                kept += __popc(bal);
            }
        }
        if (lane == 0) vfilter_finish(S, C, v, kept, deg, nd, newdeg, moved, off, dst, cap);
    }
}

// The same for the vertices of degree >= kVBig, a block per vertex: the list
// is compacted in chunks of kVChunk entries (kVPer consecutive ones per
// thread), in order, by a block scan of the kept counts.  In place this is
// safe: every thread has loaded its entries of a chunk before the scan's
// barrier, and the chunk's writes land below the chunk's end.
constexpr int kVNT = 512, kVPer = 8, kVChunk = kVNT * kVPer;
static_assert(kVPer == 8 && (1 << kMinSlabLog) % kVPer == 0, "two 16-byte loads per thread, slab-aligned");

__global__ void __launch_bounds__(kVNT) k_vfilter_big(Store S, Call C) {
    __shared__ int wsum[kVNT / 32];
    __shared__ int total_s;
    if (C.sc->gate) return;
    const int nb = C.sc->n_vbig;
    const int tid = threadIdx.x, lane = lane_id(), w = warp_id();
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int32_t v = S.vbig[b];
        const int nd = S.v_ndel[v], ni = S.v_nins[v], deg = S.v_deg[v], cap = S.v_cap[v];
        const int64_t off = S.v_off[v];
        const int newdeg = deg - nd + ni;
        const bool moved = newdeg > cap;
        const int64_t dst = moved ? S.v_newoff[v] : off;
        int kept = deg;
        if (nd > 0 || moved) {
            kept = 0;
            for (int base = 0; base < deg; base += kVChunk) {
                int32_t val[kVPer];
                unsigned keep = 0;
                int cnt = 0;
                const int e0 = base + tid * kVPer;
                if (e0 + kVPer <= deg) {
                    // every slab offset is a multiple of 8 slots (slabs are
                    // 8 << c slots, handed out whole), and so is e0: two
                    // aligned 16-byte loads
                    const int4* src = reinterpret_cast<const int4*>(S.vp.arena + off + e0);
                    const int4 a = src[0], b = src[1];
                    val[0] = a.x; val[1] = a.y; val[2] = a.z; val[3] = a.w;
                    val[4] = b.x; val[5] = b.y; val[6] = b.z; val[7] = b.w;
                } else {
#pragma unroll
                    for (int i = 0; i < kVPer; ++i) val[i] = e0 + i < deg ? S.vp.arena[off + e0 + i] : 0;
                }
#pragma unroll
                for (int i = 0; i < kVPer; ++i) {
                    const int e = base + tid * kVPer + i;
                    if (e < deg && !bit_test(S.delb, val[i])) {
                        keep |= 1u << i;
                        ++cnt;
                    }
                }
                // block exclusive scan of the kept counts
                int inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int x = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += x;
                }
                if (lane == 31) wsum[w] = inc;
                __syncthreads();
                if (w == 0) {
                    int x = lane < kVNT / 32 ? wsum[lane] : 0;
                    const int own = x;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, x, o);
                        if (lane >= o) x += y;
                    }
                    if (lane < kVNT / 32) wsum[lane] = x - own;
                    if (lane == 31) total_s = x;
                }
                __syncthreads();
                int pos = kept + wsum[w] + inc - cnt;
#pragma unroll
                for (int i = 0; i < kVPer; ++i)
                    if (keep & (1u << i)) S.vp.arena[dst + pos++] = val[i];
                kept += total_s;
                __syncthreads();  // wsum and total_s are rewritten by the next chunk
            }
        }
        if (tid == 0) vfilter_finish(S, C, v, kept, deg, nd, newdeg, moved, off, dst, cap);
        __syncthreads();
    }
}

// Copy the sorted members of every insert into its h2v slab and append its
// ID to the v2h list of each member.
__global__ void k_ins_write(Store S, Call C) {
    if (C.sc->gate) return;
    const int lane = lane_id();
    ESC_FOR_WARPS(j, nins(C)) {
        int32_t id = C.ids[j];
        int64_t p0 = C.ins_off[j];
        int64_t hoff = S.h_off[id];
        int k = C.card[j];
        for (int t = lane; t < k; t += 32) {
            int32_t v = C.sorted[p0 + t];
            S.hp.arena[hoff + t] = v;
            S.vp.arena[S.v_off[v] + S.v_base[v] + C.slot[p0 + t]] = id;
        }
    }
}

__global__ void k_vfree(Store S, Call C) {
    if (C.sc->gate) return;
    int nr = C.sc->n_realloc;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        int32_t v = S.realloc_v[r];
        int oldcap = S.v_newcap[v];
        if (oldcap > 0) pool_free(S.vp, slab_class(oldcap), S.v_newoff[v]);
    }
}

// ---------------------------------------------------------------------------
// finish
// ---------------------------------------------------------------------------

__global__ void k_fold_counts(Store S, Call C) {
    const bool ok = C.sc->gate == 0;
    for (int bi = blockIdx.x; bi < nbat(C); bi += gridDim.x) {
        const int g = C.batches[bi].graph;
        uint64_t* cur = S.counts + int64_t(g) * kCStride;
        uint64_t* dd = S.dcounts + int64_t(g) * kCStride;
        uint64_t* di = S.dcounts + (int64_t(S.n_graphs) + g) * kCStride;
        for (int k = threadIdx.x; k < kCStride; k += blockDim.x) {
            if (ok) cur[k] += di[k] - dd[k];
            dd[k] = 0;
            di[k] = 0;
        }
    }
}

__global__ void k_cleanup(Store S, Call C) {
    bool ran = C.sc->ran != 0;
    bool ok = C.sc->gate == 0;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t stride = int64_t(gridDim.x) * blockDim.x;
    if (ran) {
        for (int64_t d = i; d < ndel(C); d += stride) {
            int32_t h = C.del[d];
            if (h >= 0) atomicAnd(&S.delb[h >> 5], ~(1u << (h & 31)));
        }
        int nt = C.sc->n_touched;
        for (int64_t t = i; t < nt; t += stride) {
            int32_t v = C.touched[t];
            S.v_ndel[v] = 0;
            S.v_nins[v] = 0;
            S.v_touch[v] = 0;
        }
    }
    if (ok) {
        for (int64_t j = i; j < nins(C); j += stride) {
            int32_t id = C.ids[j];
            atomicAnd(&S.insb[id >> 5], ~(1u << (id & 31)));
            C.out_local[j] = int32_t(id - S.ebase[C.ins_g[j]]);
        }
    }
}

inline unsigned grid_for(int64_t n, int nt) {
    int64_t g = (n + nt - 1) / nt;
    if (g < 1) g = 1;
    if (g > (1 << 30)) g = 1 << 30;
    return unsigned(g);
}

}  // namespace

#define ESC_LAUNCH(lc, ...)                 \
    do {                                    \
        __VA_ARGS__;                        \
        ++(lc).total;                       \
        cudaError_t e_ = cudaGetLastError(); \
        if (e_ != cudaSuccess) return e_;   \
    } while (0)

// grids: one thread or one warp per element, at most 16 blocks per SM (the
// kernels stride over what is left)
static unsigned g_thr(int64_t n, int sm) { return std::min<unsigned>(grid_for(n, kBlk), unsigned(sm) * 16u); }
static unsigned g_warp(int64_t n, int sm) { return std::min<unsigned>(grid_for(n * 32, kBlk), unsigned(sm) * 16u); }

void store_prepare() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(k_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxCard * sizeof(int32_t)));
    done = true;
}

cudaError_t store_ingest(const Store& S, const Call& C, const int64_t* b_ins_lo, const int64_t* b_del_lo,
                         int64_t max_u, int sm_count, cudaStream_t st, LaunchCounter& lc) {
    store_prepare();
    const int64_t gi = C.grid_ins, gd = C.grid_del;
    const bool any_i = C.fixed || gi > 0, any_d = C.fixed || gd > 0;
    ESC_LAUNCH(lc, k_plan<<<1, 1024, 0, st>>>(C));
    if (any_i || any_d)
        ESC_LAUNCH(lc, k_gather<<<g_thr(gi + gd, sm_count), kBlk, 0, st>>>(S, C, b_ins_lo, b_del_lo));
    if (any_i) ESC_LAUNCH(lc, k_gather_mem<<<sm_count * 8, kBlk, 0, st>>>(S, C));
    ESC_LAUNCH(lc, k_latch<<<1, 1, 0, st>>>(C.sc, 1));
    if (any_i) {
        ESC_LAUNCH(lc, k_sort_small<<<g_warp(gi, sm_count), kBlk, 0, st>>>(S, C));
        ESC_LAUNCH(lc, k_sort_big<<<sm_count * 2, kSortNT, kMaxCard * sizeof(int32_t), st>>>(S, C));
    }
    if (any_d) {
        ESC_LAUNCH(lc, k_del_check<<<g_thr(gd, sm_count), kBlk, 0, st>>>(S, C));
        ESC_LAUNCH(lc, k_touch_del<<<g_warp(gd, sm_count), kBlk, 0, st>>>(S, C));
    }
    if (C.fixed || C.pinned) ESC_LAUNCH(lc, k_pin_check<<<unsigned(std::max<int64_t>(C.grid_batches, 1)), kBlk, 0, st>>>(S, C));
    if (any_i) ESC_LAUNCH(lc, k_touch_ins<<<g_warp(gi, sm_count), kBlk, 0, st>>>(S, C));
    ESC_LAUNCH(lc, k_vplan<<<sm_count * 4, kBlk, 0, st>>>(S, C));
    if (any_i) ESC_LAUNCH(lc, k_ins_u<<<g_warp(gi, sm_count), kBlk, 0, st>>>(S, C));
    ESC_LAUNCH(lc, k_check<<<1, 32, 0, st>>>(S, C, max_u));
    ESC_LAUNCH(lc, k_latch<<<1, 1, 0, st>>>(C.sc, 0));
    return cudaSuccess;
}

cudaError_t store_delete(const Store& S, const Call& C, int sm_count, cudaStream_t st, LaunchCounter& lc) {
    if (C.fixed || C.grid_del > 0) ESC_LAUNCH(lc, k_hdel<<<g_thr(C.grid_del, sm_count), kBlk, 0, st>>>(S, C));
    return cudaSuccess;
}

cudaError_t store_insert(const Store& S, const Call& C, int sm_count, cudaStream_t st, LaunchCounter& lc) {
    const int64_t gi = C.grid_ins;
    const bool any_i = C.fixed || gi > 0;
    if (any_i) {
        ESC_LAUNCH(lc, k_select<<<unsigned(std::max<int64_t>(C.grid_batches, 1)), kSelNT, 0, st>>>(S, C));
        ESC_LAUNCH(lc, k_hins<<<g_thr(gi, sm_count), kBlk, 0, st>>>(S, C));
    }
    ESC_LAUNCH(lc, k_valloc<<<sm_count, kBlk, 0, st>>>(S, C));
    ESC_LAUNCH(lc, k_vfilter<<<sm_count * 8, kBlk, 0, st>>>(S, C));
    ESC_LAUNCH(lc, k_vfilter_big<<<sm_count * 2, kVNT, 0, st>>>(S, C));
    if (any_i) ESC_LAUNCH(lc, k_ins_write<<<g_warp(gi, sm_count), kBlk, 0, st>>>(S, C));
    ESC_LAUNCH(lc, k_vfree<<<sm_count, kBlk, 0, st>>>(S, C));
    return cudaSuccess;
}

cudaError_t store_latch(const Call& C, cudaStream_t st, LaunchCounter& lc) {
    ESC_LAUNCH(lc, k_latch<<<1, 1, 0, st>>>(C.sc, 0));
    return cudaSuccess;
}

cudaError_t store_finish(const Store& S, const Call& C, int sm_count, cudaStream_t st, LaunchCounter& lc) {
    ESC_LAUNCH(lc, k_fold_counts<<<unsigned(std::max<int64_t>(C.grid_batches, 1)), 160, 0, st>>>(S, C));
    ESC_LAUNCH(lc, k_cleanup<<<sm_count * 4, kBlk, 0, st>>>(S, C));
    return cudaSuccess;
}

}  // namespace esc

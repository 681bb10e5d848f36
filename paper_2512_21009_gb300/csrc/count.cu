// count.cu -- incremental triad counting (paper Algorithm 3, steps 2 and 5).
//
// The paper counts the triads of the affected regions before and after the
// update.  Here the same change is computed exactly as
//     new = old - T_old(holding >= 1 deleted) + T_new(holding >= 1 inserted),
// since a triad of unchanged hyperedges keeps its class.  For one set of
// changed hyperedges X, every triad holding a member of X is counted once, at
// its member of X with the smallest ID (the "attribution" rule); the kernel
// therefore enumerates, for each h in X, the triads {h, a, b} in which no
// other member of X with a smaller ID appears.
//
// For a changed h with neighbourhood N(h) (hyperedges sharing a vertex with
// h, paper Section II: neighbouring hyperedges), the connected triples
// holding h are exactly
//   (i)  {h, g1, g2} with g1, g2 in N(h)        -- closed if g1 meets g2,
//                                                   else open with centre h;
//   (ii) {h, g1, f}  with g1 in N(h), f in N(g1) outside N(h) and f != h
//                                                -- open with centre g1.
// One work item is (h, a range of h's incidence positions).  Its block builds
// N(h) in a hash table with x_hg = |h & g|, takes as candidates the g1 first
// met inside its position range, and for each candidate builds N(g1) with
// x = |g1 & f| and t = |h & g1 & f| in a second hash table; type (ii) triads
// come from scanning that table, type (i) from probing it with every g2 > g1
// of N(h).  Venn region sizes follow from |a|, |b|, |c|, the three pairwise
// intersections and t by inclusion-exclusion; the 7-bit pattern is mapped to
// its class by the tables of tables.cu.
//
// The incident-vertex types (Section II) come from the same quantities:
//   type 1 = sum over h of C(|h|, 3)
//   type 2 = sum over hyperedge pairs {h, g} of C(x_hg, 2) (|h| + |g| - 4)
//   type 3 = sum over closed triples {a, b, c} of
//            x_ab x_bc x_ac - t (x_ab + x_bc + x_ac) + 2 t
// (choose a vertex in each pairwise intersection, all three distinct).
#include <climits>

#include "escher_internal.cuh"
#include "store_api.cuh"

namespace esc {

namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int NH_S = 2048;   // shared-memory N(h) table slots
constexpr int T1_S = 4096;   // shared-memory N(g1) table slots
constexpr int HM_S = 1024;   // members of h kept in shared memory
constexpr int SEG = NT;      // members per segment
constexpr int CHUNK = 256;   // incidence positions of h per work item
constexpr int32_t EMPTY = -1;
constexpr int kHistT = kNH;  // temporal bins start here in the shared histograms
constexpr int kHistN = kNH + kNT;

__constant__ ClassTables c_tables;

struct CountArgs {
    Store S;
    Scalars* sc;
    const int32_t* changed;
    const int32_t* changed_g;
    const uint32_t* chg;
    int64_t lo, hi;
    const int64_t* item_start;  // [hi-lo+1]
    int side;
    uint64_t* dc;               // [G][kCStride]
    int32_t* g_keys;
    uint32_t* g_vals;
    int32_t* g_aux;
    int32_t* g_list;
    int64_t g_slots;
    uint32_t nh_smem_cap, t1_smem_cap;  // shared-memory table limits (<= NH_S, T1_S)
};

struct __align__(16) Smem {
    unsigned long long acc[128];
    uint32_t hist[NW][128];
    int32_t nh_keys[NH_S];
    uint32_t nh_x[NH_S];
    int32_t nh_fp[NH_S];
    int32_t nh_list[NH_S / 2];
    int32_t t1_keys[T1_S];
    uint32_t t1_vals[T1_S];
    int32_t t1_list[T1_S / 2];
    int32_t hm[HM_S];
    int64_t seg_off[SEG];
    int32_t seg_pre[SEG + 1];
    uint8_t seg_inh[SEG];
    int32_t cand_g[CHUNK];
    uint32_t cand_x[CHUNK];
    int8_t cls30[128];
    int8_t cls96[128];
    uint8_t perm[6][128];
    int warp_tmp[32];
    long long red[NW];
    long long item;
    int n_nh, n_t1, n_cand;
};

// MurmurHash3's 32-bit finaliser (Appleby, public domain), used as the slot hash.
__device__ __forceinline__ uint32_t fmix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
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

__device__ __forceinline__ long long block_sum(long long v, Smem& s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0) s.red[warp_id()] = v;
    __syncthreads();
    long long t = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += s.red[w];
    __syncthreads();
    return t;
}

// Load members mem[0..n) (n <= SEG) into the segment arrays: v2h offset,
// optionally "also in h", and the exclusive prefix of their degrees.
// Returns the number of incidence entries of the segment.
__device__ __forceinline__ int load_segment(const Store& S, const int32_t* mem, int n, bool want_inh,
                                            const int32_t* hmem, int kh, Smem& s) {
    int d = 0;
    if (int(threadIdx.x) < n) {
        int32_t v = mem[threadIdx.x];
        d = S.v_deg[v];
        s.seg_off[threadIdx.x] = S.v_off[v];
        if (want_inh) s.seg_inh[threadIdx.x] = contains_sorted(hmem, kh, v) ? 1 : 0;
    }
    int tot;
    int pre = block_exclusive_scan<NT>(d, &tot, s.warp_tmp);
    if (int(threadIdx.x) < n) s.seg_pre[threadIdx.x] = pre;
    if (threadIdx.x == 0) s.seg_pre[n] = tot;
    __syncthreads();
    return tot;
}

// member index of incidence entry e of the loaded segment
__device__ __forceinline__ int seg_member(const Smem& s, int n, int e) {
    int lo = 0, hi = n;  // largest m with seg_pre[m] <= e
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s.seg_pre[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct Accum {
    unsigned long long v1, v2, v3;
    unsigned long long n_v2h, n_h2v, n_meta, n_tri;
};

// Classify the triad (a, b, c) with sizes ka, kb, kc, pairwise intersections
// xab, xbc, xac and triple intersection t.
__device__ __forceinline__ void classify(Smem& s, uint32_t fam, int64_t delta, int32_t ia, int32_t ib,
                                         int32_t ic, int ka, int kb, int kc, int xab, int xbc, int xac, int t,
                                         int64_t ta, int64_t tb, int64_t tc, Accum& acc) {
    int ra = ka - xab - xac + t, rb = kb - xab - xbc + t, rc = kc - xbc - xac + t;
    int m = (ra > 0) | ((rb > 0) << 1) | ((rc > 0) << 2) | ((xab - t > 0) << 3) | ((xbc - t > 0) << 4) |
            ((xac - t > 0) << 5) | ((t > 0) << 6);
    uint32_t* hist = s.hist[warp_id()];
    ++acc.n_tri;
    if (fam & kFamH) {
        int c = s.cls30[m];
        if (c >= 0) atomicAdd(&hist[c], 1u);
    }
    if (fam & kFamT) {
        // order the labels 0 (a), 1 (b), 2 (c) by (timestamp, ID)
        int64_t T[3] = {ta, tb, tc};
        int32_t I[3] = {ia, ib, ic};
        int o0 = 0, o1 = 1, o2 = 2, tmp;
#define ESC_BEFORE(x, y) (T[x] < T[y] || (T[x] == T[y] && I[x] < I[y]))
        if (ESC_BEFORE(o1, o0)) { tmp = o0; o0 = o1; o1 = tmp; }
        if (ESC_BEFORE(o2, o1)) { tmp = o1; o1 = o2; o2 = tmp; }
        if (ESC_BEFORE(o1, o0)) { tmp = o0; o0 = o1; o1 = tmp; }
#undef ESC_BEFORE
        if (T[o2] - T[o0] <= delta) {
            int c = s.cls96[s.perm[perm_index(o0, o1)][m]];
            if (c >= 0) atomicAdd(&hist[kHistT + c], 1u);
        }
    }
}

__device__ void flush(const CountArgs& A, Smem& s, int g, Accum& acc) {
    uint64_t* out = A.dc + int64_t(g) * kCStride;
    for (int b = threadIdx.x; b < kHistN; b += NT) {
        unsigned long long v = s.acc[b];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(b < kNH ? &out[b] : &out[kOffT + (b - kHistT)]), v);
        s.acc[b] = 0;
    }
    long long v1 = block_sum((long long)acc.v1, s);
    long long v2 = block_sum((long long)acc.v2, s);
    long long v3 = block_sum((long long)acc.v3, s);
    if (threadIdx.x == 0) {
        if (v1) atomicAdd(reinterpret_cast<unsigned long long*>(&out[kOffV + 0]), (unsigned long long)v1);
        if (v2) atomicAdd(reinterpret_cast<unsigned long long*>(&out[kOffV + 1]), (unsigned long long)v2);
        if (v3) atomicAdd(reinterpret_cast<unsigned long long*>(&out[kOffV + 2]), (unsigned long long)v3);
    }
    acc.v1 = acc.v2 = acc.v3 = 0;
    __syncthreads();
}

__global__ void __launch_bounds__(NT, 2) k_count(CountArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& s = *reinterpret_cast<Smem*>(smem_raw);
    const Store& S = A.S;
    if (A.sc->gate) return;
    const int tid = threadIdx.x;
    const uint32_t fam = S.fam;
    const int64_t delta = S.delta;
    const bool want_open = (fam & (kFamH | kFamT)) != 0;
    const int32_t* v2h = S.vp.arena;
    const int32_t* h2v = S.hp.arena;

    for (int i = tid; i < 128; i += NT) {
        s.cls30[i] = c_tables.cls30[i];
        s.cls96[i] = c_tables.cls96[i];
        s.acc[i] = 0;
        for (int q = 0; q < 6; ++q) s.perm[q][i] = c_tables.perm[q][i];
        for (int w = 0; w < NW; ++w) s.hist[w][i] = 0;
    }
    for (int i = tid; i < NH_S; i += NT) {
        s.nh_keys[i] = EMPTY;
        s.nh_x[i] = 0;
        s.nh_fp[i] = INT_MAX;
    }
    for (int i = tid; i < T1_S; i += NT) {
        s.t1_keys[i] = EMPTY;
        s.t1_vals[i] = 0;
    }
    if (tid == 0) s.n_nh = s.n_t1 = s.n_cand = 0;
    __syncthreads();

    const int64_t gs = A.g_slots;
    const int64_t r_nh = int64_t(blockIdx.x) * 2, r_t1 = r_nh + 1;
    Tab gNH{A.g_keys + r_nh * gs, A.g_vals + r_nh * gs, A.g_aux + r_nh * gs, A.g_list + r_nh * (gs / 2),
            &s.n_nh, uint32_t(gs - 1), int(gs / 2)};
    Tab gT1{A.g_keys + r_t1 * gs, A.g_vals + r_t1 * gs, nullptr, A.g_list + r_t1 * (gs / 2), &s.n_t1,
            uint32_t(gs - 1), int(gs / 2)};

    Accum acc = {0, 0, 0, 0, 0, 0, 0};
    const int64_t n_items = A.sc->items[A.side];
    const int64_t n_changed = A.hi - A.lo;
    int cur_g = -1;

    for (;;) {
        __syncthreads();
        if (tid == 0) s.item = (long long)atomicAdd(&A.sc->queue[A.side], 1ull);
        __syncthreads();
        const int64_t item = s.item;
        if (item >= n_items) break;
        const int64_t i = upper_bound_dev(A.item_start, n_changed + 1, item) - 1;
        const int64_t chunk = item - A.item_start[i];
        const int32_t h = A.changed[A.lo + i];
        const int g = A.changed_g ? A.changed_g[A.lo + i] : 0;
        if (g != cur_g) {
            if (cur_g >= 0) flush(A, s, cur_g, acc);
            cur_g = g;
        }
        const int kh = S.h_card[h];
        const int32_t* hmem = h2v + S.h_off[h];
        const int64_t tsh = S.h_ts[h];
        const bool hm_smem = kh <= HM_S;
        long long uh = 0;
        for (int t = tid; t < kh; t += NT) {
            int32_t v = hmem[t];
            if (hm_smem) s.hm[t] = v;
            uh += S.v_deg[v];
        }
        acc.n_h2v += (tid < kh) ? (kh - tid + NT - 1) / NT : 0;
        uh = block_sum(uh, s);  // also orders the hm writes before use
        const int32_t* hm = hm_smem ? s.hm : hmem;

        // ---- N(h) with x_hg and the first incidence position of every g
        Tab NH;
        const uint32_t nh_cap = pow2_at_least(2 * uh);
        if (nh_cap <= A.nh_smem_cap) {
            NH = Tab{s.nh_keys, s.nh_x, s.nh_fp, s.nh_list, &s.n_nh, nh_cap - 1, NH_S / 2};
        } else if ((int64_t)nh_cap <= gs) {
            NH = gNH;
            NH.mask = nh_cap - 1;
        } else {
            if (tid == 0) set_error(A.sc, kErrUnsupported, -8, h, uh);
            continue;
        }
        const bool single_h = kh <= SEG;
        int seg_n = 0, seg_tot = 0;
        {
            long long pos_base = 0;
            for (int m0 = 0; m0 < kh; m0 += SEG) {
                seg_n = min(SEG, kh - m0);
                seg_tot = load_segment(S, hmem + m0, seg_n, false, nullptr, 0, s);
                for (int e = tid; e < seg_tot; e += NT) {
                    int m = seg_member(s, seg_n, e);
                    int32_t f = v2h[s.seg_off[m] + (e - s.seg_pre[m])];
                    if (f != h) tab_insert(NH, f, 1u, int32_t(pos_base + e), A.sc);
                }
                acc.n_v2h += (tid < seg_tot) ? (seg_tot - tid + NT - 1) / NT : 0;
                pos_base += seg_tot;
                __syncthreads();
            }
        }
        const int n_nh = min(s.n_nh, NH.list_cap);

        // ---- candidates g1: first met at a position of this chunk, and not
        //      a changed hyperedge of smaller ID
        const long long p_lo = chunk * CHUNK, p_hi = min(p_lo + CHUNK, (long long)uh);
        {
            long long pos_base = 0;
            for (int m0 = 0; m0 < kh && pos_base < p_hi; m0 += SEG) {
                int n = min(SEG, kh - m0);
                int tot = single_h ? seg_tot : load_segment(S, hmem + m0, n, false, nullptr, 0, s);
                long long lo = max(p_lo - pos_base, 0LL), hi = min(p_hi - pos_base, (long long)tot);
                for (long long e = lo + tid; e < hi; e += NT) {
                    int m = seg_member(s, n, int(e));
                    int32_t f = v2h[s.seg_off[m] + (e - s.seg_pre[m])];
                    if (f == h) continue;
                    int sl = tab_find(NH, f);
                    if (sl < 0 || NH.aux[sl] != int32_t(pos_base + e)) continue;
                    if (f < h && bit_test(A.chg, f)) continue;
                    int c = atomicAdd(&s.n_cand, 1);
                    s.cand_g[c] = f;
                    s.cand_x[c] = NH.vals[sl];
                }
                pos_base += tot;
                __syncthreads();
            }
        }
        const int n_cand = s.n_cand;

        // ---- every candidate g1
        for (int c = 0; c < n_cand; ++c) {
            const int32_t g1 = s.cand_g[c];
            const int xh1 = int(s.cand_x[c]);
            const int k1 = S.h_card[g1];
            const int32_t* g1mem = h2v + S.h_off[g1];
            const int64_t ts1 = S.h_ts[g1];
            const bool single = k1 <= SEG;
            long long u1;
            int n1seg = 0;
            if (single) {
                n1seg = k1;
                u1 = load_segment(S, g1mem, k1, true, hm, kh, s);
            } else {
                long long u = 0;
                for (int t = tid; t < k1; t += NT) u += S.v_deg[g1mem[t]];
                u1 = block_sum(u, s);
            }
            acc.n_h2v += (tid < k1) ? (k1 - tid + NT - 1) / NT : 0;
            Tab T1;
            int P = 1;
            const uint32_t t1_cap = pow2_at_least(2 * u1);
            if (t1_cap <= A.t1_smem_cap) {
                T1 = Tab{s.t1_keys, s.t1_vals, nullptr, s.t1_list, &s.n_t1, t1_cap - 1, T1_S / 2};
            } else {
                T1 = gT1;
                if ((int64_t)t1_cap <= gs) T1.mask = t1_cap - 1;
                else P = int((4 * u1 + gs - 1) / gs);
            }
            for (int p = 0; p < P; ++p) {
                // build N(g1): x in the low 16 bits, t (also in h) in the high 16
                for (int m0 = 0; m0 < k1; m0 += SEG) {
                    int n = single ? n1seg : min(SEG, k1 - m0);
                    int tot = single ? int(u1) : load_segment(S, g1mem + m0, n, true, hm, kh, s);
                    for (int e = tid; e < tot; e += NT) {
                        int m = seg_member(s, n, e);
                        int32_t f = v2h[s.seg_off[m] + (e - s.seg_pre[m])];
                        if (f == g1) continue;
                        if (P > 1 && part_of(f, P) != p) continue;
                        tab_insert(T1, f, 1u | (uint32_t(s.seg_inh[m]) << 16), 0, A.sc);
                    }
                    acc.n_v2h += (tid < tot) ? (tot - tid + NT - 1) / NT : 0;
                    if (!single) __syncthreads();
                }
                __syncthreads();
                const int n_t1 = min(s.n_t1, T1.list_cap);
                // (ii) open at g1: f in N(g1), not in N(h), not h
                if (want_open) {
                    for (int q = tid; q < n_t1; q += NT) {
                        const int sl = T1.list[q];
                        const int32_t f = T1.keys[sl];
                        if (f == h) continue;
                        if (tab_find(NH, f) >= 0) continue;
                        ++acc.n_meta;
                        if (f < h && bit_test(A.chg, f)) continue;
                        const int kf = S.h_card[f];
                        const int64_t tf = (fam & kFamT) ? S.h_ts[f] : 0;
                        classify(s, fam, delta, h, g1, f, kh, k1, kf, xh1, int(T1.vals[sl] & 0xffffu), 0, 0, tsh,
                                 ts1, tf, acc);
                    }
                }
                // (i) g2 in N(h) with g2 > g1: closed if g2 is in N(g1), else open at h
                for (int q = tid; q < n_nh; q += NT) {
                    const int sl2 = NH.list[q];
                    const int32_t g2 = NH.keys[sl2];
                    if (g2 <= g1) continue;
                    if (P > 1 && part_of(g2, P) != p) continue;
                    if (g2 < h && bit_test(A.chg, g2)) continue;
                    const int s1 = tab_find(T1, g2);
                    const uint32_t val = s1 >= 0 ? T1.vals[s1] : 0u;
                    const int x12 = int(val & 0xffffu), t = int(val >> 16);
                    if (x12 == 0 && !want_open) continue;
                    ++acc.n_meta;
                    const int xh2 = int(NH.vals[sl2]);
                    const int k2 = S.h_card[g2];
                    const int64_t t2 = (fam & kFamT) ? S.h_ts[g2] : 0;
                    if (want_open) classify(s, fam, delta, h, g1, g2, kh, k1, k2, xh1, x12, xh2, t, tsh, ts1, t2, acc);
                    if ((fam & kFamV) && x12 > 0)
                        acc.v3 += (unsigned long long)xh1 * x12 * xh2 - (unsigned long long)t * (xh1 + x12 + xh2) +
                                  2ull * t;
                }
                __syncthreads();
                tab_clear(T1, n_t1);
                __syncthreads();
                if (tid == 0) s.n_t1 = 0;
                __syncthreads();
            }
        }

        // ---- pairs {h, g} (type 2) and h itself (type 1), once per h
        if (chunk == 0 && (fam & kFamV)) {
            for (int q = tid; q < n_nh; q += NT) {
                const int sl = NH.list[q];
                const int32_t g2 = NH.keys[sl];
                if (g2 < h && bit_test(A.chg, g2)) continue;
                const unsigned long long x = NH.vals[sl];
                if (x >= 2) acc.v2 += (x * (x - 1) / 2) * (unsigned long long)(kh + S.h_card[g2] - 4);
            }
            if (tid == 0 && kh >= 3) acc.v1 += (unsigned long long)kh * (kh - 1) * (kh - 2) / 6;
        }

        // ---- fold the warp histograms, clear N(h)
        __syncthreads();
        for (int b = tid; b < kHistN; b += NT) {
            unsigned long long v = 0;
            for (int w = 0; w < NW; ++w) {
                v += s.hist[w][b];
                s.hist[w][b] = 0;
            }
            s.acc[b] += v;
        }
        tab_clear(NH, n_nh);
        __syncthreads();
        if (tid == 0) {
            s.n_nh = 0;
            s.n_cand = 0;
        }
    }
    __syncthreads();
    if (cur_g >= 0) flush(A, s, cur_g, acc);
    long long r0 = block_sum((long long)acc.n_v2h, s);
    long long r1 = block_sum((long long)acc.n_h2v, s);
    long long r2 = block_sum((long long)acc.n_meta, s);
    long long r3 = block_sum((long long)acc.n_tri, s);
    if (tid == 0) {
        atomicAdd(&A.sc->stats[0], (unsigned long long)r0);
        atomicAdd(&A.sc->stats[1], (unsigned long long)r1);
        atomicAdd(&A.sc->stats[2], (unsigned long long)r2);
        atomicAdd(&A.sc->stats[3], (unsigned long long)r3);
    }
}

// ---- work list: chunks of every changed hyperedge, then their prefix sum

__global__ void k_chunks(Store S, Scalars* sc, const int32_t* changed, int64_t lo, int64_t n, int32_t* chunks,
                         int64_t max_u) {
    int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int lane = lane_id();
    if (i >= n) return;
    if (sc->gate) {  // the call failed earlier: the changed list may hold invalid IDs
        if (lane == 0) chunks[i] = 1;
        return;
    }
    int32_t h = changed[lo + i];
    int k = S.h_card[h];
    const int32_t* m = S.hp.arena + S.h_off[h];
    long long u = 0;
    for (int t = lane; t < k; t += 32) u += S.v_deg[m[t]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (lane == 0) {
        if (u > max_u) set_error(sc, kErrUnsupported, -4, h, u);
        long long c = (u + CHUNK - 1) / CHUNK;
        chunks[i] = int32_t(c < 1 ? 1 : c);
    }
}

constexpr int kScanNT = 1024, kScanPer = 4, kScanBlock = kScanNT * kScanPer;

__global__ void k_scan_sums(const int32_t* in, int64_t n, int64_t* sums) {
    __shared__ int64_t red[kScanNT / 32];
    int64_t base = int64_t(blockIdx.x) * kScanBlock;
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

__global__ void k_scan_top(int64_t* sums, int64_t nb, int64_t* total_out) {
    if (threadIdx.x != 0) return;
    int64_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t v = sums[b];
        sums[b] = run;
        run += v;
    }
    *total_out = run;
}

__global__ void k_scan_apply(const int32_t* in, int64_t n, const int64_t* sums, int64_t* out) {
    __shared__ int64_t wsum[kScanNT / 32];
    int64_t base = int64_t(blockIdx.x) * kScanBlock;
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

__global__ void k_items_from_total(Scalars* sc, int side, const int64_t* item_start, int64_t n) {
    sc->items[side] = sc->gate ? 0 : item_start[n];
    sc->queue[side] = 0;
}

}  // namespace

size_t count_scratch_bytes(int64_t cap, int64_t g_slots, int n_cta) {
    int64_t regions = int64_t(n_cta) * 2;
    size_t b = 0;
    b += (cap + 1) * sizeof(int32_t);
    b += (cap + 2) * sizeof(int64_t);
    b += ((cap + kScanBlock - 1) / kScanBlock + 2) * sizeof(int64_t);
    b += regions * g_slots * (sizeof(int32_t) + sizeof(uint32_t) + sizeof(int32_t));
    b += regions * (g_slots / 2) * sizeof(int32_t);
    return b + 1024;
}

cudaError_t count_scratch_init(CountScratch* cs, void* mem, int64_t cap, int64_t g_slots, int n_cta,
                               cudaStream_t st) {
    auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
    char* p = static_cast<char*>(mem);
    size_t o = 0;
    int64_t regions = int64_t(n_cta) * 2;
    cs->cap = cap;
    cs->g_slots = g_slots;
    cs->n_cta = n_cta;
    cs->chunks = reinterpret_cast<int32_t*>(p + o);
    o = align(o + (cap + 1) * sizeof(int32_t));
    cs->item_start = reinterpret_cast<int64_t*>(p + o);
    o = align(o + (cap + 2) * sizeof(int64_t));
    cs->block_sums = reinterpret_cast<int64_t*>(p + o);
    o = align(o + ((cap + kScanBlock - 1) / kScanBlock + 2) * sizeof(int64_t));
    cs->g_keys = reinterpret_cast<int32_t*>(p + o);
    o = align(o + regions * g_slots * sizeof(int32_t));
    cs->g_vals = reinterpret_cast<uint32_t*>(p + o);
    o = align(o + regions * g_slots * sizeof(uint32_t));
    cs->g_aux = reinterpret_cast<int32_t*>(p + o);
    o = align(o + regions * g_slots * sizeof(int32_t));
    cs->g_list = reinterpret_cast<int32_t*>(p + o);
    cudaError_t e;
    if ((e = cudaMemsetAsync(cs->g_keys, 0xff, regions * g_slots * sizeof(int32_t), st))) return e;
    if ((e = cudaMemsetAsync(cs->g_vals, 0, regions * g_slots * sizeof(uint32_t), st))) return e;
    if ((e = cudaMemsetAsync(cs->g_aux, 0x7f, regions * g_slots * sizeof(int32_t), st))) return e;
    return cudaSuccess;
}

cudaError_t upload_tables(cudaStream_t st) {
    static ClassTables t;
    static bool built = false;
    if (!built) {
        build_class_tables(&t);
        built = true;
    }
    return cudaMemcpyToSymbolAsync(c_tables, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
}

cudaError_t count_launch(const Store& S, Scalars* sc, const int32_t* changed, const int32_t* changed_g,
                         const uint32_t* chg_bits, int64_t lo, int64_t hi, int side, uint64_t* dcounts_side,
                         const CountScratch& cs, int64_t max_u, cudaStream_t st, LaunchCounter& lc) {
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(Smem)));
        attr_done = true;
    }
    int64_t n = hi - lo;
    if (n <= 0) return cudaSuccess;
    if (n > cs.cap) return cudaErrorInvalidValue;
    unsigned gb = unsigned((n * 32 + 255) / 256);
    k_chunks<<<gb, 256, 0, st>>>(S, sc, changed, lo, n, cs.chunks, max_u);
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_sums<<<unsigned(nb), kScanNT, 0, st>>>(cs.chunks, n, cs.block_sums);
    k_scan_top<<<1, 32, 0, st>>>(cs.block_sums, nb, cs.block_sums + nb);
    k_scan_apply<<<unsigned(nb), kScanNT, 0, st>>>(cs.chunks, n, cs.block_sums, cs.item_start);
    k_items_from_total<<<1, 1, 0, st>>>(sc, side, cs.item_start, n);
    CountArgs A{S, sc, changed, changed_g, chg_bits, lo, hi, cs.item_start, side, dcounts_side,
                cs.g_keys, cs.g_vals, cs.g_aux, cs.g_list, cs.g_slots,
                uint32_t(cs.smem_slots < NH_S ? cs.smem_slots : NH_S),
                uint32_t(cs.smem_slots < T1_S ? cs.smem_slots : T1_S)};
    k_count<<<cs.n_cta, NT, sizeof(Smem), st>>>(A);
    lc.total += 6;
    lc.count += 1;
    return cudaGetLastError();
}

}  // namespace esc

// debug.cu -- the incidence store's invariants, checked on the device after
// every successful call of a graph or group created with esc_config.debug = 1
// (Table II's two views must describe the same hypergraph; Sec. III-B's
// deletion and insertion keep them so).  It reads the whole store, so it is
// for tests and for hunting a suspected race or slab-pool fault, not for
// production calls.  Checked, per graph g:
//   a hyperedge ID is live exactly when its size is non-zero, and a live one
//     lies below the graph's high-water mark;
//   a live hyperedge has 1..kMaxCard members, strictly increasing, all inside
//     the graph's vertex range;
//   every vertex's degree fits its v2h slab, and every entry of its list is
//     a live hyperedge of the same graph;
//   the sizes of the live hyperedges add up to the degrees of the vertices,
//     and the live hyperedges number n_live[g].
// A failed check records its code and two values in the call's status word.
#include "escher_internal.cuh"
#include "store_api.cuh"

namespace esc {

namespace {

constexpr int kDbgNT = 256;

__device__ __forceinline__ int graph_of(const int64_t* base, int n, int64_t x) {
    int lo = 0, hi = n;  // the last graph whose base is <= x
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kDbgNT) k_dbg_h(Store S, Scalars* sc, unsigned long long* acc) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t h = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; h < S.e_total; h += stride) {
        const bool live = bit_test(S.live, h);
        const int k = S.h_card[h];
        if (!live) {
            if (k != 0) set_error(sc, kErrInternal, -20, h, k);
            continue;
        }
        const int g = graph_of(S.ebase, S.n_graphs, h);
        if (h - S.ebase[g] >= S.ecap[g] || h - S.ebase[g] >= S.hw[g]) {
            set_error(sc, kErrInternal, -21, h, g);
            continue;
        }
        if (k < 1 || k > kMaxCard) {
            set_error(sc, kErrInternal, -22, h, k);
            continue;
        }
        const int32_t* m = S.hp.arena + S.h_off[h];
        const int64_t v0 = S.vbase[g], v1 = v0 + S.nv[g];
        for (int i = 0; i < k; ++i) {
            const int32_t v = m[i];
            if (v < v0 || v >= v1) set_error(sc, kErrInternal, -23, h, v);
            if (i > 0 && m[i - 1] >= v) set_error(sc, kErrInternal, -24, h, v);
        }
        atomicAdd(&acc[2 * g], (unsigned long long)k);
        atomicAdd(&acc[2 * g + 1], 1ull);
    }
}

// a warp per vertex, its lanes over the v2h list
__global__ void __launch_bounds__(kDbgNT) k_dbg_v(Store S, Scalars* sc, unsigned long long* acc) {
    const int lane = lane_id();
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t v = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; v < S.nv_total; v += nw) {
        const int d = S.v_deg[v], cap = S.v_cap[v];
        if (d < 0 || (d > 0 && d > cap)) {
            if (lane == 0) set_error(sc, kErrInternal, -25, v, d);
            continue;
        }
        const int g = graph_of(S.vbase, S.n_graphs, v);
        const int32_t* l = S.vp.arena + S.v_off[v];
        for (int e = lane; e < d; e += 32) {
            const int32_t h = l[e];
            if (h < 0 || h >= S.e_total || !bit_test(S.live, h)) {
                set_error(sc, kErrInternal, -26, v, h);
                continue;
            }
            if (graph_of(S.ebase, S.n_graphs, h) != g) set_error(sc, kErrInternal, -27, v, h);
        }
        if (lane == 0) atomicAdd(&acc[2 * S.n_graphs + g], (unsigned long long)d);
    }
}

__global__ void k_dbg_sum(Store S, Scalars* sc, const unsigned long long* acc) {
    for (int g = threadIdx.x; g < S.n_graphs; g += blockDim.x) {
        if (acc[2 * g] != acc[2 * S.n_graphs + g]) set_error(sc, kErrInternal, -28, g, int64_t(acc[2 * g]));
        if (int64_t(acc[2 * g + 1]) != S.n_live[g]) set_error(sc, kErrInternal, -29, g, int64_t(acc[2 * g + 1]));
    }
}

}  // namespace

cudaError_t store_debug_check(const Store& S, Scalars* sc, unsigned long long* acc, int sm_count, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 3 * size_t(S.n_graphs), st))) return e;
    k_dbg_h<<<unsigned(sm_count) * 4, kDbgNT, 0, st>>>(S, sc, acc);
    k_dbg_v<<<unsigned(sm_count) * 8, kDbgNT, 0, st>>>(S, sc, acc);
    k_dbg_sum<<<1, 256, 0, st>>>(S, sc, acc);
    return cudaGetLastError();
}

}  // namespace esc

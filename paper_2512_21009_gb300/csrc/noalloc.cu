// noalloc.cu -- esc_count_static_noalloc: triad counts of a static hypergraph
// computed without allocating any memory.
//
// Some callers cannot call cudaMalloc: code that owns a fixed memory budget
// handed out by its own allocator, or code in a process whose allocator must
// not be re-entered.  This entry point serves them.  The caller passes the
// inputs and the output; every temporary buffer (vertex->hyperedge lists,
// work lists, counter hash tables, status words) lives in one file-scope
// device array of fixed size, kNoAllocBytes, that every GPU which loads this
// library holds until the process exits.
//
// The call synchronises the stream it is given (it reads the member count and
// the status back to the host), so it returns only when the counts are
// written.
//
// The device address of that array is looked up once per device with
// cudaGetSymbolAddress, with the device current, on the first call made on
// that device.  All calls share the array and it keeps the last call's
// contents, so each call clears what must start at zero; calls whose GPU work
// overlaps (two streams, two host threads) race on it and must be serialised
// by the caller.
#include <mutex>
#include <string>

#include "escher.h"
#include "escher_internal.cuh"
#include "store_api.cuh"

namespace esc {
extern thread_local std::string t_create_error;  // api.cu: esc_last_error(NULL)

namespace {

constexpr int64_t kNAMaxHyperedges = int64_t(1) << 18;
constexpr int64_t kNAMaxIncidences = int64_t(1) << 21;
constexpr int64_t kNAMaxVertices = int64_t(1) << 19;
constexpr int kNABlocks = 64;           // blocks of each counting kernel
constexpr int64_t kNATableSlots = 2048; // per counter overflow table
constexpr int64_t kNAListEntries = int64_t(1) << 19;  // neighbour-list entries per counting run
constexpr size_t kNoAllocBytes = size_t(128) << 20;

CountShape na_shape() {
    CountShape sh;
    sh.cap = kNAMaxHyperedges;
    sh.list_cap = kNAListEntries;
    sh.e_cap = kNAMaxHyperedges;
    sh.gs_nh = sh.gs_c = kNATableSlots;
    sh.n_cta_nh = sh.n_cta_c = kNABlocks;
    sh.r_cap = 0;  // no restricted lists
    sh.with_ts = true;
    // no global sort scratch for long lists: their open triads at h are
    // classified pair by pair by the centre kernel (the fixed array holds
    // no room for it)
    sh.open_global = false;
    sh.c_per_sm = 2;
    return sh;
}

thread_local int64_t t_word;  // host word the counter reads back (pageable: no allocation)

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t sc, dc, card, ts, changed, chg, voff, vdeg, vfill, v2h, count, total;
};

Layout layout() {
    Layout L{};
    size_t o = 0;
    L.sc = o;      o = align256(o + sizeof(Scalars));
    L.dc = o;      o = align256(o + sizeof(uint64_t) * kCStride);
    L.card = o;    o = align256(o + sizeof(int32_t) * kNAMaxHyperedges);
    L.ts = o;      o = align256(o + sizeof(int64_t) * kNAMaxHyperedges);
    L.changed = o; o = align256(o + sizeof(int32_t) * kNAMaxHyperedges);
    L.chg = o;     o = align256(o + kNAMaxHyperedges / 8);
    L.voff = o;    o = align256(o + sizeof(int64_t) * (kNAMaxVertices + 1));
    L.vdeg = o;    o = align256(o + sizeof(int32_t) * kNAMaxVertices);
    L.vfill = o;   o = align256(o + sizeof(int32_t) * kNAMaxVertices);
    L.v2h = o;     o = align256(o + sizeof(int32_t) * kNAMaxIncidences);
    L.count = o;   o = align256(o + count_scratch_bytes(na_shape()));
    L.total = o;
    return L;
}

// Check every hyperedge (its offsets inside [0, nnz] and not decreasing,
// non-empty, at most kMaxCard members, members sorted ascending without
// repeats and inside [0, n_vertices)), record its size and count vertex
// degrees.  Members are read only once the offsets are known to lie inside
// the member array.
__global__ void k_na_check(const int64_t* off, const int32_t* mem, int64_t n, int64_t nnz, int32_t nv,
                           int32_t* card, int32_t* changed, int32_t* vdeg, Scalars* sc) {
    int64_t h = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (h >= n) return;
    int64_t a = off[h], b = off[h + 1];
    int64_t k = b - a;
    changed[h] = int32_t(h);
    if (a < 0 || b < a || b > nnz) {
        set_error(sc, kErrInvalid, -1, h, b);
        card[h] = 0;
        return;
    }
    if (k < 1 || k > kMaxCard) {
        set_error(sc, k < 1 ? kErrInvalid : kErrUnsupported, -1, h, k);
        card[h] = 0;
        return;
    }
    card[h] = int32_t(k);
    int32_t prev = -1;
    for (int64_t p = a; p < b; ++p) {
        int32_t v = mem[p];
        if (v < 0 || v >= nv || v <= prev) {
            set_error(sc, kErrInvalid, -1, h, v);
            return;
        }
        prev = v;
        atomicAdd(&vdeg[v], 1);
    }
}

// Exclusive prefix of the vertex degrees (one block; n <= kNAMaxVertices).
__global__ void k_na_scan(const int32_t* vdeg, int64_t n, int64_t* voff) {
    __shared__ int warp_tmp[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        int64_t i = base + threadIdx.x;
        int d = i < n ? vdeg[i] : 0;
        int tot;
        int pre = block_exclusive_scan<1024>(d, &tot, warp_tmp);
        if (i < n) voff[i] = carry + pre;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) voff[n] = carry;
}

__global__ void k_na_fill(const int64_t* off, const int32_t* mem, int64_t n, const int64_t* voff, int32_t* vfill,
                          int32_t* v2h, const Scalars* sc) {
    if (sc->status) return;
    int64_t h = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (h >= n) return;
    for (int64_t p = off[h]; p < off[h + 1]; ++p) {
        int32_t v = mem[p];
        v2h[voff[v] + atomicAdd(&vfill[v], 1)] = int32_t(h);
    }
}

__global__ void k_na_latch(Scalars* sc) { sc->gate = sc->status; }

__global__ void k_na_out(const uint64_t* dc, uint64_t* out, const Scalars* sc) {
    int i = threadIdx.x;
    if (i < kNCount) out[i] = sc->status ? 0 : dc[i];
}

// the reason of a failed call, for esc_last_error(NULL)
esc_status na_fail(esc_status s, const std::string& why) {
    t_create_error = "esc_count_static_noalloc: " + why;
    return s;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace esc

extern "C" esc_status esc_count_static_noalloc(int32_t n_vertices, int64_t n_he, const int64_t* offsets,
                                               const int32_t* members, const int64_t* timestamps,
                                               uint32_t families, int64_t delta, uint64_t* out_counts,
                                               void* cuda_stream) {
    using namespace esc;
    if (n_vertices <= 0 || n_he < 0 || !offsets || !out_counts || (n_he > 0 && !members))
        return na_fail(ESC_ERR_INVALID_ARG, "bad arguments");
    if (families == 0 || (families & ~7u) || delta < 0) return na_fail(ESC_ERR_INVALID_ARG, "bad families or delta");
    if (!on_device(offsets) || !on_device(out_counts) || (n_he > 0 && !on_device(members)) ||
        (timestamps && !on_device(timestamps)))
        return na_fail(ESC_ERR_INVALID_ARG, "inputs and output must be device memory");
    if (n_he > kNAMaxHyperedges) return na_fail(ESC_ERR_UNSUPPORTED, "more than 262,144 hyperedges");
    if (n_vertices > kNAMaxVertices) return na_fail(ESC_ERR_UNSUPPORTED, "more than 524,288 vertices");
    static_assert(sizeof(Scalars) < 4096, "layout");
    const Layout L = layout();
    if (L.total > kNoAllocBytes) return na_fail(ESC_ERR_UNSUPPORTED, "internal layout exceeds the scratch array");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return na_fail(ESC_ERR_CUDA, "no current device");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return na_fail(ESC_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
            }
            g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_scratch_ptr[dev];
    }
    // the member count is needed on the host to check the limit
    int64_t nnz = 0;
    if (n_he > 0) {
        if (cudaMemcpyAsync(&nnz, offsets + n_he, sizeof(int64_t), cudaMemcpyDefault, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return na_fail(ESC_ERR_CUDA, "reading offsets failed");
        int64_t first = 0;
        if (cudaMemcpyAsync(&first, offsets, sizeof(int64_t), cudaMemcpyDefault, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return na_fail(ESC_ERR_CUDA, "reading offsets failed");
        if (first != 0 || nnz < 0) return na_fail(ESC_ERR_INVALID_ARG, "offsets must start at 0");
        if (nnz > kNAMaxIncidences) return na_fail(ESC_ERR_UNSUPPORTED, "more than 2,097,152 incidences");
    }
    Scalars* sc = reinterpret_cast<Scalars*>(base + L.sc);
    uint64_t* dc = reinterpret_cast<uint64_t*>(base + L.dc);
    int32_t* card = reinterpret_cast<int32_t*>(base + L.card);
    int64_t* tsz = reinterpret_cast<int64_t*>(base + L.ts);
    int32_t* changed = reinterpret_cast<int32_t*>(base + L.changed);
    uint32_t* chg = reinterpret_cast<uint32_t*>(base + L.chg);
    int64_t* voff = reinterpret_cast<int64_t*>(base + L.voff);
    int32_t* vdeg = reinterpret_cast<int32_t*>(base + L.vdeg);
    int32_t* vfill = reinterpret_cast<int32_t*>(base + L.vfill);
    int32_t* v2h = reinterpret_cast<int32_t*>(base + L.v2h);
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    ok(cudaMemsetAsync(sc, 0, sizeof(Scalars), st));
    ok(cudaMemsetAsync(dc, 0, sizeof(uint64_t) * kCStride, st));
    ok(cudaMemsetAsync(vdeg, 0, sizeof(int32_t) * n_vertices, st));
    ok(cudaMemsetAsync(vfill, 0, sizeof(int32_t) * n_vertices, st));
    ok(cudaMemsetAsync(chg, 0xff, size_t((n_he + 31) / 32) * 4, st));
    if (!timestamps) ok(cudaMemsetAsync(tsz, 0, sizeof(int64_t) * (n_he > 0 ? n_he : 1), st));
    CountScratch cs;
    ok(count_scratch_init(&cs, base + L.count, na_shape(), &t_word, st));
    ok(upload_tables(st));
    if (e != cudaSuccess) return na_fail(ESC_ERR_CUDA, cudaGetErrorString(e));
    LaunchCounter lc;
    if (n_he > 0) {
        unsigned gb = unsigned((n_he + 255) / 256);
        k_na_check<<<gb, 256, 0, st>>>(offsets, members, n_he, nnz, n_vertices, card, changed, vdeg, sc);
        k_na_scan<<<1, 1024, 0, st>>>(vdeg, n_vertices, voff);
        k_na_fill<<<gb, 256, 0, st>>>(offsets, members, n_he, voff, vfill, v2h, sc);
        k_na_latch<<<1, 1, 0, st>>>(sc);
        Store S{};
        S.n_graphs = 1;
        S.nv_total = n_vertices;
        S.e_total = n_he;
        S.fam = families;
        S.delta = delta;
        S.h_off = const_cast<int64_t*>(offsets);
        S.h_card = card;
        S.h_ts = timestamps ? const_cast<int64_t*>(timestamps) : tsz;
        S.v_off = voff;
        S.v_deg = vdeg;
        S.hp.arena = const_cast<int32_t*>(members);
        S.vp.arena = v2h;
        ok(count_launch(S, sc, changed, nullptr, chg, 0, n_he, 1, dc, cs, count_max_u(na_shape()), st, lc));
    }
    k_na_out<<<1, 160, 0, st>>>(dc, out_counts, sc);
    ok(cudaGetLastError());
    Scalars h{};
    ok(cudaMemcpyAsync(&h, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    ok(cudaStreamSynchronize(st));
    if (e != cudaSuccess) return na_fail(ESC_ERR_CUDA, cudaGetErrorString(e));
    if (h.status != 0)
        return na_fail(esc_status(h.status), "device check " + std::to_string(h.detail[0]) + " failed (" +
                                                 std::to_string(h.detail[1]) + ", " + std::to_string(h.detail[2]) + ")");
    return ESC_OK;
}


/*
 * escher.h -- C ABI of the GB300 dynamic-hypergraph triad-count engine.
 *
 * The engine keeps hypergraphs resident on one GPU as a two-way incidence
 * store (hyperedge -> vertices, "h2v", and vertex -> hyperedges, "v2h"; paper
 * Section III, "Enabling Multiple Formats" and Table II), applies batches of
 * hyperedge insertions and deletions to it (Section III-B, vertical
 * operations), and after every batch refreshes three families of exact triad
 * counts incrementally from the hyperedges the batch touched (Algorithm 3):
 *
 *   ESC_TRIAD_HYPEREDGE  30 uint64: hyperedge triads by Venn pattern class
 *                        (Section II; the 26 classes of MoCHy, plus 4
 *                        classes that only arise when two hyperedges hold the
 *                        same vertex set).
 *   ESC_TRIAD_VERTEX     3 uint64: incident-vertex triads of types 1, 2, 3
 *                        (Section II): a vertex triple plus one witnessing
 *                        hyperedge per vertex pair, typed by the number of
 *                        distinct witnesses.
 *   ESC_TRIAD_TEMPORAL   96 uint64: temporal triads (Section II) -- three
 *                        connected hyperedges ordered by timestamp, equal
 *                        timestamps ordered by hyperedge ID, with
 *                        t_last - t_first <= delta -- by ordered pattern.
 *
 * Class numbering.  Venn region bits of an ordered triple (a,b,c): 0 a only,
 * 1 b only, 2 c only, 3 a&b not c, 4 b&c not a, 5 a&c not b, 6 a&b&c.  A
 * hyperedge class is the orbit of the 7-bit pattern under relabelling;
 * classes 0..25 are the orbits without two identical hyperedges ranked by
 * their smallest pattern, 26..29 the orbits with two identical hyperedges
 * ranked the same way.  A temporal class is the rank of the ordered pattern
 * (earliest hyperedge as a) among the 96 valid patterns.
 *
 * All counts are uint64 and wrap modulo 2^64.
 *
 * IDs.  Initial hyperedges get IDs 0..n-1 in input order.  In every batch the
 * deletions apply first; then the j-th inserted hyperedge (input order) takes
 * the j-th smallest free ID -- an ID below the high-water mark holding no
 * live hyperedge, including IDs freed by this batch -- and, once those run
 * out, fresh IDs upward from the high-water mark (Section III-B, insertion
 * Case 1 and Algorithm 2: a new hyperedge reuses a freed hyperedge's ID).
 * Vertex IDs lie in [0, n_vertices).  A hyperedge is a vertex set: repeated
 * members of an inserted hyperedge collapse to one (Section II).
 *
 * Pointers.  Every array argument may be a host pointer or a device pointer
 * of the graph's device; the library tells them apart itself.  Inputs are
 * borrowed for the duration of the call only.  Output arrays belong to the
 * caller.  A graph (or group) owns all the device memory it allocates until
 * it is destroyed.
 *
 * Errors.  Functions return an esc_status and never throw.  Every batch is
 * validated in full on the device before anything is changed: a failed
 * esc_apply_batch / esc_group_apply leaves the store and all counts as they
 * were.  esc_last_error() gives a one-line reason for the last failure.
 *
 * Threads.  A graph or group may be used by one host thread at a time.
 *
 * Environment switches, read when a graph or group is created.  They select
 * internal paths of the counter for tests and measurements; results are the
 * same exact counts whatever they are set to.  Unset (the default) is what the
 * library is tuned for.
 *   ESC_COUNT_ORIENT=0        count closed pairs with the earlier centre
 *                             kernel (both sides of every closed pair visited,
 *                             N(h) marked inside N(g1)) instead of searching
 *                             each closed pair once in (|g|, g) order.
 *   ESC_COUNT_LIST=n          neighbour-list arena of one count run, in
 *                             entries (>= 4096): a small arena forces several
 *                             runs per batch side.
 *   ESC_COUNT_TABLE_SLOTS=n   slots of the per-block overflow hash tables (a
 *                             power of two >= 1024).
 *   ESC_COUNT_SMEM_SLOTS=n    cap on shared-memory hash-table slots (a power
 *                             of two >= 64): small values force the
 *                             global-table, partitioned and in-place paths.
 *   ESC_COUNT_RPOOL=n         int32 entries of the restricted-list pool
 *                             (0, the default, disables restricted lists).
 *   ESC_COUNT_RMIN=n          neighbourhood size from which restricted lists
 *                             are built when the pool is enabled.
 *   ESC_COUNT_BIGNH=n         neighbourhood size (>= 16) above which N(h) gets
 *                             a hash table and a membership filter.
 *   ESC_COUNT_M1PCT=p         weight (percent) of a visit of N(g1) against a
 *                             visit of N(h) in the per-pair choice of which
 *                             side to scan.
 *   ESC_COUNT_OPEN_MAX=n      temporal family: longest N'(h) (0..65536)
 *                             whose open triads centred at h are counted from
 *                             its time order; longer ones have every pair
 *                             classified by the centre kernel.
 *   ESC_COUNT_OPEN_SMEM=n     temporal family: longest N'(h) (0..8192) sorted
 *                             in shared memory for that count; longer ones are
 *                             sorted in global scratch.
 *   ESC_CENTER_SMALL=s        centre-kernel launch shape, as
 *                             esc_tune_result.center_shape (0..3).
 *   ESC_CALL_GRAPH=1          graph launch on from creation (as
 *                             esc_set_graph_launch).
 *   ESC_STATS_JSONL=path      append one JSON line per call of every graph
 *                             or group created afterwards: call number,
 *                             batches, inserts, deletes, status, kernels
 *                             launched, and, with profiling on, the stage
 *                             times and counter work of esc_batch_stats.
 */
#ifndef ESCHER_H
#define ESCHER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ESC_OK = 0,
    ESC_ERR_INVALID_ARG = 1,   /* malformed input: bad sizes, vertex out of
                                  range, empty hyperedge, duplicate delete  */
    ESC_ERR_NOT_FOUND = 2,     /* delete of an ID that holds no live hyperedge */
    ESC_ERR_OUT_OF_MEMORY = 3, /* a preallocated capacity would be exceeded  */
    ESC_ERR_UNSUPPORTED = 4,   /* a size beyond a documented engine limit, a
                                  family not maintained, another window   */
    ESC_ERR_TIMEOUT = 5,       /* a bounded device wait ran out (reserved:
                                  no kernel of this build waits on the device,
                                  so no call returns it)                      */
    ESC_ERR_CUDA = 6,          /* a CUDA runtime call failed                 */
    ESC_ERR_BUSY = 7,          /* a server's queue is full; nothing was kept */
    ESC_ERR_INTERNAL = 8       /* debug mode: a store invariant was found
                                  broken after the call (esc_config.debug)   */
} esc_status;

typedef enum {
    ESC_TRIAD_HYPEREDGE = 0,
    ESC_TRIAD_VERTEX = 1,
    ESC_TRIAD_TEMPORAL = 2
} esc_triad_type;

#define ESC_FAMILY_HYPEREDGE 1u
#define ESC_FAMILY_VERTEX 2u
#define ESC_FAMILY_TEMPORAL 4u
/* Incident-vertex types 1 and 2 only, kept from vertex-pair statistics
 * (type 3 is not maintained and reads 0; esc_triads(ESC_TRIAD_VERTEX) gives
 * the three values).  With m_uv the number of hyperedges holding the vertex
 * pair {u, v} and S_uv the sum of their sizes, type 1 = sum over hyperedges
 * of C(|h|, 3) and type 2 = sum over vertex pairs of
 * (m_uv - 1) S_uv - 4 C(m_uv, 2) (Sec. II's types, this library's reading of
 * them); a batch costs the sum over its hyperedges of C(|h|, 2), whatever the
 * vertex degrees, so graphs with hub vertices stay cheap.  Needs
 * capacity_vertex_pairs > 0 and at most 2^24 hyperedge IDs; excludes
 * ESC_FAMILY_VERTEX.  esc_local_triads does not report it. */
#define ESC_FAMILY_VERTEX12 8u

#define ESC_N_HYPEREDGE_CLASSES 30
#define ESC_N_VERTEX_TYPES 3
#define ESC_N_TEMPORAL_CLASSES 96

/* Largest hyperedge cardinality the engine accepts (after duplicate members
 * are removed). */
#define ESC_MAX_CARDINALITY 16384

/* Capacities are preallocated once (paper Section IV: GPU memory is
 * preallocated with a tunable amount of slack so that updates need no
 * host-device round trips). */
typedef struct {
    int32_t n_vertices;             /* vertex universe [0, n_vertices)             */
    int64_t capacity_hyperedges;    /* IDs available: [0, capacity_hyperedges)     */
    int64_t capacity_incidences;    /* live (hyperedge, vertex) pairs, at most     */
    int64_t max_batch_hyperedges;   /* n_ins + n_del of one call, at most          */
    int64_t max_batch_incidences;   /* inserted members of one call, at most       */
    uint32_t families;              /* ESC_FAMILY_* bits of the families to keep   */
    int64_t delta;                  /* temporal window (timestamp units)           */
    int32_t debug;                  /* 1: after every successful call, check the
                                       store's invariants on the device (the two
                                       views agree, members sorted and in range,
                                       degrees within slabs, live counts); a
                                       violation fails the call with
                                       ESC_ERR_INTERNAL.  Reads the whole store:
                                       for tests.  0: off                          */
    int64_t capacity_vertex_pairs;  /* ESC_FAMILY_VERTEX12: distinct vertex pairs
                                       (pairs of members of one hyperedge) the
                                       graph may hold at once; 0 otherwise.  A
                                       batch whose inserted hyperedges could
                                       exceed it fails with OUT_OF_MEMORY        */
} esc_config;

typedef struct esc_graph esc_graph;
typedef struct esc_group esc_group;

/* Create a graph on the current CUDA device from an initial hypergraph of
 * n_he hyperedges in CSR form: the members of hyperedge i are
 * members[offsets[i] .. offsets[i+1]), offsets[0] == 0 (offsets int64[n_he+1],
 * members int32[offsets[n_he]], any order, repeats allowed).  timestamps is
 * int64[n_he] and required when ESC_FAMILY_TEMPORAL is kept, otherwise it
 * may be NULL.  All device work runs on cuda_stream (a cudaStream_t; NULL
 * for the legacy default stream).  The initial counts are computed on the
 * device by the same incremental kernels (every initial hyperedge counts as
 * inserted).  Paper Section III-B, "Hypergraph initialization".
 * Errors: INVALID_ARG (config or input malformed), OUT_OF_MEMORY (device
 * allocation or capacity), UNSUPPORTED (cardinality above
 * ESC_MAX_CARDINALITY), CUDA. */
esc_status esc_create(const esc_config* cfg, int64_t n_he, const int64_t* offsets,
                      const int32_t* members, const int64_t* timestamps, void* cuda_stream,
                      esc_graph** out);

/* Apply one batch: delete n_del hyperedges (del_ids int32[n_del], distinct,
 * live) and insert n_ins hyperedges (CSR as in esc_create; ins_timestamps
 * int64[n_ins], required when the temporal family is kept), then refresh
 * every kept count (Algorithm 3: counts of triads holding a deleted
 * hyperedge are removed on the old graph, counts of triads holding an
 * inserted hyperedge are added on the new graph).  If out_ins_ids is not
 * NULL it receives the n_ins assigned IDs (int32, input order).  The call
 * returns once the store and counts are updated.  Either count may be 0.
 * Errors: INVALID_ARG, NOT_FOUND, OUT_OF_MEMORY, UNSUPPORTED, CUDA; on any
 * error the graph is unchanged. */
esc_status esc_apply_batch(esc_graph* g, int64_t n_ins, const int64_t* ins_offsets,
                           const int32_t* ins_members, const int64_t* ins_timestamps,
                           int64_t n_del, const int32_t* del_ids, int32_t* out_ins_ids);

/* Horizontal update (Sec. III-B: incident vertices inserted into and deleted
 * from live hyperedges): live hyperedge ids[j] gets the vertex set
 * members[offsets[j] .. offsets[j+1]) (offsets int64[n+1], offsets[0] == 0;
 * repeated members collapse) and keeps its ID and timestamp.  All counts are
 * refreshed: every triad holding an updated hyperedge leaves its old class
 * and enters its new one.  ids: int32[n], distinct; pointers host or device.
 * Errors: INVALID_ARG (repeated ID, malformed sets), NOT_FOUND (an ID not
 * live), OUT_OF_MEMORY / UNSUPPORTED as esc_apply_batch; a failed call
 * changes nothing. */
esc_status esc_update_members(esc_graph* g, int64_t n, const int32_t* ids, const int64_t* offsets,
                              const int32_t* members);

/* Insert hyperedges under IDs the caller gives, e.g. to rebuild a graph from
 * esc_export's output: hyperedge j, with vertex set members[offsets[j] ..
 * offsets[j+1]) and timestamp timestamps[j], takes ID ids[j].  ids: int32[n],
 * distinct, each in [0, capacity_hyperedges) and not live.  timestamps:
 * int64[n], required when the temporal family is kept, else NULL means 0.
 * The new hyperedges' triads are counted as for esc_apply_batch's inserts
 * (Algorithm 3, inserted side).  Later inserts keep the ID rule over the IDs
 * left free (free IDs below the largest used one, smallest first, then fresh
 * ones), so IDs depend only on which IDs are live.  Pointers host or device.
 * Errors: INVALID_ARG (repeated or live ID, malformed sets, missing
 * timestamps), NOT_FOUND (an ID outside the range), OUT_OF_MEMORY and
 * UNSUPPORTED as esc_apply_batch; a failed call changes nothing. */
esc_status esc_insert_with_ids(esc_graph* g, int64_t n, const int32_t* ids, const int64_t* offsets,
                               const int32_t* members, const int64_t* timestamps);

/* Create a graph that holds a checkpointed state: esc_create with cfg and no
 * hyperedges, then the n_he hyperedges inserted under their IDs (the ids,
 * timestamps, offsets and members arrays of esc_export), in batches of at
 * most max_batch_hyperedges hyperedges and max_batch_incidences members.
 * The result has the exported graph's store, counts and future ID
 * assignment.  Errors as esc_create and esc_insert_with_ids; on failure
 * nothing is allocated, *out is NULL and esc_last_error(NULL) says why. */
esc_status esc_restore(const esc_config* cfg, int64_t n_he, const int32_t* ids, const int64_t* offsets,
                       const int32_t* members, const int64_t* timestamps, void* cuda_stream, esc_graph** out);

/* Copy the current counts of one family into out (uint64[n_out]; n_out must be
 * at least 30, 3 or 96).  window is the temporal window and must equal the
 * configured delta for ESC_TRIAD_TEMPORAL; it is ignored otherwise.
 * Errors: INVALID_ARG (n_out too small, bad type), UNSUPPORTED (family not
 * kept, other window). */
esc_status esc_triads(esc_graph* g, esc_triad_type type, int64_t window, uint64_t* out,
                      int32_t n_out);

/* Counts of the triads of the current graph that hold at least one of the
 * given live hyperedges (ids int32[n_ids], distinct), for every kept family;
 * out_hyperedge uint64[30], out_vertex uint64[3], out_temporal uint64[96]
 * (each may be NULL).  The type-1 and type-2 vertex counts attribute vertex
 * triples to the hyperedges and hyperedge pairs that witness them.  Passing
 * every live ID recounts the whole graph from scratch.  The graph is not
 * changed.  This is the counting step of Algorithm 3 on its own.
 * Errors: INVALID_ARG, NOT_FOUND, UNSUPPORTED, CUDA. */
esc_status esc_local_triads(esc_graph* g, int64_t n_ids, const int32_t* ids,
                            uint64_t* out_hyperedge, uint64_t* out_vertex,
                            uint64_t* out_temporal);

/* Release every resource of the graph.  NULL is accepted. */
esc_status esc_destroy(esc_graph* g);

/* One-line description of the last failure on this graph (or of the last
 * failed esc_create on this thread when g is NULL).  Owned by the library. */
const char* esc_last_error(const esc_graph* g);

/* Sizes needed by esc_export. */
esc_status esc_export_sizes(esc_graph* g, int64_t* n_live, int64_t* n_incidences);

/* Copy the incidence store to host arrays: for the n_live live hyperedges in
 * ascending ID order, ids int32[n_live], timestamps int64[n_live] (may be
 * NULL), offsets int64[n_live+1] and sorted members int32[n_incidences]; and,
 * for every vertex, v_offsets int64[n_vertices+1] and v_members
 * int32[n_incidences] holding the IDs of the hyperedges that contain it, in
 * ascending order.  Any pointer may be NULL to skip that part.  Meant for
 * tests and checkpoints (Table II: the h2v and v2h views); esc_restore
 * rebuilds a graph from the ids, timestamps, offsets and members arrays.
 * Errors: INVALID_ARG, CUDA. */
esc_status esc_export(esc_graph* g, int32_t* ids, int64_t* timestamps, int64_t* offsets,
                      int32_t* members, int64_t* v_offsets, int32_t* v_members);

/* The h2h mapping (Sec. III, Table II: the line graph, each hyperedge with the list
 * of hyperedges it is connected to): for the n_live live hyperedges in
 * ascending ID order (the order of esc_export), offsets int64[n_live+1] and
 * neighbours int32[n_entries] list the other live hyperedges that share at
 * least s vertices with it (s >= 1; s = 1 is the line graph, s > 1 the
 * s-line graph), ascending, and overlaps int32[n_entries] the number of
 * vertices shared.  *n_entries receives the total.  Any pointer may be NULL
 * (call once with neighbours NULL to size the arrays).  Assembled on the
 * host from a copy of the store: meant for small graphs and tests.
 * Errors: INVALID_ARG (s < 1), CUDA. */
esc_status esc_export_h2h(esc_graph* g, int32_t s, int64_t* n_entries, int64_t* offsets, int32_t* neighbours,
                          int32_t* overlaps);

/* Per-batch measurements of the last esc_apply_batch, filled when
 * esc_set_profiling(g, 1) is on.  Stage times are device times measured with
 * CUDA events on the graph's stream (the time split of the paper's Fig. 11b:
 * data-structure management versus count update). */
typedef struct {
    float ms_total;          /* whole batch                                   */
    float ms_ingest;         /* gather, sort/dedup, validation                 */
    float ms_count_del;      /* counting on the old graph (deleted side)       */
    float ms_store;          /* store update (delete + insert)                 */
    float ms_count_ins;      /* counting on the new graph (inserted side)      */
    int64_t launches;        /* kernels launched by the call                   */
    int64_t count_launches;  /* triad-count kernel launches                    */
    int64_t v2h_reads;       /* vertex->hyperedge entries read by the counter  */
    int64_t h2v_reads;       /* hyperedge->vertex entries read by the counter  */
    int64_t meta_reads;      /* per-neighbour metadata lookups by the counter  */
    int64_t triads;          /* triads classified by the counter               */
    int64_t alg_entries;     /* incidence entries the method reads for the
                                changed hyperedges (earlier accounting: for
                                each changed h, |h| + sum of its members'
                                degrees, plus, for each candidate neighbour
                                g1 of h, |g1| + sum of g1's members' degrees;
                                the four terms below replace it)             */
    int64_t work[6];         /* counter work: centre items, N(g1) build entries,
                                pair-pass visits, closed pairs, slow-path
                                triple-intersection steps, aggregate-pass visits */
    float ms_center;         /* device time of the centre kernel launches      */
    int32_t center_launches; /* centre kernel launches timed in ms_center      */
    int64_t alg_center;      /* the part of alg_entries read on behalf of the
                                candidate neighbours g1 (the centre kernel's
                                share: |g1| + sum of member degrees per pair)  */
    /* Algorithmic int32 entries (4 bytes each) of the batch by term: what a
     * method must read for the changed hyperedges, whatever it caches.     */
    int64_t alg_store;       /* store: 2 |h| + a 4-entry header per changed h */
    int64_t alg_build;       /* neighbourhoods: sum of the members' degrees
                                per changed h                                 */
    int64_t alg_closed;      /* closed pairs: min(|g1|, |g2|) per closed pair
                                {g1, g2} of N(h) counted                      */
    int64_t alg_open;        /* open paths: sum of g1's members' degrees per
                                pair (h, g1), g1 a candidate neighbour of h   */
} esc_batch_stats;

esc_status esc_set_profiling(esc_graph* g, int32_t on);
esc_status esc_last_stats(esc_graph* g, esc_batch_stats* out);

/* Total kernel launches of this graph so far (a monotone counter). */
int64_t esc_launch_count(const esc_graph* g);

/* ------------------------------------------------------------------------
 * Groups: many independent hypergraphs behind one store, updated together.
 *
 * A group holds n_graphs hypergraphs with the same families and delta.  One
 * esc_group_apply call takes update batches for any subset of them and runs
 * the whole pipeline -- validation, store update, triad counting -- for all
 * of them in the same kernel launches, the counting work of every graph
 * balanced across the GPU together.  Triads never span two graphs.  Each
 * graph has its own ID space, vertex universe, high-water mark and counts,
 * exactly as if it were an esc_graph of its own.  Batches are all-or-nothing
 * per call: if any batch is invalid, no graph changes.
 * ------------------------------------------------------------------------ */

typedef struct {
    int32_t graph;                  /* which graph of the group                    */
    int64_t n_ins;
    const int64_t* ins_offsets;     /* int64[n_ins+1], offsets[0] == 0            */
    const int32_t* ins_members;
    const int64_t* ins_timestamps;  /* int64[n_ins] or NULL when not temporal     */
    int64_t n_del;
    const int32_t* del_ids;         /* int32[n_del], this graph's IDs             */
    int32_t* out_ins_ids;           /* int32[n_ins] or NULL                       */
} esc_batch;

/* Create a group of empty graphs; graph_cfg[i] gives graph i's n_vertices,
 * capacity_hyperedges and capacity_incidences; families, delta and the
 * per-call batch limits come from shared_cfg.  Errors: INVALID_ARG,
 * OUT_OF_MEMORY, CUDA. */
esc_status esc_group_create(const esc_config* shared_cfg, int32_t n_graphs,
                            const esc_config* graph_cfg, void* cuda_stream, esc_group** out);

/* Device bytes that esc_group_create would allocate for the same arguments
 * (a sizing pass: nothing is allocated, no kernel runs).  A caller admits
 * graphs while this figure stays within the free device memory
 * (cudaMemGetInfo) or its own budget.  Errors: INVALID_ARG, UNSUPPORTED,
 * CUDA (no device). */
esc_status esc_group_bytes(const esc_config* shared_cfg, int32_t n_graphs, const esc_config* graph_cfg,
                           int64_t* out_bytes);

/* Apply n batches (each graph at most once per call) in one pass.  Returns
 * when every store and count is updated.  Errors as esc_apply_batch; the
 * failing batch is named by esc_group_last_error. */
esc_status esc_group_apply(esc_group* grp, int32_t n, const esc_batch* batches);

/* esc_update_members for graph `graph` of the group (that graph's IDs). */
esc_status esc_group_update_members(esc_group* grp, int32_t graph, int64_t n, const int32_t* ids,
                                    const int64_t* offsets, const int32_t* members);

/* esc_insert_with_ids for graph `graph` of the group (that graph's IDs); one
 * call, so n and the members must fit the group's batch limits. */
esc_status esc_group_insert_with_ids(esc_group* grp, int32_t graph, int64_t n, const int32_t* ids,
                                     const int64_t* offsets, const int32_t* members, const int64_t* timestamps);

/* esc_export_sizes / esc_export for graph `graph` of the group, in that
 * graph's own hyperedge and vertex IDs. */
esc_status esc_group_export_sizes(esc_group* grp, int32_t graph, int64_t* n_live, int64_t* n_incidences);
esc_status esc_group_export(esc_group* grp, int32_t graph, int32_t* ids, int64_t* timestamps, int64_t* offsets,
                            int32_t* members, int64_t* v_offsets, int32_t* v_members);
esc_status esc_group_export_h2h(esc_group* grp, int32_t graph, int32_t s, int64_t* n_entries, int64_t* offsets,
                                int32_t* neighbours, int32_t* overlaps);

esc_status esc_group_triads(esc_group* grp, int32_t graph, esc_triad_type type, int64_t window,
                            uint64_t* out, int32_t n_out);
esc_status esc_group_destroy(esc_group* grp);
const char* esc_group_last_error(const esc_group* grp);
esc_status esc_group_set_profiling(esc_group* grp, int32_t on);
esc_status esc_group_last_stats(esc_group* grp, esc_batch_stats* out);
int64_t esc_group_launch_count(const esc_group* grp);

/* ------------------------------------------------------------------------
 * Serving loop over a group's resident graphs.  The paper applies one batch
 * at a time (Alg. 3); the server adds the request layer around that step:
 * update requests (one batch for one graph) are queued as they arrive, and
 * a worker thread per group applies them by continuous batching -- each call
 * takes the oldest pending request of as many distinct graphs of the group
 * as fit its max_batch_hyperedges / max_batch_incidences (and
 * max_batches_per_call when > 0), so that requests arriving during a call
 * join the next one.  Requests of one graph are applied in submission order,
 * so a graph's IDs and counts are those of its batches applied one by one
 * with esc_group_apply.  A server starts with one group and takes more while
 * it runs (esc_server_add_group); the workers of different groups make their
 * calls at the same time, each on its own group's stream, so that one
 * group's ingest, store update and counting overlap another's on the device.
 * Graphs are numbered server-wide: the graphs of the first group, then those
 * of each group added, in the order added.
 * ------------------------------------------------------------------------ */
typedef struct esc_server esc_server;

typedef struct {
    int32_t status;        /* esc_status of the request                              */
    int32_t call_batches;  /* requests applied by the same call                      */
    int64_t t_arrival_ns;  /* CLOCK_MONOTONIC times (ns): arrival, call start, done  */
    int64_t t_start_ns;
    int64_t t_done_ns;
    int64_t call_updates;  /* inserts + deletes applied by the same call             */
} esc_request_info;

typedef struct {
    int64_t submitted, rejected, completed, failed;
    int64_t calls;    /* esc_group_apply calls made by the worker (retries of a failed call not counted) */
    int64_t updates;  /* inserts + deletes of completed requests                              */
    int64_t pending_updates;  /* inserts + deletes of submitted, unfinished requests          */
} esc_server_stats;

/* Start a server on grp.  While it runs, the group must not be used except
 * through the server.  max_pending_updates bounds the inserts + deletes of
 * submitted, unfinished requests (admission: a submit beyond it returns
 * ESC_ERR_BUSY); max_batches_per_call 0 = as many as fit, 1 = one request
 * per call.  Errors: INVALID_ARG. */
esc_status esc_server_create(esc_group* grp, int64_t max_pending_updates, int32_t max_batches_per_call,
                             esc_server** out);

/* Add a group of resident graphs (created and loaded by the caller) to a
 * running server; its graphs become the server's graphs *first_graph ..
 * *first_graph + n_graphs - 1 (first_graph may be NULL).  From then on the
 * group must only be used through the server.  For calls that overlap on
 * the device, create each group on its own stream.  Errors: INVALID_ARG
 * (the group is already served, or the server is stopping). */
esc_status esc_server_add_group(esc_server* srv, esc_group* grp, int32_t* first_graph);

/* Admission by free device memory: *fits = 1 when a group of the given
 * configuration (esc_group_bytes) fits in the current device's free memory
 * (cudaMemGetInfo) less reserve_bytes, else 0.  Nothing is allocated.
 * Errors: INVALID_ARG, CUDA. */
esc_status esc_group_fits(const esc_config* shared_cfg, int32_t n_graphs, const esc_config* graph_cfg,
                          int64_t reserve_bytes, int32_t* fits);

/* Queue one request.  All pointers are host memory and are copied before
 * the call returns, except out_ins_ids (host int32[n_ins] or NULL), which
 * receives the inserted IDs before the request is reported done and must
 * stay valid until then.  t_arrival_ns: CLOCK_MONOTONIC time of arrival in
 * ns (0: now), used for the request's latency.  *ticket identifies the
 * request for esc_server_wait.  Errors: INVALID_ARG (bad graph, empty
 * request, device pointers, offsets not starting at 0), OUT_OF_MEMORY (the
 * request alone exceeds the per-call limits), BUSY (queue full). */
esc_status esc_server_submit(esc_server* srv, const esc_batch* batch, int64_t t_arrival_ns, int64_t* ticket);

/* Block until request `ticket` is done; fill *info (may be NULL) and return
 * the request's own status.  Each ticket is collected once; a second wait
 * returns NOT_FOUND.  A request that fails changes nothing in its graph
 * (the worker applies the requests of a failed call one by one). */
esc_status esc_server_wait(esc_server* srv, int64_t ticket, esc_request_info* info);

/* Block until every submitted request is done. */
esc_status esc_server_drain(esc_server* srv);

/* esc_group_triads of a server graph, through the server (serialised with
 * the calls of that graph's worker). */
esc_status esc_server_triads(esc_server* srv, int32_t graph, esc_triad_type type, int64_t window,
                             uint64_t* out, int32_t n_out);

esc_status esc_server_get_stats(esc_server* srv, esc_server_stats* out);

/* Finish every queued request, stop the workers and free the server (not
 * the groups). */
esc_status esc_server_destroy(esc_server* srv);

/* Allocation-free counting.  The paper has no counterpart of this call; it
 * exists for callers that cannot allocate device memory -- code confined to a
 * memory budget handed out by its own allocator, or code whose allocator must
 * not be re-entered -- and so cannot use esc_create.
 *
 * Counts every triad of one static hypergraph: n_he hyperedges in CSR form
 * (offsets int64[n_he+1] with offsets[0] == 0; members int32[offsets[n_he]],
 * each hyperedge's members sorted ascending without repeats, vertex IDs in
 * [0, n_vertices)); timestamps int64[n_he] or NULL (all zero).  families and
 * delta as in esc_config.  out_counts receives uint64[129]: 30 hyperedge
 * classes, then the 3 vertex types, then the 96 temporal classes (families
 * not asked for read 0, and all 129 read 0 after an error).  Hyperedge i
 * has ID i.  Every pointer must be device memory of the current device; the
 * call runs on cuda_stream, synchronises it (it reads the member count and
 * its status back) and returns once out_counts is written.
 *
 * It calls no cudaMalloc or cudaFree: its temporary buffers live in one
 * fixed array of device memory (128 MiB) that every GPU which loads the
 * library holds until the process exits.  The first call on a device looks
 * up that array's device address.  All calls share the array and every call
 * resets what it needs, so calls whose GPU work overlaps race on it:
 * serialise them.
 *
 * Limits: n_he <= 262,144; offsets[n_he] <= 2,097,152; n_vertices <=
 * 524,288; each hyperedge at most ESC_MAX_CARDINALITY members; for every
 * hyperedge, the sum of its members' degrees at most 65,536.
 * Errors: INVALID_ARG (bad arguments, host pointers, malformed hypergraph),
 * UNSUPPORTED (a limit exceeded), CUDA. */
esc_status esc_count_static_noalloc(int32_t n_vertices, int64_t n_he, const int64_t* offsets,
                                    const int32_t* members, const int64_t* timestamps, uint32_t families,
                                    int64_t delta, uint64_t* out_counts, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Graph launch.  With it on, every call of the graph (or group) replays one
 * CUDA graph holding the whole device work of a call -- ingest, both counts,
 * store update, fold -- captured at the first call: its kernels read the
 * call's sizes on the device and plan the count runs there, so the same graph
 * serves calls of any size within the configured limits.  A call whose
 * neighbour lists do not fit one count run per side (the arena holds 512
 * entries per batch hyperedge) is detected inside the graph before anything
 * changes and is run again without the graph.  Results
 * are identical either way; what changes is the host's launch work per call.
 * A graph created on the legacy default stream moves to a stream of its own
 * (calls still return only when done).  Errors: INVALID_ARG, CUDA.
 * ------------------------------------------------------------------------ */
esc_status esc_set_graph_launch(esc_graph* g, int32_t on);
esc_status esc_group_set_graph_launch(esc_group* grp, int32_t on);

/* ------------------------------------------------------------------------
 * Work split of one hypergraph across ranks (one process per GPU).  The
 * paper runs on one GPU; this is how the count of one graph spreads over
 * several.  Every rank creates the same graph and applies the same batches
 * (the ID rule is deterministic, so the replicas stay identical); after
 * esc_set_split(g, rank, world) each rank counts only its share of every
 * batch's changed hyperedges: per side (deleted, inserted), the contiguous
 * range of them whose neighbourhood sizes (sum of member degrees, plus one
 * each) fall in the rank's equal part of the side's total.  Algorithm 3's
 * count change is a sum over the changed hyperedges, each triad counted at
 * its changed member of smallest ID, so the shares of the ranks add up to
 * the whole change.  From the call on, esc_triads / esc_group_triads return
 * this rank's share: the counts are the sum of the shares over all ranks,
 * modulo 2^64 (one all-reduce of at most 129 uint64 per family read).  Rank
 * 0 keeps the counts held at the call; the other ranks' shares start at
 * zero.  esc_local_triads still returns whole counts.  The split is set once
 * per graph and needs graph launch off (esc_set_graph_launch then refuses
 * to turn it on).  world >= 2, 0 <= rank < world.
 * Errors: INVALID_ARG, UNSUPPORTED (already split, or graph launch on), CUDA.
 * ------------------------------------------------------------------------ */
esc_status esc_set_split(esc_graph* g, int32_t rank, int32_t world);
esc_status esc_group_set_split(esc_group* grp, int32_t rank, int32_t world);

/* ------------------------------------------------------------------------
 * Autotuning.  Timed on the graph's own data -- the triads holding a sample
 * of live hyperedges (ids: that graph's IDs, host or device memory) are
 * counted and discarded, `reps` timed runs per candidate after one warm-up
 * run -- the fastest candidate of each choice is kept for later calls:
 *   1. the counter's launch shape (centre blocks per SM x threads: 0: 1 x 512,
 *      1: 2 x 256, 2: 2 x 512, 3: 3 x 256) and, without the temporal family,
 *      whether large neighbourhoods get restricted incidence lists;
 *   2. with that shape, the intersection strategy by neighbourhood size: the
 *      N(h) size from which N(h) gets a hash table and a membership filter
 *      (below it a pair (h, g1) can only scan N(h) against N(g1)'s table;
 *      above it, it may probe N(h)'s filter and table with N(g1)'s list
 *      instead) -- 256, 512 or 1024 entries;
 *   3. with those, the weight of a visit of N(g1) against a visit of N(h) in
 *      that per-pair choice -- 50%, 100% or 200%.
 * Counts and store are left unchanged.  The paper fixes no such choice; it
 * is a property of this implementation.  Errors: INVALID_ARG, NOT_FOUND (an
 * ID not live), CUDA.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t center_shape;  /* the chosen shape, 0..3 as above                    */
    int32_t restricted;    /* 1: restricted lists chosen                          */
    float ms[8];           /* best time of each candidate: shapes 0..3 without,
                              then with restricted lists (-1: not run)            */
    int32_t table_from;    /* the chosen N(h) size for a table and filter         */
    int32_t m1_pct;        /* the chosen weight of an N(g1) visit, percent        */
    float ms_table[3];     /* best time with table_from 256, 512, 1024            */
    float ms_m1[3];        /* best time with m1_pct 50, 100, 200                  */
} esc_tune_result;

esc_status esc_autotune(esc_graph* g, int64_t n_ids, const int32_t* ids, int32_t reps, esc_tune_result* out);
esc_status esc_group_autotune(esc_group* grp, int32_t graph, int64_t n_ids, const int32_t* ids, int32_t reps,
                              esc_tune_result* out);

/* Library version string. */
const char* esc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ESCHER_H */

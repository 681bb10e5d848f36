/*
 * escher_oracle.c -- plain, slow, CPU reference for hypergraph triad counts.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU baseline of the
 * benchmark use it.  It shares no code, header or table with the CUDA
 * library: every class table below is enumerated here from the definitions.
 *
 * What it computes (paper Section II, "Hypergraph Triads"):
 *
 *  - Hyperedge triads (MoCHy h-motifs, Section II, first item): an unordered
 *    triple {a,b,c} of distinct live hyperedges in which at least two of the
 *    three pairwise intersections are non-empty.  Its pattern is which of the
 *    seven Venn regions of (a,b,c) are non-empty; its class is the pattern up
 *    to relabelling of a,b,c.  Without identical hyperedges there are 26
 *    classes (the paper's "26 unique hypergraph triads"); identical vertex
 *    sets can occur in a dynamic multiset of hyperedges and add 4 classes, so
 *    30 counters are kept.
 *  - Incident-vertex triads (Section II, second item; types of StatHyper): a
 *    vertex triple {u,v,w} together with one witnessing hyperedge for each of
 *    its three vertex pairs; the type is the number of distinct hyperedges in
 *    the witness assignment (1, 2 or 3).
 *  - Temporal triads (Section II, third item): three connected hyperedges
 *    ordered by time, t_i < t_j < t_k with t_k - t_i <= delta; the class is
 *    the ordered pattern (earliest hyperedge first).  Equal timestamps are
 *    ordered by hyperedge ID.  There are 96 ordered patterns.
 *
 * Class numbering (a convention of this project, identical on both sides):
 *   region bits: 0 a-only, 1 b-only, 2 c-only, 3 (a&b)\c, 4 (b&c)\a,
 *                5 (a&c)\b, 6 a&b&c.
 *   static index:   orbits without two identical hyperedges, ranked by their
 *                   smallest mask (0..25); then orbits with two identical
 *                   hyperedges ranked the same way (26..29).
 *   temporal index: rank of the ordered mask among the 96 valid masks.
 *
 * Every count is an exact uint64; a true value of 2^64 or more is reported as
 * an error (ORC_ERR_OVERFLOW) instead of wrapping.
 *
 * Inputs: n hyperedges in CSR form (off[n+1], mem[off[n]]) whose member lists
 * are sorted ascending without repeats, their IDs (ids[n], used only to order
 * equal timestamps and to name hyperedges) and timestamps (ts[n], may be NULL
 * when the temporal family is not asked for).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INPUT 1
#define ORC_ERR_OVERFLOW 2
#define ORC_ERR_NOMEM 3

#define FAM_HYPEREDGE 1u
#define FAM_VERTEX 2u
#define FAM_TEMPORAL 4u

/* ------------------------------------------------------------------------ */
/* Venn regions                                                              */
/* ------------------------------------------------------------------------ */

/* A region is named by which of the three sets contain it.  The membership
 * triple (in_a, in_b, in_c) of each region index: */
static const int REGION_MEMBERSHIP[7][3] = {
    {1, 0, 0}, /* 0: a only          */
    {0, 1, 0}, /* 1: b only          */
    {0, 0, 1}, /* 2: c only          */
    {1, 1, 0}, /* 3: a and b, not c  */
    {0, 1, 1}, /* 4: b and c, not a  */
    {1, 0, 1}, /* 5: a and c, not b  */
    {1, 1, 1}, /* 6: all three       */
};

static int region_of(int in_a, int in_b, int in_c) {
    for (int r = 0; r < 7; ++r)
        if (REGION_MEMBERSHIP[r][0] == in_a && REGION_MEMBERSHIP[r][1] == in_b &&
            REGION_MEMBERSHIP[r][2] == in_c)
            return r;
    return -1;
}

/* Sizes of the seven Venn regions of three sorted sets, by walking their
 * union once and recording which sets hold each vertex. */
static void venn_sizes(const int32_t* a, int64_t na, const int32_t* b, int64_t nb,
                       const int32_t* c, int64_t nc, int64_t size[7]) {
    int64_t i = 0, j = 0, k = 0;
    for (int r = 0; r < 7; ++r) size[r] = 0;
    for (;;) {
        int64_t m = INT64_MAX;
        if (i < na && a[i] < m) m = a[i];
        if (j < nb && b[j] < m) m = b[j];
        if (k < nc && c[k] < m) m = c[k];
        if (m == INT64_MAX) break;
        int ia = (i < na && a[i] == m), ib = (j < nb && b[j] == m), ic = (k < nc && c[k] == m);
        size[region_of(ia, ib, ic)]++;
        i += ia; j += ib; k += ic;
    }
}

/* Pattern mask of the region sizes when the three sets are relabelled:
 * new label 0 is old set p[0], new label 1 is old p[1], new label 2 old p[2]. */
static int mask_under(const int64_t size[7], const int p[3]) {
    int mask = 0;
    for (int r = 0; r < 7; ++r) {
        if (size[r] == 0) continue;
        const int* m = REGION_MEMBERSHIP[r];
        mask |= 1 << region_of(m[p[0]], m[p[1]], m[p[2]]);
    }
    return mask;
}

static const int PERMS[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

/* ------------------------------------------------------------------------ */
/* Class tables, enumerated from the definitions                             */
/* ------------------------------------------------------------------------ */

static int g_tables_ready = 0;
static int g_static_of_mask[128];   /* -1: not a triad pattern */
static int g_temporal_of_mask[128]; /* -1: not a triad pattern */
static int g_static_rep[30];
static int g_static_closed[30];
static int g_static_dup[30];
static int g_temporal_mask[96];
static int g_n_static, g_n_static_nodup, g_n_temporal;

/* Facts about a mask read through region membership: set s non-empty, sets
 * s and t intersect, sets s and t identical. */
static int set_nonempty(int mask, int s) {
    for (int r = 0; r < 7; ++r)
        if ((mask >> r & 1) && REGION_MEMBERSHIP[r][s]) return 1;
    return 0;
}
static int sets_meet(int mask, int s, int t) {
    for (int r = 0; r < 7; ++r)
        if ((mask >> r & 1) && REGION_MEMBERSHIP[r][s] && REGION_MEMBERSHIP[r][t]) return 1;
    return 0;
}
static int sets_equal(int mask, int s, int t) {
    for (int r = 0; r < 7; ++r)
        if ((mask >> r & 1) && REGION_MEMBERSHIP[r][s] != REGION_MEMBERSHIP[r][t]) return 0;
    return 1;
}
static int is_triad_mask(int mask) {
    if (!set_nonempty(mask, 0) || !set_nonempty(mask, 1) || !set_nonempty(mask, 2)) return 0;
    int meets = sets_meet(mask, 0, 1) + sets_meet(mask, 1, 2) + sets_meet(mask, 0, 2);
    return meets >= 2;
}
static int has_identical_pair(int mask) {
    return sets_equal(mask, 0, 1) || sets_equal(mask, 1, 2) || sets_equal(mask, 0, 2);
}
static int canonical_mask(int mask) {
    /* relabel a mask: region r of the relabelled triple holds the vertices of
     * the region whose membership, read through the permutation, is r's */
    int best = 128;
    for (int q = 0; q < 6; ++q) {
        int out = 0;
        for (int r = 0; r < 7; ++r) {
            if (!(mask >> r & 1)) continue;
            const int* m = REGION_MEMBERSHIP[r];
            out |= 1 << region_of(m[PERMS[q][0]], m[PERMS[q][1]], m[PERMS[q][2]]);
        }
        if (out < best) best = out;
    }
    return best;
}

static void build_tables(void) {
    if (g_tables_ready) return;
    int reps_nodup[128], reps_dup[128], n_nodup = 0, n_dup = 0;
    for (int m = 0; m < 128; ++m) {
        g_static_of_mask[m] = -1;
        g_temporal_of_mask[m] = -1;
    }
    g_n_temporal = 0;
    for (int m = 0; m < 128; ++m) {
        if (!is_triad_mask(m)) continue;
        g_temporal_mask[g_n_temporal] = m;
        g_temporal_of_mask[m] = g_n_temporal++;
        if (canonical_mask(m) != m) continue; /* m is the smallest mask of its orbit */
        if (has_identical_pair(m)) reps_dup[n_dup++] = m;
        else reps_nodup[n_nodup++] = m;
    }
    /* masks were visited in ascending order, so both lists are sorted */
    g_n_static = 0;
    for (int i = 0; i < n_nodup; ++i) g_static_rep[g_n_static++] = reps_nodup[i];
    for (int i = 0; i < n_dup; ++i) g_static_rep[g_n_static++] = reps_dup[i];
    g_n_static_nodup = n_nodup;
    for (int i = 0; i < g_n_static; ++i) {
        int r = g_static_rep[i];
        g_static_closed[i] = sets_meet(r, 0, 1) && sets_meet(r, 1, 2) && sets_meet(r, 0, 2);
        g_static_dup[i] = i >= n_nodup;
    }
    for (int m = 0; m < 128; ++m) {
        if (!is_triad_mask(m)) continue;
        int c = canonical_mask(m);
        for (int i = 0; i < g_n_static; ++i)
            if (g_static_rep[i] == c) g_static_of_mask[m] = i;
    }
    g_tables_ready = 1;
}

int orc_num_static_classes(void) { build_tables(); return g_n_static; }
int orc_num_static_classes_nodup(void) { build_tables(); return g_n_static_nodup; }
int orc_num_temporal_classes(void) { build_tables(); return g_n_temporal; }
int orc_static_rep(int idx) { build_tables(); return (idx >= 0 && idx < g_n_static) ? g_static_rep[idx] : -1; }
int orc_static_closed(int idx) { build_tables(); return (idx >= 0 && idx < g_n_static) ? g_static_closed[idx] : -1; }
int orc_static_dup(int idx) { build_tables(); return (idx >= 0 && idx < g_n_static) ? g_static_dup[idx] : -1; }
int orc_static_class_of_mask(int m) { build_tables(); return (m >= 0 && m < 128) ? g_static_of_mask[m] : -1; }
int orc_temporal_class_of_mask(int m) { build_tables(); return (m >= 0 && m < 128) ? g_temporal_of_mask[m] : -1; }
int orc_temporal_mask(int idx) { build_tables(); return (idx >= 0 && idx < g_n_temporal) ? g_temporal_mask[idx] : -1; }

/* ------------------------------------------------------------------------ */
/* helpers                                                                   */
/* ------------------------------------------------------------------------ */

static int add_u64(uint64_t* acc, uint64_t v) {
    return __builtin_add_overflow(*acc, v, acc) ? ORC_ERR_OVERFLOW : ORC_OK;
}

static int check_csr(int64_t n, const int64_t* off, const int32_t* mem) {
    if (n < 0 || !off) return ORC_ERR_INPUT;
    if (n > 0 && !mem && off[n] > 0) return ORC_ERR_INPUT;
    if (off[0] != 0) return ORC_ERR_INPUT;
    for (int64_t i = 0; i < n; ++i) {
        if (off[i + 1] < off[i]) return ORC_ERR_INPUT;
        for (int64_t p = off[i] + 1; p < off[i + 1]; ++p)
            if (mem[p] <= mem[p - 1]) return ORC_ERR_INPUT; /* sorted, no repeats */
        for (int64_t p = off[i]; p < off[i + 1]; ++p)
            if (mem[p] < 0) return ORC_ERR_INPUT;
    }
    return ORC_OK;
}

/* Does hyperedge i come before hyperedge j in time (timestamp, then ID)? */
static int before(const int64_t* ts, const int32_t* ids, int64_t i, int64_t j) {
    if (ts[i] != ts[j]) return ts[i] < ts[j];
    return ids[i] < ids[j];
}

/* The vertex family is counted in vertex space by its own routines below;
 * the hyperedge-triple walkers only feed the hyperedge and temporal families. */
typedef struct {
    uint32_t fam;
    int64_t delta;
    const int64_t* ts;
    const int32_t* ids;
    uint64_t* h30;
    uint64_t* t96;
} counters;

/* Classify one connected triple (positions a, b, c) into every requested
 * family.  `size` are its Venn region sizes with the labels (a, b, c). */
static int record_triad(counters* C, int64_t a, int64_t b, int64_t c, const int64_t size[7]) {
    int rc = ORC_OK;
    if (C->fam & FAM_HYPEREDGE) {
        int best = 128;
        for (int q = 0; q < 6; ++q) {
            int m = mask_under(size, PERMS[q]);
            if (m < best) best = m;
        }
        int cls = -1;
        for (int i = 0; i < g_n_static; ++i)
            if (g_static_rep[i] == best) cls = i;
        if (cls < 0) return ORC_ERR_INPUT;
        rc |= add_u64(&C->h30[cls], 1);
    }
    if (C->fam & FAM_TEMPORAL) {
        int64_t o[3] = {a, b, c};
        /* sort the three positions by time */
        for (int x = 0; x < 3; ++x)
            for (int y = x + 1; y < 3; ++y)
                if (before(C->ts, C->ids, o[y], o[x])) { int64_t t = o[x]; o[x] = o[y]; o[y] = t; }
        if (C->ts[o[2]] - C->ts[o[0]] <= C->delta) {
            /* permutation taking labels (a,b,c) to time order */
            int p[3];
            for (int x = 0; x < 3; ++x) p[x] = (o[x] == a) ? 0 : (o[x] == b) ? 1 : 2;
            int m = mask_under(size, p);
            int cls = g_temporal_of_mask[m];
            if (cls < 0) return ORC_ERR_INPUT;
            rc |= add_u64(&C->t96[cls], 1);
        }
    }
    return rc;
}

static int is_connected_triple(const int64_t size[7]) {
    int ab = size[3] + size[6] > 0, bc = size[4] + size[6] > 0, ac = size[5] + size[6] > 0;
    return ab + bc + ac >= 2;
}

#define EDGE(i) (mem + off[i]), (off[(i) + 1] - off[i])

/* ------------------------------------------------------------------------ */
/* hyperedge and temporal families: brute force over all triples              */
/* ------------------------------------------------------------------------ */

/* Every unordered triple of hyperedges, by definition.  O(n^3) triples; each
 * connected one is classified from its literal Venn regions. */
int orc_count_brute(int64_t n, const int64_t* off, const int32_t* mem, const int64_t* ts,
                    const int32_t* ids, int64_t delta, uint32_t fam,
                    uint64_t* h30, uint64_t* t96) {
    build_tables();
    int rc = check_csr(n, off, mem);
    if (rc) return rc;
    if ((fam & FAM_TEMPORAL) && (!ts || !ids)) return ORC_ERR_INPUT;
    if (h30) memset(h30, 0, 30 * sizeof(uint64_t));
    if (t96) memset(t96, 0, 96 * sizeof(uint64_t));
    counters C = {fam & (FAM_HYPEREDGE | FAM_TEMPORAL), delta, ts, ids, h30, t96};
    if (n > 20000) return ORC_ERR_INPUT; /* brute force is for tiny inputs */
    /* meets[a*n+b]: do hyperedges a and b share a vertex?  A triple is
     * connected exactly when at least two of its three pairs meet, so triples
     * failing that are skipped before their Venn regions are computed. */
    unsigned char* meets = calloc((size_t)n * (size_t)(n > 0 ? n : 1), 1);
    if (!meets) return ORC_ERR_NOMEM;
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = a + 1; b < n; ++b) {
            const int32_t *x = mem + off[a], *y = mem + off[b];
            int64_t i = 0, j = 0, nx = off[a + 1] - off[a], ny = off[b + 1] - off[b];
            while (i < nx && j < ny && x[i] != y[j]) {
                if (x[i] < y[j]) ++i;
                else ++j;
            }
            meets[a * n + b] = meets[b * n + a] = (i < nx && j < ny);
        }
    int64_t size[7];
    for (int64_t a = 0; a < n && !rc; ++a)
        for (int64_t b = a + 1; b < n && !rc; ++b)
            for (int64_t c = b + 1; c < n && !rc; ++c) {
                if (meets[a * n + b] + meets[b * n + c] + meets[a * n + c] < 2) continue;
                venn_sizes(EDGE(a), EDGE(b), EDGE(c), size);
                if (!is_connected_triple(size)) { rc = ORC_ERR_INPUT; break; }
                rc |= record_triad(&C, a, b, c, size);
            }
    free(meets);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* vertex -> hyperedge lists and hyperedge neighbourhoods                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t nv;
    int64_t* voff; /* nv+1 */
    int64_t* vh;   /* positions of hyperedges containing each vertex, ascending */
} v2h_t;

static int build_v2h(int64_t n, const int64_t* off, const int32_t* mem, v2h_t* V) {
    int64_t nv = 0;
    for (int64_t p = 0; p < off[n]; ++p)
        if (mem[p] + 1 > nv) nv = mem[p] + 1;
    V->nv = nv;
    V->voff = calloc((size_t)nv + 1, sizeof(int64_t));
    V->vh = malloc(sizeof(int64_t) * (size_t)(off[n] > 0 ? off[n] : 1));
    if (!V->voff || !V->vh) return ORC_ERR_NOMEM;
    for (int64_t p = 0; p < off[n]; ++p) V->voff[mem[p] + 1]++;
    for (int64_t v = 0; v < nv; ++v) V->voff[v + 1] += V->voff[v];
    int64_t* fill = malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    if (!fill) return ORC_ERR_NOMEM;
    for (int64_t v = 0; v < nv; ++v) fill[v] = V->voff[v];
    for (int64_t i = 0; i < n; ++i) /* ascending i, so each list is sorted */
        for (int64_t p = off[i]; p < off[i + 1]; ++p) V->vh[fill[mem[p]]++] = i;
    free(fill);
    return ORC_OK;
}

static void free_v2h(v2h_t* V) { free(V->voff); free(V->vh); }

static int cmp_i64(const void* x, const void* y) {
    int64_t a = *(const int64_t*)x, b = *(const int64_t*)y;
    return (a > b) - (a < b);
}

/* N(h): positions of the hyperedges other than h sharing a vertex with h,
 * ascending and without repeats.  Caller frees *out. */
static int neighbours(int64_t h, const int64_t* off, const int32_t* mem, const v2h_t* V,
                      int64_t** out, int64_t* n_out) {
    int64_t cap = 0;
    for (int64_t p = off[h]; p < off[h + 1]; ++p) cap += V->voff[mem[p] + 1] - V->voff[mem[p]];
    int64_t* buf = malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
    if (!buf) return ORC_ERR_NOMEM;
    int64_t m = 0;
    for (int64_t p = off[h]; p < off[h + 1]; ++p)
        for (int64_t q = V->voff[mem[p]]; q < V->voff[mem[p] + 1]; ++q)
            if (V->vh[q] != h) buf[m++] = V->vh[q];
    qsort(buf, (size_t)m, sizeof(int64_t), cmp_i64);
    int64_t u = 0;
    for (int64_t i = 0; i < m; ++i)
        if (u == 0 || buf[u - 1] != buf[i]) buf[u++] = buf[i];
    *out = buf;
    *n_out = u;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* hyperedge and temporal families: wedge enumeration                        */
/* ------------------------------------------------------------------------ */

/* Every connected triple has a hyperedge meeting both others (its centre).
 * For each centre b and each pair {a,c} of its neighbours: if a and c are
 * disjoint the triple is open and b is its only centre; otherwise it is
 * closed, has three centres, and is counted at the centre of smallest
 * position. */
int orc_count_wedge(int64_t n, const int64_t* off, const int32_t* mem, const int64_t* ts,
                    const int32_t* ids, int64_t delta, uint32_t fam,
                    uint64_t* h30, uint64_t* t96) {
    build_tables();
    int rc = check_csr(n, off, mem);
    if (rc) return rc;
    if ((fam & FAM_TEMPORAL) && (!ts || !ids)) return ORC_ERR_INPUT;
    if (h30) memset(h30, 0, 30 * sizeof(uint64_t));
    if (t96) memset(t96, 0, 96 * sizeof(uint64_t));
    counters C = {fam & (FAM_HYPEREDGE | FAM_TEMPORAL), delta, ts, ids, h30, t96};
    v2h_t V;
    rc = build_v2h(n, off, mem, &V);
    if (rc) return rc;
    int64_t size[7];
    for (int64_t b = 0; b < n && !rc; ++b) {
        int64_t *nb, m;
        rc = neighbours(b, off, mem, &V, &nb, &m);
        if (rc) break;
        for (int64_t i = 0; i < m && !rc; ++i)
            for (int64_t j = i + 1; j < m && !rc; ++j) {
                int64_t a = nb[i], c = nb[j];
                venn_sizes(EDGE(a), EDGE(b), EDGE(c), size);
                int closed = size[5] + size[6] > 0; /* a meets c */
                if (closed && !(b < a && b < c)) continue;
                rc |= record_triad(&C, a, b, c, size);
            }
        free(nb);
    }
    free_v2h(&V);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* triads containing at least one selected hyperedge                         */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t x, y, z; } trip;

static int cmp_trip(const void* p, const void* q) {
    const trip *a = p, *b = q;
    if (a->x != b->x) return (a->x > b->x) - (a->x < b->x);
    if (a->y != b->y) return (a->y > b->y) - (a->y < b->y);
    return (a->z > b->z) - (a->z < b->z);
}

static int push_trip(trip** buf, int64_t* len, int64_t* cap, int64_t a, int64_t b, int64_t c) {
    if (*len == *cap) {
        int64_t nc = *cap ? 2 * *cap : 1024;
        trip* nb = realloc(*buf, sizeof(trip) * (size_t)nc);
        if (!nb) return ORC_ERR_NOMEM;
        *buf = nb;
        *cap = nc;
    }
    /* store sorted */
    int64_t t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    (*buf)[(*len)++] = (trip){a, b, c};
    return ORC_OK;
}

/* All connected triples containing at least one of the selected positions,
 * listed from each selected h (its neighbours, and its neighbours'
 * neighbours), then sorted and deduplicated before being classified. */
int orc_count_containing(int64_t n, const int64_t* off, const int32_t* mem, const int64_t* ts,
                         const int32_t* ids, int64_t delta, uint32_t fam,
                         int64_t n_sel, const int64_t* sel_pos,
                         uint64_t* h30, uint64_t* t96) {
    build_tables();
    int rc = check_csr(n, off, mem);
    if (rc) return rc;
    if ((fam & FAM_TEMPORAL) && (!ts || !ids)) return ORC_ERR_INPUT;
    if (h30) memset(h30, 0, 30 * sizeof(uint64_t));
    if (t96) memset(t96, 0, 96 * sizeof(uint64_t));
    counters C = {fam & (FAM_HYPEREDGE | FAM_TEMPORAL), delta, ts, ids, h30, t96};
    v2h_t V;
    rc = build_v2h(n, off, mem, &V);
    if (rc) return rc;
    trip* buf = NULL;
    int64_t len = 0, cap = 0;
    for (int64_t s = 0; s < n_sel && !rc; ++s) {
        int64_t h = sel_pos[s];
        if (h < 0 || h >= n) { rc = ORC_ERR_INPUT; break; }
        int64_t *nh, m;
        rc = neighbours(h, off, mem, &V, &nh, &m);
        if (rc) break;
        for (int64_t i = 0; i < m && !rc; ++i) {
            int64_t g = nh[i];
            for (int64_t j = i + 1; j < m && !rc; ++j) rc = push_trip(&buf, &len, &cap, h, g, nh[j]);
            int64_t *ng, mg;
            if (!rc) rc = neighbours(g, off, mem, &V, &ng, &mg);
            if (rc) break;
            for (int64_t j = 0; j < mg && !rc; ++j)
                if (ng[j] != h) rc = push_trip(&buf, &len, &cap, h, g, ng[j]);
            free(ng);
        }
        free(nh);
    }
    if (!rc) {
        qsort(buf, (size_t)len, sizeof(trip), cmp_trip);
        int64_t size[7];
        for (int64_t i = 0; i < len && !rc; ++i) {
            if (i > 0 && cmp_trip(&buf[i], &buf[i - 1]) == 0) continue;
            venn_sizes(EDGE(buf[i].x), EDGE(buf[i].y), EDGE(buf[i].z), size);
            if (!is_connected_triple(size)) continue;
            rc |= record_triad(&C, buf[i].x, buf[i].y, buf[i].z, size);
        }
    }
    free(buf);
    free_v2h(&V);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* incident-vertex family                                                    */
/* ------------------------------------------------------------------------ */

static int contains(const int32_t* e, int64_t k, int32_t v) {
    int64_t lo = 0, hi = k;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (e[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < k && e[lo] == v;
}

/* Literal enumeration (tiny inputs): for every vertex triple u<v<w and every
 * assignment of a hyperedge a to pair uv, b to pair vw and c to pair uw with
 * each hyperedge containing its pair, add 1 to the type given by the number
 * of distinct hyperedges among a, b, c. */
int orc_vertex_literal(int64_t n, const int64_t* off, const int32_t* mem, int32_t n_vertices,
                       uint64_t* v3) {
    int rc = check_csr(n, off, mem);
    if (rc) return rc;
    memset(v3, 0, 3 * sizeof(uint64_t));
    int64_t *Luv = malloc(sizeof(int64_t) * (size_t)(n + 1)), *Lvw = malloc(sizeof(int64_t) * (size_t)(n + 1)),
            *Luw = malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!Luv || !Lvw || !Luw) return ORC_ERR_NOMEM;
    for (int32_t u = 0; u < n_vertices && !rc; ++u)
        for (int32_t v = u + 1; v < n_vertices && !rc; ++v)
            for (int32_t w = v + 1; w < n_vertices && !rc; ++w) {
                int64_t nuv = 0, nvw = 0, nuw = 0;
                for (int64_t h = 0; h < n; ++h) {
                    int hu = contains(EDGE(h), u), hv = contains(EDGE(h), v), hw = contains(EDGE(h), w);
                    if (hu && hv) Luv[nuv++] = h;
                    if (hv && hw) Lvw[nvw++] = h;
                    if (hu && hw) Luw[nuw++] = h;
                }
                for (int64_t i = 0; i < nuv; ++i)
                    for (int64_t j = 0; j < nvw; ++j)
                        for (int64_t k = 0; k < nuw; ++k) {
                            int64_t a = Luv[i], b = Lvw[j], c = Luw[k];
                            int distinct = 1 + (b != a) + (c != a && c != b);
                            rc |= add_u64(&v3[distinct - 1], 1);
                        }
            }
    free(Luv); free(Lvw); free(Luw);
    return rc;
}

static int64_t isect2(const int64_t* a, int64_t na, const int64_t* b, int64_t nb) {
    int64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

static int64_t isect3(const int64_t* a, int64_t na, const int64_t* b, int64_t nb,
                      const int64_t* c, int64_t nc) {
    int64_t i = 0, j = 0, k = 0, cnt = 0;
    while (i < na && j < nb && k < nc) {
        int64_t m = a[i];
        if (b[j] > m) m = b[j];
        if (c[k] > m) m = c[k];
        while (i < na && a[i] < m) ++i;
        while (j < nb && b[j] < m) ++j;
        while (k < nc && c[k] < m) ++k;
        if (i < na && j < nb && k < nc && a[i] == m && b[j] == m && c[k] == m) { ++cnt; ++i; ++j; ++k; }
    }
    return cnt;
}

/* Per vertex triple (medium inputs).  With m_p the number of hyperedges
 * holding pair p and m_uvw the number holding all three vertices, the
 * witness assignments split as: all one hyperedge -> m_uvw ways; exactly two
 * distinct -> one hyperedge holding all three covers two pairs and a
 * different one covers the third: m_uvw * (m_uv + m_vw + m_uw - 3) ways; all
 * three distinct -> the remaining m_uv*m_vw*m_uw minus both.  Only vertex
 * triples whose three pairs each share a hyperedge contribute; they are found
 * as triangles of the vertex co-membership graph. */
int orc_vertex_triples(int64_t n, const int64_t* off, const int32_t* mem, uint64_t* v3) {
    int rc = check_csr(n, off, mem);
    if (rc) return rc;
    memset(v3, 0, 3 * sizeof(uint64_t));
    v2h_t V;
    rc = build_v2h(n, off, mem, &V);
    if (rc) return rc;
    int64_t nv = V.nv;
    /* co-membership adjacency: sorted unique neighbours of each vertex */
    int64_t* aoff = calloc((size_t)nv + 1, sizeof(int64_t));
    int64_t** adj = calloc((size_t)(nv > 0 ? nv : 1), sizeof(int64_t*));
    if (!aoff || !adj) return ORC_ERR_NOMEM;
    for (int64_t u = 0; u < nv && !rc; ++u) {
        int64_t cap = 0;
        for (int64_t q = V.voff[u]; q < V.voff[u + 1]; ++q) cap += off[V.vh[q] + 1] - off[V.vh[q]];
        int64_t* buf = malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
        if (!buf) { rc = ORC_ERR_NOMEM; break; }
        int64_t m = 0;
        for (int64_t q = V.voff[u]; q < V.voff[u + 1]; ++q)
            for (int64_t p = off[V.vh[q]]; p < off[V.vh[q] + 1]; ++p)
                if (mem[p] != u) buf[m++] = mem[p];
        qsort(buf, (size_t)m, sizeof(int64_t), cmp_i64);
        int64_t k = 0;
        for (int64_t i = 0; i < m; ++i)
            if (k == 0 || buf[k - 1] != buf[i]) buf[k++] = buf[i];
        adj[u] = buf;
        aoff[u] = k; /* degree in the co-membership graph */
    }
    for (int64_t u = 0; u < nv && !rc; ++u) {
        const int64_t* Eu = V.vh + V.voff[u];
        int64_t du = V.voff[u + 1] - V.voff[u];
        for (int64_t i = 0; i < aoff[u] && !rc; ++i) {
            int64_t v = adj[u][i];
            if (v <= u) continue;
            const int64_t* Ev = V.vh + V.voff[v];
            int64_t dv = V.voff[v + 1] - V.voff[v];
            uint64_t muv = (uint64_t)isect2(Eu, du, Ev, dv);
            for (int64_t j = i + 1; j < aoff[u] && !rc; ++j) {
                int64_t w = adj[u][j];
                if (w <= v) continue;
                /* is w adjacent to v? */
                const int64_t* Ew = V.vh + V.voff[w];
                int64_t dw = V.voff[w + 1] - V.voff[w];
                uint64_t mvw = (uint64_t)isect2(Ev, dv, Ew, dw);
                if (mvw == 0) continue;
                uint64_t muw = (uint64_t)isect2(Eu, du, Ew, dw);
                uint64_t muvw = (uint64_t)isect3(Eu, du, Ev, dv, Ew, dw);
                unsigned __int128 total = (unsigned __int128)muv * mvw * muw;
                unsigned __int128 t1 = muvw;
                unsigned __int128 t2 = (unsigned __int128)muvw * (muv + mvw + muw - 3);
                unsigned __int128 t3 = total - t1 - t2;
                if (t3 >> 64) { rc = ORC_ERR_OVERFLOW; break; }
                rc |= add_u64(&v3[0], (uint64_t)t1);
                rc |= add_u64(&v3[1], (uint64_t)t2);
                rc |= add_u64(&v3[2], (uint64_t)t3);
            }
        }
    }
    for (int64_t u = 0; u < nv; ++u) free(adj[u]);
    free(adj);
    free(aoff);
    free_v2h(&V);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* incident-vertex instances with at least one selected witness              */
/* ------------------------------------------------------------------------ */

/* Literal (tiny inputs): as orc_vertex_literal, but an assignment (a, b, c)
 * of witnesses to the pairs uv, vw, uw counts only when at least one of a, b,
 * c is selected (sel[position] != 0).  With every hyperedge selected this is
 * orc_vertex_literal itself. */
int orc_vertex_literal_containing(int64_t n, const int64_t* off, const int32_t* mem, int32_t n_vertices,
                                  const uint8_t* sel, uint64_t* v3) {
    int rc = check_csr(n, off, mem);
    if (rc) return rc;
    if (!sel && n > 0) return ORC_ERR_INPUT;
    memset(v3, 0, 3 * sizeof(uint64_t));
    int64_t *Luv = malloc(sizeof(int64_t) * (size_t)(n + 1)), *Lvw = malloc(sizeof(int64_t) * (size_t)(n + 1)),
            *Luw = malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!Luv || !Lvw || !Luw) return ORC_ERR_NOMEM;
    for (int32_t u = 0; u < n_vertices && !rc; ++u)
        for (int32_t v = u + 1; v < n_vertices && !rc; ++v)
            for (int32_t w = v + 1; w < n_vertices && !rc; ++w) {
                int64_t nuv = 0, nvw = 0, nuw = 0;
                for (int64_t h = 0; h < n; ++h) {
                    int hu = contains(EDGE(h), u), hv = contains(EDGE(h), v), hw = contains(EDGE(h), w);
                    if (hu && hv) Luv[nuv++] = h;
                    if (hv && hw) Lvw[nvw++] = h;
                    if (hu && hw) Luw[nuw++] = h;
                }
                for (int64_t i = 0; i < nuv; ++i)
                    for (int64_t j = 0; j < nvw; ++j)
                        for (int64_t k = 0; k < nuw; ++k) {
                            int64_t a = Luv[i], b = Lvw[j], c = Luw[k];
                            if (!sel[a] && !sel[b] && !sel[c]) continue;
                            int distinct = 1 + (b != a) + (c != a && c != b);
                            rc |= add_u64(&v3[distinct - 1], 1);
                        }
            }
    free(Luv); free(Lvw); free(Luw);
    return rc;
}

/* Common members of two ascending position lists: all of them (*all) and
 * those at unselected positions (*unsel). */
static void isect2_sel(const int64_t* a, int64_t na, const int64_t* b, int64_t nb, const uint8_t* sel,
                       uint64_t* all, uint64_t* unsel) {
    int64_t i = 0, j = 0;
    *all = *unsel = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else {
            ++*all;
            if (!sel[a[i]]) ++*unsel;
            ++i;
            ++j;
        }
    }
}

static void isect3_sel(const int64_t* a, int64_t na, const int64_t* b, int64_t nb, const int64_t* c, int64_t nc,
                       const uint8_t* sel, uint64_t* all, uint64_t* unsel) {
    int64_t i = 0, j = 0, k = 0;
    *all = *unsel = 0;
    while (i < na && j < nb && k < nc) {
        int64_t m = a[i];
        if (b[j] > m) m = b[j];
        if (c[k] > m) m = c[k];
        while (i < na && a[i] < m) ++i;
        while (j < nb && b[j] < m) ++j;
        while (k < nc && c[k] < m) ++k;
        if (i < na && j < nb && k < nc && a[i] == m && b[j] == m && c[k] == m) {
            ++*all;
            if (!sel[m]) ++*unsel;
            ++i;
            ++j;
            ++k;
        }
    }
}

/* The three type counts of one vertex triple from its pair multiplicities
 * m_uv, m_vw, m_uw and its triple multiplicity m_uvw (see
 * orc_vertex_triples): type 1 = m_uvw, type 2 = m_uvw (m_uv + m_vw + m_uw - 3),
 * type 3 = the remaining m_uv m_vw m_uw.  Computed in 128 bits. */
static void triple_types(uint64_t muv, uint64_t mvw, uint64_t muw, uint64_t muvw, unsigned __int128 t[3]) {
    unsigned __int128 total = (unsigned __int128)muv * mvw * muw;
    t[0] = muvw;
    t[1] = muvw ? (unsigned __int128)muvw * (muv + mvw + muw - 3) : 0;
    t[2] = total - t[0] - t[1];
}

/* Per vertex triple (large graphs, small selections).  An instance has at
 * least one selected witness unless all three of its witnesses are
 * unselected, and the instances with only unselected witnesses are exactly
 * those of the hypergraph without the selected hyperedges.  So, per triple,
 * each type's count here is its value over all hyperedges minus its value
 * with the multiplicities counted among unselected hyperedges only.  Only a
 * triple with a pair inside a selected hyperedge s can give a difference;
 * those triples are listed from every pair {u, v} of s and every co-member w
 * of u, then sorted and deduplicated.  Cost grows as the sum over selected s
 * of |s|^2 times the co-membership degree. */
int orc_vertex_containing(int64_t n, const int64_t* off, const int32_t* mem, int64_t n_sel,
                          const int64_t* sel_pos, uint64_t* v3) {
    int rc = check_csr(n, off, mem);
    if (rc) return rc;
    memset(v3, 0, 3 * sizeof(uint64_t));
    uint8_t* sel = calloc((size_t)(n > 0 ? n : 1), 1);
    if (!sel) return ORC_ERR_NOMEM;
    for (int64_t s = 0; s < n_sel; ++s) {
        if (sel_pos[s] < 0 || sel_pos[s] >= n) { free(sel); return ORC_ERR_INPUT; }
        sel[sel_pos[s]] = 1;
    }
    v2h_t V;
    rc = build_v2h(n, off, mem, &V);
    if (rc) { free(sel); return rc; }
    trip* buf = NULL;
    int64_t len = 0, cap = 0;
    for (int64_t s = 0; s < n_sel && !rc; ++s) {
        const int64_t h = sel_pos[s];
        for (int64_t p = off[h]; p < off[h + 1] && !rc; ++p)
            for (int64_t q = p + 1; q < off[h + 1] && !rc; ++q) {
                const int64_t u = mem[p], v = mem[q];
                for (int64_t e = V.voff[u]; e < V.voff[u + 1] && !rc; ++e) {
                    const int64_t f = V.vh[e];
                    for (int64_t r = off[f]; r < off[f + 1] && !rc; ++r) {
                        const int64_t w = mem[r];
                        if (w == u || w == v) continue;
                        rc = push_trip(&buf, &len, &cap, u, v, w);
                    }
                }
            }
    }
    if (!rc) qsort(buf, (size_t)len, sizeof(trip), cmp_trip);
    for (int64_t i = 0; i < len && !rc; ++i) {
        if (i > 0 && cmp_trip(&buf[i], &buf[i - 1]) == 0) continue;
        const int64_t u = buf[i].x, v = buf[i].y, w = buf[i].z;
        const int64_t *Eu = V.vh + V.voff[u], *Ev = V.vh + V.voff[v], *Ew = V.vh + V.voff[w];
        const int64_t du = V.voff[u + 1] - V.voff[u], dv = V.voff[v + 1] - V.voff[v],
                      dw = V.voff[w + 1] - V.voff[w];
        uint64_t muv, muv0, mvw, mvw0, muw, muw0, muvw, muvw0;
        isect2_sel(Eu, du, Ev, dv, sel, &muv, &muv0);
        isect2_sel(Ev, dv, Ew, dw, sel, &mvw, &mvw0);
        isect2_sel(Eu, du, Ew, dw, sel, &muw, &muw0);
        isect3_sel(Eu, du, Ev, dv, Ew, dw, sel, &muvw, &muvw0);
        unsigned __int128 all[3], rest[3];
        triple_types(muv, mvw, muw, muvw, all);
        triple_types(muv0, mvw0, muw0, muvw0, rest);
        for (int t = 0; t < 3 && !rc; ++t) {
            const unsigned __int128 d = all[t] - rest[t];
            if (d >> 64) rc = ORC_ERR_OVERFLOW;
            else rc |= add_u64(&v3[t], (uint64_t)d);
        }
    }
    free(buf);
    free_v2h(&V);
    free(sel);
    return rc;
}

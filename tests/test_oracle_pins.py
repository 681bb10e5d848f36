"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something independent of its code: the
class counts printed in the paper, hand-derived fixtures (tests/golden), set
arithmetic done here in Python, closed forms, networkx/numpy routines, or a
second oracle algorithm.  A dropped Venn term, a wrong relabelling or a wrong
attribution in the oracle breaks at least one of them.
"""
import itertools
import json
import math
import os

import networkx as nx
import numpy as np
import pytest

import gen
from oracle import OracleHypergraph
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
REGION_KEYS = ["a_only", "b_only", "c_only", "ab_not_c", "bc_not_a", "ac_not_b", "abc"]
BIG = 1 << 62


# ---------------------------------------------------------------------------
# independent Python set arithmetic (no code shared with the oracle)
# ---------------------------------------------------------------------------

def regions_py(a, b, c):
    a, b, c = set(a), set(b), set(c)
    return [a - b - c, b - a - c, c - a - b, (a & b) - c, (b & c) - a, (a & c) - b, a & b & c]


def mask_py(a, b, c):
    return sum(1 << i for i, r in enumerate(regions_py(a, b, c)) if r)


def canonical_py(a, b, c):
    return min(mask_py(*p) for p in itertools.permutations((a, b, c)))


def connected_py(a, b, c):
    a, b, c = set(a), set(b), set(c)
    return (bool(a & b) + bool(b & c) + bool(a & c)) >= 2


def valid_masks_py(allow_identical):
    """Masks of three non-empty, connected sets, by building a concrete
    triple of sets for each mask (one fresh vertex per non-empty region)."""
    out = []
    for m in range(128):
        sets = [set(), set(), set()]
        memb = [(0,), (1,), (2,), (0, 1), (1, 2), (0, 2), (0, 1, 2)]
        for r in range(7):
            if m >> r & 1:
                for s in memb[r]:
                    sets[s].add(r)
        a, b, c = sets
        if not (a and b and c) or not connected_py(a, b, c):
            continue
        if not allow_identical and (a == b or b == c or a == c):
            continue
        out.append((m, (a, b, c)))
    return out


def expected_counts_py(edges, ts=None, delta=None):
    """Static and temporal class counts by Python sets over all triples."""
    t = O.tables()
    h30 = np.zeros(30, np.uint64)
    t96 = np.zeros(96, np.uint64)
    rep_index = {r: i for i, r in enumerate(t["static_rep"])}
    tmask_index = {m: i for i, m in enumerate(t["temporal_mask"])}
    for i, j, k in itertools.combinations(range(len(edges)), 3):
        a, b, c = edges[i], edges[j], edges[k]
        if not connected_py(a, b, c):
            continue
        h30[rep_index[canonical_py(a, b, c)]] += 1
        if ts is not None:
            order = sorted((i, j, k), key=lambda x: (ts[x], x))
            if ts[order[2]] - ts[order[0]] <= delta:
                t96[tmask_index[mask_py(*(edges[x] for x in order))]] += 1
    return h30, t96


def csr_of(edges):
    off = np.zeros(len(edges) + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.array([v for e in edges for v in sorted(e)], np.int32)
    return off, mem


# ---------------------------------------------------------------------------
# class tables
# ---------------------------------------------------------------------------

def test_class_counts_match_paper():
    t = O.tables()
    # "26 unique hypergraph triads" (paper Section II, hyperedge triads)
    assert t["n_static_nodup"] == 26
    # "96 temporal hypergraph motifs" (paper Section VI on THyMe+)
    assert t["n_temporal"] == 96
    assert t["n_static"] == 30
    # MoCHy's split of the 26: 20 closed, 6 open
    assert sum(t["static_closed"][:26]) == 20
    assert sum(1 - c for c in t["static_closed"][:26]) == 6


def test_class_tables_match_python_enumeration():
    t = O.tables()
    nodup = valid_masks_py(False)
    withdup = valid_masks_py(True)
    assert len(nodup) == 86 and len(withdup) == 96
    # temporal index = rank of the mask among the valid ordered masks
    assert t["temporal_mask"] == [m for m, _ in withdup]
    # static reps: smallest mask of each orbit, non-identical orbits first
    reps_nodup = sorted({canonical_py(*s) for _, s in nodup})
    reps_all = sorted({canonical_py(*s) for _, s in withdup})
    reps_dup = sorted(set(reps_all) - set(reps_nodup))
    assert t["static_rep"] == reps_nodup + reps_dup
    for m, s in withdup:
        assert t["static_rep"][t["static_of_mask"][m]] == canonical_py(*s)
    valid = {m for m, _ in withdup}
    for m in range(128):
        if m not in valid:
            assert t["static_of_mask"][m] == -1 and t["temporal_of_mask"][m] == -1


# ---------------------------------------------------------------------------
# hand-derived fixtures
# ---------------------------------------------------------------------------

def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


FIXTURES = ["fig1_reconstruction.json", "closed_nested.json", "identical_and_dyadic.json"]


@pytest.mark.parametrize("name", FIXTURES)
def test_fixture_hand_derivation_is_consistent(name):
    """The hand-written regions and masks agree with set arithmetic, and the
    listed triads are exactly the connected triples."""
    d = _load(name)
    E = d["hyperedges"]
    for tr in d["triads"]:
        a, b, c = (E[i] for i in tr["members"])
        got = regions_py(a, b, c)
        assert [sorted(r) for r in got] == [sorted(tr["regions"][k]) for k in REGION_KEYS]
        assert mask_py(a, b, c) == tr["mask"]
    listed = {tuple(sorted(tr["members"])) for tr in d["triads"]}
    conn = {t for t in itertools.combinations(range(len(E)), 3) if connected_py(*(E[i] for i in t))}
    assert listed == conn
    for tr in d.get("temporal", []):
        a, b, c = (E[i] for i in tr["time_order"])
        assert mask_py(a, b, c) == tr["ordered_mask"]
        if "ordered_regions" in tr:
            assert [sorted(r) for r in regions_py(a, b, c)] == \
                [sorted(tr["ordered_regions"][k]) for k in REGION_KEYS]


@pytest.mark.parametrize("name", FIXTURES)
@pytest.mark.parametrize("method", ["brute", "wedge"])
def test_oracle_on_fixture(name, method):
    d = _load(name)
    E = d["hyperedges"]
    off, mem = csr_of(E)
    ts = np.array(d["timestamps"], np.int64)
    ids = np.arange(len(E), dtype=np.int32)
    t = O.tables()
    exp_h = np.zeros(30, np.uint64)
    for tr in d["triads"]:
        a, b, c = (E[i] for i in tr["members"])
        cls = t["static_rep"].index(canonical_py(a, b, c))
        assert bool(t["static_closed"][cls]) == tr["closed"]
        assert bool(t["static_dup"][cls]) == tr.get("identical_pair", False)
        exp_h[cls] += 1
    h, tt = O.count_hyperedge_temporal(off, mem, ts, ids, BIG, O.FAM_HYPEREDGE | O.FAM_TEMPORAL, method)
    assert np.array_equal(h, exp_h)
    # temporal: hand masks and windows (inclusive t_k - t_i <= delta)
    for tr in d.get("temporal", []):
        span = tr["span"]
        cls = t["temporal_mask"].index(tr["ordered_mask"])
        _, t_at = O.count_hyperedge_temporal(off, mem, ts, ids, span, O.FAM_TEMPORAL, method)
        _, t_below = O.count_hyperedge_temporal(off, mem, ts, ids, span - 1, O.FAM_TEMPORAL, method)
        assert t_at[cls] >= 1
        assert t_at[cls] - t_below[cls] >= 1
    v = O.count_vertex(off, mem, d["n_vertices"], "triples")
    assert list(v) == d["vertex"]
    v_lit = O.count_vertex(off, mem, d["n_vertices"], "literal")
    assert list(v_lit) == d["vertex"]


def test_fig1_temporal_window_exact():
    d = _load("fig1_reconstruction.json")
    off, mem = csr_of(d["hyperedges"])
    ts = np.array(d["timestamps"], np.int64)
    ids = np.arange(4, dtype=np.int32)
    t = O.tables()
    c31 = t["temporal_mask"].index(31)
    c28 = t["temporal_mask"].index(28)
    for delta, want in [(14, {}), (15, {c28: 1}), (19, {c28: 1}), (20, {c28: 1, c31: 1})]:
        _, tt = O.count_hyperedge_temporal(off, mem, ts, ids, delta, O.FAM_TEMPORAL, "brute")
        exp = np.zeros(96, np.uint64)
        for k, v in want.items():
            exp[k] = v
        assert np.array_equal(tt, exp), delta


# ---------------------------------------------------------------------------
# random inputs: independent routes must agree
# ---------------------------------------------------------------------------

def _random_edges(seed, nv, ne, kmin, kmax, dup_frac=0.0):
    rng = np.random.default_rng(seed)
    E = []
    for _ in range(ne):
        k = int(rng.integers(kmin, kmax + 1))
        E.append(sorted(rng.choice(nv, size=k, replace=False).tolist()))
    for i in range(len(E)):
        if rng.random() < dup_frac and i > 0:
            E[i] = list(E[int(rng.integers(0, i))])
    return E


@pytest.mark.parametrize("seed", range(6))
def test_oracle_vs_python_sets(seed):
    E = _random_edges(seed, 14, 16, 1, 5, dup_frac=0.15)
    off, mem = csr_of(E)
    rng = np.random.default_rng(100 + seed)
    ts = rng.integers(0, 30, size=len(E)).astype(np.int64)   # ties on purpose
    ids = np.arange(len(E), dtype=np.int32)
    delta = int(rng.integers(0, 30))
    exp_h, exp_t = expected_counts_py(E, ts, delta)
    for method in ("brute", "wedge"):
        h, tt = O.count_hyperedge_temporal(off, mem, ts, ids, delta,
                                           O.FAM_HYPEREDGE | O.FAM_TEMPORAL, method)
        assert np.array_equal(h, exp_h), method
        assert np.array_equal(tt, exp_t), method


@pytest.mark.parametrize("seed", range(4))
def test_brute_equals_wedge_medium(seed):
    s = gen.random_small(seed, 300, 250, 2, 9)
    g = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
    off, mem, ts, ids = g.csr()
    delta = int(np.median(np.diff(ts)) * 40)
    hb, tb = O.count_hyperedge_temporal(off, mem, ts, ids, delta, 5, "brute")
    hw, tw = O.count_hyperedge_temporal(off, mem, ts, ids, delta, 5, "wedge")
    assert np.array_equal(hb, hw) and np.array_equal(tb, tw)
    assert hb.sum() > 0 and tb.sum() > 0


def test_connected_triples_from_networkx_line_graph():
    s = gen.random_small(7, 400, 300, 2, 6)
    g = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members)
    off, mem, ts, ids = g.csr()
    h, _ = O.count_hyperedge_temporal(off, mem, ts, ids, 0, O.FAM_HYPEREDGE, "wedge")
    # line graph: hyperedges are nodes, adjacent when they share a vertex
    L = nx.Graph()
    L.add_nodes_from(range(len(ids)))
    by_v = {}
    for i in range(len(ids)):
        for v in mem[off[i]:off[i + 1]]:
            by_v.setdefault(int(v), []).append(i)
    for hs in by_v.values():
        L.add_edges_from(itertools.combinations(hs, 2))
    tri = sum(nx.triangles(L).values()) // 3
    wedges = sum(math.comb(d, 2) for _, d in L.degree())
    t = O.tables()
    closed = sum(int(h[i]) for i in range(30) if t["static_closed"][i])
    open_ = sum(int(h[i]) for i in range(30) if not t["static_closed"][i])
    assert closed == tri
    assert open_ == wedges - 3 * tri
    assert int(h.sum()) == wedges - 2 * tri


def test_dyadic_graph_closed_forms():
    """Card-2 hyperedges of a simple graph: triangles, 3-stars and 3-paths."""
    G = nx.gnm_random_graph(60, 200, seed=3)
    E = [sorted(e) for e in G.edges()]
    off, mem = csr_of(E)
    h, _ = O.count_hyperedge_temporal(off, mem, None, None, 0, O.FAM_HYPEREDGE, "wedge")
    t = O.tables()
    tri = sum(nx.triangles(G).values()) // 3
    stars = sum(math.comb(d, 3) for _, d in G.degree())
    paths = sum((G.degree(u) - 1) * (G.degree(v) - 1) for u, v in G.edges()) - 3 * tri
    exp = np.zeros(30, np.uint64)
    exp[t["static_of_mask"][56]] = tri       # pairwise-only regions: triangle
    exp[t["static_of_mask"][71]] = stars     # one shared vertex: star
    exp[t["static_of_mask"][29]] = paths     # chain a-b-c
    assert np.array_equal(h, exp)
    v = O.count_vertex(off, mem, 60, "triples")
    assert list(v) == [0, 0, tri]


@pytest.mark.parametrize("seed", range(4))
def test_vertex_literal_equals_per_triple(seed):
    E = _random_edges(seed, 12, 10, 1, 6, dup_frac=0.2)
    off, mem = csr_of(E)
    assert np.array_equal(O.count_vertex(off, mem, 12, "literal"),
                          O.count_vertex(off, mem, 12, "triples"))


def test_vertex_closed_forms():
    s = gen.random_small(11, 150, 120, 2, 7)
    g = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members)
    off, mem, ts, ids = g.csr()
    v = O.count_vertex(off, mem, None, "triples")
    sizes = np.diff(off)
    assert int(v[0]) == sum(math.comb(int(k), 3) for k in sizes)
    # co-membership multiplicity matrix M (zero diagonal): sum over vertex
    # triples of m_uv m_vw m_uw = trace(M^3)/6 = T1 + T2 + T3
    n = s.n_vertices
    M = np.zeros((n, n), np.int64)
    for i in range(len(ids)):
        e = mem[off[i]:off[i + 1]]
        M[np.ix_(e, e)] += 1
    np.fill_diagonal(M, 0)
    assert int(np.trace(M @ M @ M)) // 6 == int(v.sum())


def test_temporal_fold_equals_static():
    s = gen.random_small(5, 200, 160, 2, 6)
    g = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
    off, mem, ts, ids = g.csr()
    h, tt = O.count_hyperedge_temporal(off, mem, ts, ids, BIG, 5, "wedge")
    t = O.tables()
    fold = np.zeros(30, np.uint64)
    for i, m in enumerate(t["temporal_mask"]):
        fold[t["static_of_mask"][m]] += tt[i]
    assert np.array_equal(fold, h)


def test_relabelling_invariance():
    s = gen.random_small(9, 200, 150, 2, 6)
    g = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
    off, mem, ts, ids = g.csr()
    h, tt = O.count_hyperedge_temporal(off, mem, ts, ids, BIG, 5, "wedge")
    v = O.count_vertex(off, mem)
    rng = np.random.default_rng(1)
    vperm = rng.permutation(s.n_vertices)
    eperm = rng.permutation(len(ids))
    E = [sorted(vperm[mem[off[i]:off[i + 1]]].tolist()) for i in eperm]
    off2, mem2 = csr_of(E)
    ts2 = ts[eperm]
    h2, t2 = O.count_hyperedge_temporal(off2, mem2, ts2, np.arange(len(E), dtype=np.int32),
                                        BIG, 5, "wedge")
    assert np.array_equal(h, h2) and np.array_equal(tt, t2)   # timestamps are distinct
    assert np.array_equal(v, O.count_vertex(off2, mem2))


# ---------------------------------------------------------------------------
# dynamic behaviour: ID rule and incremental = recount
# ---------------------------------------------------------------------------

def test_id_reuse_rule_hand_cases():
    g = OracleHypergraph(10, *csr_of([[0], [1], [2], [3], [4]]), np.arange(5))
    assert list(g.live_ids()) == [0, 1, 2, 3, 4]
    off, mem = csr_of([[5, 5, 6], [7], [8]])
    ids = g.apply_batch(off, mem, np.array([9, 9, 9]), np.array([3, 1]))
    assert list(ids) == [1, 3, 5]               # freed IDs ascending, then fresh
    assert list(g.edge(1)) == [5, 6]            # repeated member collapsed
    off, mem = csr_of([[9], [9, 8]])
    ids = g.apply_batch(off, mem, None, np.array([5, 0]))
    assert list(ids) == [0, 5]
    with pytest.raises(ValueError):
        g.apply_batch(*csr_of([]), None, np.array([2, 2]))     # duplicate delete
    with pytest.raises(ValueError):
        g.apply_batch(*csr_of([]), None, np.array([7]))        # not live
    with pytest.raises(ValueError):
        g.apply_batch(*csr_of([[10]]), None, np.array([]))     # vertex out of range
    assert list(g.live_ids()) == [0, 1, 2, 3, 4, 5]            # failed batches changed nothing


def _apply(g, batch):
    dels = g.resolve_ranks(batch.del_ranks)
    return dels, g.apply_batch(batch.inserts.offsets, batch.inserts.members,
                               batch.inserts.timestamps, dels)


def test_incremental_equals_recount_and_insert_delete_restores():
    s = gen.random_small(21, 300, 220, 2, 7, n_batches=3, n_ins=25, n_del=25)
    g = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
    delta = BIG
    before = O.counts(g, 7, delta)
    base = {k: v.copy() for k, v in before.items()}
    for b in s.batches:
        off0, mem0, ts0, ids0 = g.csr()
        dels, new_ids = _apply(g, b)
        off1, mem1, ts1, ids1 = g.csr()
        pos0 = np.searchsorted(ids0, dels)
        pos1 = np.searchsorted(ids1, new_ids)
        d_h, d_t = O.count_containing(off0, mem0, ts0, ids0, delta, 5, pos0)
        i_h, i_t = O.count_containing(off1, mem1, ts1, ids1, delta, 5, pos1)
        after = O.counts(g, 7, delta)
        assert np.array_equal(after["hyperedge"], before["hyperedge"] - d_h + i_h)
        assert np.array_equal(after["temporal"], before["temporal"] - d_t + i_t)
        before = after


def test_insert_then_delete_restores_counts():
    s = gen.random_small(22, 300, 220, 2, 7, n_batches=1, n_ins=25, n_del=25)
    g = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
    base = O.counts(g, 7, BIG)
    b = s.batches[0]
    dels = g.resolve_ranks(b.del_ranks)
    old_sets = [g.edge(int(d)).tolist() for d in dels]
    old_ts = np.array([g.ts[int(d)] for d in dels], np.int64)
    new_ids = g.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels)
    assert not np.array_equal(O.counts(g, 7, BIG)["hyperedge"], base["hyperedge"])
    off_d, mem_d = csr_of(old_sets)
    g.apply_batch(off_d, mem_d, old_ts, new_ids)      # timestamps are distinct
    restored = O.counts(g, 7, BIG)
    for k in base:
        assert np.array_equal(restored[k], base[k]), k


def test_generator_is_deterministic_and_well_formed():
    a, b = gen.tiny(0), gen.tiny(0)
    assert np.array_equal(a.initial.members, b.initial.members)
    assert np.array_equal(a.batches[0].del_ranks, b.batches[0].del_ranks)
    c = gen.tiny(1)
    assert not np.array_equal(a.initial.members, c.initial.members)
    sz = a.initial.sizes()
    assert sz.min() >= 2 and sz.max() <= 8 and a.initial.n == 1000
    for i in range(a.initial.n):
        m = a.initial.members[a.initial.offsets[i]:a.initial.offsets[i + 1]]
        assert len(set(m.tolist())) == len(m)
    r = a.batches[0].del_ranks
    assert len(set(r.tolist())) == 100 and r.max() < 1000
    z = gen.zipf_cardinalities(np.random.default_rng(0), 200000, 2.0, 2, 1000)
    assert z.min() == 2 and z.max() <= 1000
    # truncated Zipf(2): P(k=2) = 2^-2 / sum_{k=2}^{1000} k^-2
    p2 = 0.25 / sum(k ** -2.0 for k in range(2, 1001))
    assert abs((z == 2).mean() - p2) < 0.01


def test_horizontal_update_counts_as_delete_and_insert():
    """A horizontal update keeps the ID and timestamp; its static counts are
    those of deleting the hyperedge and inserting the new set as a new one
    (the classes do not depend on labels), and updating back restores the
    counts exactly."""
    s = gen.random_small(91, 40, 30, 2, 5)
    init = s.initial
    a = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    b = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    before = O.counts(a, 3, 0)
    old = a.edge(4).copy()
    new = np.array([0, 1, 2, 39], np.int32)
    a.update_members(np.array([4]), np.array([0, 4]), new)
    assert np.array_equal(a.edge(4), new) and a.ts[4] == init.timestamps[4]
    b.apply_batch(np.array([0, 4]), new, np.array([init.timestamps[4]]), np.array([4]))
    ca, cb = O.counts(a, 3, 0), O.counts(b, 3, 0)
    assert np.array_equal(ca["hyperedge"], cb["hyperedge"]) and np.array_equal(ca["vertex"], cb["vertex"])
    a.update_members(np.array([4]), np.array([0, old.size]), old)
    back = O.counts(a, 3, 0)
    assert np.array_equal(back["hyperedge"], before["hyperedge"]) and np.array_equal(back["vertex"], before["vertex"])


# ---------------------------------------------------------------------------
# incident-vertex instances holding a selected witness (Alg. 3 for the
# vertex family: the count change of a batch is the instances holding an
# inserted hyperedge on the new graph minus those holding a deleted one on
# the old graph)
# ---------------------------------------------------------------------------

def test_vertex_containing_hand_case():
    # A = {0,1,2}, B = {0,1}, C = {1,2}.  Triple {0,1,2}: pair 01 has
    # witnesses A, B; pair 12 has A, C; pair 02 has A.  The four assignments
    # (01, 12, 02) are (A,A,A) type 1, (A,C,A) and (B,A,A) type 2, (B,C,A)
    # type 3.  Those holding B: (B,A,A), (B,C,A).  Those holding C: (A,C,A),
    # (B,C,A).  Every assignment holds A.
    off, mem = csr_of([[0, 1, 2], [0, 1], [1, 2]])
    assert O.count_vertex(off, mem, 3, "literal").tolist() == [1, 2, 1]
    for method in ("literal", "triples"):
        assert O.count_vertex_containing(off, mem, [1], 3, method).tolist() == [0, 1, 1], method
        assert O.count_vertex_containing(off, mem, [2], 3, method).tolist() == [0, 1, 1], method
        assert O.count_vertex_containing(off, mem, [0], 3, method).tolist() == [1, 2, 1], method
        assert O.count_vertex_containing(off, mem, [1, 2], 3, method).tolist() == [0, 2, 1], method
        assert O.count_vertex_containing(off, mem, [], 3, method).tolist() == [0, 0, 0], method


@pytest.mark.parametrize("seed", range(5))
def test_vertex_containing_per_triple_equals_literal(seed):
    E = _random_edges(40 + seed, 11, 10, 1, 6, dup_frac=0.2)
    off, mem = csr_of(E)
    rng = np.random.default_rng(seed)
    for k in (1, 2, 4):
        sel = np.sort(rng.choice(len(E), size=k, replace=False))
        lit = O.count_vertex_containing(off, mem, sel, 11, "literal")
        tri = O.count_vertex_containing(off, mem, sel, 11, "triples")
        assert np.array_equal(lit, tri), (k, lit, tri)
    every = np.arange(len(E))
    assert np.array_equal(O.count_vertex_containing(off, mem, every, 11, "triples"),
                          O.count_vertex(off, mem, 11, "literal"))


def test_vertex_containing_gives_the_incremental_change():
    s = gen.random_small(31, 260, 200, 2, 8, n_batches=3, n_ins=20, n_del=20)
    g = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members)
    before = [int(x) for x in O.count_vertex(*g.csr()[:2])]
    moved = 0
    for b in s.batches:
        off0, mem0, _, ids0 = g.csr()
        dels, new_ids = _apply(g, b)
        off1, mem1, _, ids1 = g.csr()
        d = O.count_vertex_containing(off0, mem0, np.searchsorted(ids0, dels))
        i = O.count_vertex_containing(off1, mem1, np.searchsorted(ids1, new_ids))
        after = [int(x) for x in O.count_vertex(off1, mem1)]
        assert after == [before[t] - int(d[t]) + int(i[t]) for t in range(3)]
        moved += int(d.sum()) + int(i.sum())
        before = after
    assert moved > 0

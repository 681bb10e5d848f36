"""Host-side logic that needs no GPU: the serving client's copy of the ID
rule (bench.py) against the oracle's, and the seeded serving generators."""
import numpy as np

import gen
from oracle import OracleHypergraph


def test_client_id_model_follows_the_id_rule():
    import bench
    rng = np.random.default_rng(1)
    nv, n0 = 50, 40
    off = np.arange(0, 2 * n0 + 1, 2, dtype=np.int64)
    mem = np.concatenate([np.sort(rng.choice(nv, 2, replace=False)) for _ in range(n0)]).astype(np.int32)
    og = OracleHypergraph(nv, off, mem, np.zeros(n0, np.int64))
    m = bench._IdModel(n0)
    for step in range(300):
        nd, ni = int(rng.integers(0, 8)), int(rng.integers(0, 10))
        idx, d = m.pick(rng, nd)
        edges = [np.sort(rng.choice(nv, 3, replace=False)) for _ in range(ni)]
        io = np.zeros(ni + 1, np.int64)
        io[1:] = np.cumsum([3] * ni)
        im = np.concatenate(edges).astype(np.int32) if ni else np.zeros(0, np.int32)
        want = og.apply_batch(io, im, np.zeros(ni, np.int64), np.sort(d).astype(np.int64))
        got = m.commit(idx, d, ni)
        assert np.array_equal(got, want), step
        assert sorted(m.live[:m.n].tolist()) == og.live_ids().tolist()


def test_serving_generators_are_seeded_and_shaped():
    a = gen.resident_graphs(seed=5, n_graphs=6, e_hi=5e3)
    b = gen.resident_graphs(seed=5, n_graphs=6, e_hi=5e3)
    for x, y in zip(a.graphs, b.graphs):
        assert np.array_equal(x.initial.members, y.initial.members)
        e0 = x.initial.n
        assert 1000 <= e0 <= 5000 and x.n_vertices == max(256, e0 // 2)
        k = np.diff(x.initial.offsets)
        assert k.min() >= 2 and k.max() <= 256
        assert x.initial.members.max() < x.n_vertices
    off, u = gen.insert_pool(6, 1000)
    assert len(off) == 1001 and off[-1] == len(u)
    assert u.dtype == np.float32 and 0.0 <= u.min() and u.max() < 1.0
    t, g, s = gen.serving_arrivals(7, 10, 500, 100.0)
    assert np.all(np.diff(t) > 0) and g.max() < 10 and s.min() >= 10 and s.max() <= 10000


def test_sweep_generators_are_seeded_and_shaped():
    a = gen.spread_cardinalities(np.random.default_rng(0), 100_000, 4.0, 8.0, 4096)
    b = gen.spread_cardinalities(np.random.default_rng(0), 100_000, 4.0, 8.0, 4096)
    assert np.array_equal(a, b) and a.min() >= 2
    assert abs(a.mean() - 4.0) < 0.1 and abs(a.std() - 8.0) < 0.8
    assert np.all(gen.spread_cardinalities(np.random.default_rng(0), 50, 4.0, 0.0, 10) == 4)
    d = gen.dyadic_graph(3, 40, 500)
    assert np.array_equal(d.offsets, np.arange(501) * 2)
    assert np.all(d.members[0::2] != d.members[1::2]) and d.members.max() < 40
    for L in (gen.spread_inserts(4, 30, 2, 20, 4.0, 2.0, kmax=30), gen.insert_batches(5, 30, 2, 20, 12)):
        for c in L:
            assert c.n == 20 and np.all(np.diff(c.offsets) >= 2)
            for i in range(c.n):
                e = c.members[c.offsets[i]:c.offsets[i + 1]]
                assert np.unique(e).size == e.size and e.max() < 30
    h = gen.random_hypergraph(6, 300, 1000, 50)
    assert h.n == 1000 and np.diff(h.offsets).max() <= 50 and np.all(np.diff(h.timestamps) > 0)


def test_restored_oracle_graph_hands_out_the_same_ids():
    """A graph rebuilt from its live hyperedges alone (the largest live ID +
    1 as its high-water mark) gives later inserts the same IDs as the graph
    it was taken from, also after its largest IDs were deleted."""
    rng = np.random.default_rng(5)
    nv = 40
    og = OracleHypergraph(nv)
    for step in range(60):
        live = og.live_ids()
        nd = int(rng.integers(0, min(6, live.size) + 1))
        dels = rng.choice(live, size=nd, replace=False) if nd else np.zeros(0, np.int64)
        if step % 7 == 3 and live.size > 3:  # delete the top IDs: holes above the largest live one
            dels = np.union1d(dels, live[-3:])
        ni = int(rng.integers(0, 8))
        off = np.arange(ni + 1, dtype=np.int64) * 3
        og.apply_batch(off, rng.integers(0, nv, size=3 * ni), np.full(ni, step, np.int64), dels)
        if step % 10 == 9:
            off_c, mem_c, ts_c, ids_c = og.csr()
            r = OracleHypergraph.from_checkpoint(nv, ids_c, off_c, mem_c, ts_c)
            assert r.high_water <= og.high_water
            for _ in range(3):
                live = og.live_ids()
                dels = rng.choice(live, size=min(2, live.size), replace=False)
                ni = int(rng.integers(1, 12))
                off = np.arange(ni + 1, dtype=np.int64) * 2
                mem = rng.integers(0, nv, size=2 * ni)
                a = og.apply_batch(off, mem, np.zeros(ni, np.int64), dels)
                b = r.apply_batch(off, mem, np.zeros(ni, np.int64), dels)
                assert np.array_equal(a, b)
            for x, y in zip(og.csr(), r.csr()):
                assert np.array_equal(x, y)


def _pair_stats(E):
    """m_uv and S_uv over all vertex pairs of the hyperedges E."""
    import itertools
    st = {}
    for e in E:
        for u, v in itertools.combinations(sorted(set(e)), 2):
            m, s = st.get((u, v), (0, 0))
            st[(u, v)] = (m + 1, s + len(set(e)))
    return st


def test_vertex_types_1_2_from_pair_statistics_match_the_oracle():
    """The vertex-pair form the GPU's ESC_FAMILY_VERTEX12 keeps: type 1 =
    sum C(|h|,3), type 2 = sum over vertex pairs of (m-1) S - 4 C(m,2), and
    the per-step changes S + m (k - 4) (add) / (S - k) + (m - 1)(k - 4)
    (remove) telescoping to the recount -- checked against the oracle's
    per-triple and literal counts on random hypergraphs with repeated sets."""
    import itertools
    import math
    from oracle import oracle as O
    rng = np.random.default_rng(8)
    for trial in range(6):
        nv = 12
        E = [sorted(rng.choice(nv, size=int(rng.integers(2, 7)), replace=False).tolist()) for _ in range(14)]
        E += [list(E[int(rng.integers(0, len(E)))]) for _ in range(3)]   # identical sets
        off = np.concatenate([[0], np.cumsum([len(e) for e in E])]).astype(np.int64)
        mem = np.concatenate([np.array(e, np.int32) for e in E])
        want = O.count_vertex(off, mem, nv, "literal")
        t1 = sum(math.comb(len(e), 3) for e in E)
        t2 = sum((m - 1) * s - 4 * math.comb(m, 2) for m, s in _pair_stats(E).values())
        assert [t1, t2] == [int(want[0]), int(want[1])], trial
        # incremental: add the hyperedges one by one, then remove some
        st, acc = {}, 0
        for e in E:
            k = len(e)
            for p in itertools.combinations(e, 2):
                m, s = st.get(p, (0, 0))
                acc += s + m * (k - 4)
                st[p] = (m + 1, s + k)
        assert acc == t2
        keep = E[5:]
        for e in E[:5]:
            k = len(e)
            for p in itertools.combinations(e, 2):
                m, s = st[p]
                acc -= (s - k) + (m - 1) * (k - 4)
                st[p] = (m - 1, s - k)
        off2 = np.concatenate([[0], np.cumsum([len(e) for e in keep])]).astype(np.int64)
        mem2 = np.concatenate([np.array(e, np.int32) for e in keep])
        assert acc == int(O.count_vertex(off2, mem2, nv, "literal")[1])


def test_group_loading_in_pieces_keeps_every_graph_whole_and_in_order():
    """bench's group loader: a graph larger than one call's limits is loaded
    in pieces, in order, at most one piece of a graph per call, every call
    within both limits (hyperedges, members), and each graph's hyperedges
    arrive exactly once (so under the ID rule they keep IDs 0..n-1)."""
    import types
    import bench
    calls = []
    fake = types.SimpleNamespace(esc_group_apply=lambda grp, call: calls.append(call))
    ms = gen.resident_graphs(seed=5, n_graphs=12, e_hi=3e4)
    bench._load_group(fake, None, ms.graphs, 5000, 60000)
    got = {}
    for c in calls:
        assert sum(len(x["ins_offsets"]) - 1 for x in c) <= 5000
        assert sum(len(x["ins_members"]) for x in c) <= 60000
        gs = [x["graph"] for x in c]
        assert len(gs) == len(set(gs))
        for x in c:
            got.setdefault(x["graph"], []).append(x)
    assert len(calls) > len(ms.graphs) // 2 and max(st.initial.n for st in ms.graphs) > 5000
    for i, st in enumerate(ms.graphs):
        parts = got[i]
        assert np.array_equal(np.concatenate([x["ins_members"] for x in parts]), st.initial.members)
        assert np.array_equal(np.concatenate([x["ins_timestamps"] for x in parts]), st.initial.timestamps)
        assert np.array_equal(np.concatenate([np.diff(x["ins_offsets"]) for x in parts]),
                              np.diff(st.initial.offsets))

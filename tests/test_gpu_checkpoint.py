"""Checkpoint and restore: a graph rebuilt from its export (inserts under the
exported IDs) holds the same store and counts as the oracle that saw the whole
stream, and the IDs it gives later inserts follow the ID rule exactly as the
oracle's do.  Inserts under given IDs reject live, repeated and out-of-range
IDs and change nothing when they do."""
import numpy as np
import pytest

import gen
from oracle import OracleHypergraph
from oracle import oracle as O
from tests.harness import assert_counts_equal, assert_store_equal, caps_for, run_stream

pytestmark = pytest.mark.gpu

ALL = 7


@pytest.fixture(scope="module")
def E():
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    return escher


def _drop_top(g, og, k):
    """Delete the k largest live IDs on both sides, so the largest live ID
    ends below the high-water mark and free IDs sit above it."""
    top = og.live_ids()[-k:]
    og.apply_batch(np.zeros(1, np.int64), np.zeros(0, np.int32), None, top)
    g.apply_batch(np.zeros(1, np.int64), np.zeros(0, np.int32), None, top.astype(np.int32))


@pytest.mark.parametrize("families,batch_cap", [(ALL, None), (3, 40), (ALL, 64)])
def test_restore_round_trip(E, families, batch_cap):
    s = gen.random_small(91, 400, 300, 2, 9, n_batches=3, n_ins=60, n_del=50, membership="zipf")
    delta = int(s.initial.timestamps[-1] // 3)
    caps = caps_for(s.n_vertices, 1000, 20000, 1000, 20000)
    g, og = run_stream(E, s, families, delta, caps=caps)
    _drop_top(g, og, 7)
    ck = g.export()
    rcaps = dict(caps)
    if batch_cap is not None:  # restore in several calls
        rcaps.update(max_batch_hyperedges=batch_cap, max_batch_incidences=1024)
    r = E.Graph.restore(s.n_vertices, ck, families=families, delta=delta, **rcaps)
    assert_counts_equal(r.counts(), O.counts(og, families, delta), "restored")
    assert_store_equal(r, og)
    # the next batch: holes below the largest live ID first, then fresh IDs
    n_free = int(og.live_ids()[-1]) + 1 - len(og.live_ids())
    n_new = n_free + 6 + 12  # past the largest live ID and past the old high-water mark
    rng = np.random.default_rng(3)
    off = np.arange(n_new + 1, dtype=np.int64) * 3
    mem = rng.integers(0, s.n_vertices, size=3 * n_new).astype(np.int32)
    ts = np.sort(rng.integers(0, int(s.initial.timestamps[-1]), size=n_new)).astype(np.int64)
    dels = og.live_ids()[::11][:6]
    want = og.apply_batch(off, mem, ts, dels)
    got = r.apply_batch(off, mem, ts, dels.astype(np.int32))
    assert np.array_equal(got, want), "IDs after restore differ"
    got_orig = g.apply_batch(off, mem, ts, dels.astype(np.int32))
    assert np.array_equal(got_orig, want)
    assert_counts_equal(r.counts(), O.counts(og, families, delta), "after the next batch")
    assert_store_equal(r, og)
    g.close()
    r.close()


def test_restore_empty_and_single(E):
    cfg = dict(capacity_hyperedges=64, capacity_incidences=1024, max_batch_hyperedges=64,
               max_batch_incidences=1024)
    empty = dict(ids=np.zeros(0, np.int32), offsets=np.zeros(1, np.int64), members=np.zeros(0, np.int32),
                 timestamps=np.zeros(0, np.int64))
    r = E.Graph.restore(10, empty, families=ALL, delta=5, **cfg)
    assert r.export()["ids"].size == 0
    assert all(int(v.sum()) == 0 for v in r.counts().values())
    # one hyperedge under ID 40: the next insert takes ID 0, the ones after
    # fill the holes, and ID 41 is the first fresh one
    one = dict(ids=np.array([40], np.int32), offsets=np.array([0, 3], np.int64),
               members=np.array([1, 2, 3], np.int32), timestamps=np.array([7], np.int64))
    r2 = E.Graph.restore(10, one, families=ALL, delta=5, **cfg)
    off = np.arange(42, dtype=np.int64) * 2
    mem = np.tile(np.array([2, 4], np.int32), 41)
    ids = r2.apply_batch(off, mem, np.full(41, 9, np.int64))
    assert np.array_equal(ids, np.r_[np.arange(40), 41].astype(np.int32))
    r.close()
    r2.close()


def test_insert_with_ids_rejections_change_nothing(E):
    s = gen.random_small(93, 150, 120, 2, 6)
    init = s.initial
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    g = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=ALL, delta=1 << 40,
                **caps_for(s.n_vertices, 200, 4000, 200, 4000))
    og.apply_batch(np.zeros(1, np.int64), np.zeros(0, np.int32), None, np.array([4, 9], np.int64))
    g.apply_batch(np.zeros(1, np.int64), np.zeros(0, np.int32), None, np.array([4, 9], np.int32))
    before = g.counts()
    off = np.array([0, 2, 5], np.int64)
    mem = np.array([1, 2, 3, 4, 5], np.int32)
    ts = np.array([10, 11], np.int64)
    cap = int(g.cfg.capacity_hyperedges)
    for ids, status in (([4, 4], 1),          # repeated
                        ([4, 5], 1),          # 5 is live
                        ([9, cap + 31], 2)):  # outside the ID range
        with pytest.raises(E.EscError) as e:
            g.insert_with_ids(np.array(ids, np.int32), off, mem, ts)
        assert e.value.status == status, ids
        assert_counts_equal(g.counts(), before, f"after rejecting {ids}")
        assert_store_equal(g, og)
    with pytest.raises(E.EscError) as e:  # the temporal family needs timestamps
        g.insert_with_ids(np.array([4, 9], np.int32), off, mem, None)
    assert e.value.status == 1
    # accepted: the two freed IDs are taken back under the caller's order
    g.insert_with_ids(np.array([9, 4], np.int32), off, mem, ts)
    want_ids = og.apply_batch(np.array([0, 3, 5], np.int64), np.array([3, 4, 5, 1, 2], np.int32),
                              np.array([11, 10], np.int64), np.zeros(0, np.int64))
    assert np.array_equal(want_ids, [4, 9])  # the oracle's ID rule gives the same IDs
    assert_counts_equal(g.counts(), O.counts(og, ALL, 1 << 40), "after the accepted insert")
    assert_store_equal(g, og)
    g.close()


def test_group_export_and_restore(E):
    streams = [gen.random_small(95 + i, 160, 130, 2, 7, n_batches=2, n_ins=30, n_del=25) for i in range(3)]
    delta = 1 << 50
    shared = E.make_config(1, 1, 1, 1000, 20000, ALL, delta)
    cfgs = [E.make_config(st.n_vertices, 400, 4000, 0, 0, ALL, delta) for st in streams]
    grp = E.esc_group_create(shared, cfgs)
    grp2 = E.esc_group_create(shared, cfgs)
    try:
        ogs = []
        E.esc_group_apply(grp, [dict(graph=i, ins_offsets=st.initial.offsets, ins_members=st.initial.members,
                                     ins_timestamps=st.initial.timestamps, del_ids=None)
                                for i, st in enumerate(streams)])
        for i, st in enumerate(streams):
            og = OracleHypergraph(st.n_vertices, st.initial.offsets, st.initial.members, st.initial.timestamps)
            for b in st.batches:
                dels = og.resolve_ranks(b.del_ranks)
                og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels)
                E.esc_group_apply(grp, [dict(graph=i, ins_offsets=b.inserts.offsets, ins_members=b.inserts.members,
                                             ins_timestamps=b.inserts.timestamps,
                                             del_ids=dels.astype(np.int32))])
            ogs.append(og)
        for i, (st, og) in enumerate(zip(streams, ogs)):
            ck = E.esc_group_export(grp, i, st.n_vertices)
            off, mem, ts, ids = og.csr()
            assert np.array_equal(ck["ids"], ids) and np.array_equal(ck["members"], mem)
            assert np.array_equal(ck["offsets"], off) and np.array_equal(ck["timestamps"], ts)
            E.esc_group_insert_with_ids(grp2, i, ck["ids"], ck["offsets"], ck["members"], ck["timestamps"])
        for i, og in enumerate(ogs):
            want = O.counts(og, ALL, delta)
            for gg in (grp, grp2):
                assert np.array_equal(E.esc_group_triads(gg, i, 0), want["hyperedge"]), i
                assert np.array_equal(E.esc_group_triads(gg, i, 1), want["vertex"]), i
                assert np.array_equal(E.esc_group_triads(gg, i, 2, delta), want["temporal"]), i
            v2h = og.v2h()
            ck2 = E.esc_group_export(grp2, i, streams[i].n_vertices)
            for v in range(og.n_vertices):
                assert np.array_equal(ck2["v_members"][ck2["v_offsets"][v]:ck2["v_offsets"][v + 1]], v2h[v])
    finally:
        E.esc_group_destroy(grp)
        E.esc_group_destroy(grp2)


@pytest.mark.parametrize("s_min", [1, 2])
def test_h2h_export_is_the_line_graph(E, s_min):
    import networkx as nx
    s = gen.random_small(97, 90, 80, 2, 7, n_batches=2, n_ins=20, n_del=15)
    g, og = run_stream(E, s, 1, 0, caps=caps_for(s.n_vertices, 200, 4000, 200, 4000))
    ex = g.export_h2h(s_min)
    ids = og.live_ids()
    sets = {int(h): set(og.edge(int(h)).tolist()) for h in ids}
    for k, h in enumerate(ids):
        want = [(int(x), len(sets[int(h)] & sets[int(x)])) for x in ids
                if x != h and len(sets[int(h)] & sets[int(x)]) >= s_min]
        lo, hi = ex["offsets"][k], ex["offsets"][k + 1]
        got = list(zip(ex["neighbours"][lo:hi].tolist(), ex["overlaps"][lo:hi].tolist()))
        assert got == want, f"hyperedge {h}"
    if s_min == 1:
        # closed hyperedge triads (pairwise intersecting) are the line graph's triangles
        L = nx.Graph()
        L.add_nodes_from(ids.tolist())
        for k, h in enumerate(ids):
            for x in ex["neighbours"][ex["offsets"][k]:ex["offsets"][k + 1]]:
                L.add_edge(int(h), int(x))
        closed = O.tables()["static_closed"]
        h_counts = g.triads(E.TRIAD_HYPEREDGE)
        assert sum(int(h_counts[i]) for i in range(30) if closed[i]) == sum(nx.triangles(L).values()) // 3
    g.close()

"""Bit-exact parity of the CUDA path with the CPU oracle (uint64 counts,
identical incidence sets, identical assigned IDs), through the C ABI."""
import os

import numpy as np
import pytest

import gen
from oracle import OracleHypergraph
from oracle import oracle as O
from tests.harness import GpuLive, assert_counts_equal, assert_store_equal, caps_for, run_stream

pytestmark = pytest.mark.gpu

ALL = 7


@pytest.fixture(scope="module")
def E():
    import torch
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    torch.cuda.init()
    return escher


def test_tiny_config_all_families(E):
    """2,000 vertices, 1,000 hyperedges of 2..8 members, one batch of 100
    inserts and 100 deletes (the tiny configuration)."""
    s = gen.tiny(0)
    delta = int(s.initial.timestamps[-1] // 4)
    run_stream(E, s, ALL, delta, method="brute", local_check=True)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_multi_batch_streams(E, seed):
    s = gen.random_small(seed, 400, 300, 1, 9, n_batches=4, n_ins=40, n_del=40)
    delta = int(s.initial.timestamps[-1] // 3)
    run_stream(E, s, ALL, delta)


def test_device_resident_inputs(E):
    import torch
    s = gen.random_small(4, 300, 200, 2, 7, n_batches=2, n_ins=30, n_del=30)
    run_stream(E, s, ALL, 1 << 60, device=torch.device("cuda:0"))


@pytest.mark.parametrize("families", [ALL, 3])
def test_zipf_cards_and_hub_vertices(E, families):
    """Zipf(2) cardinalities up to 100 (the block sorter path) and Zipf(1.1)
    vertex popularity (hubs)."""
    s = gen.random_small(5, 600, 220, 2, 100, n_batches=2, n_ins=25, n_del=25,
                         membership="zipf", card="zipf")
    run_stream(E, s, families, 1 << 60)


def test_repeated_members_ties_and_identical_sets(E):
    rng = np.random.default_rng(6)
    edges = [sorted(rng.choice(40, size=rng.integers(1, 6), replace=False).tolist()) for _ in range(60)]
    edges += [list(e) for e in edges[:12]]                     # identical vertex sets
    off = np.zeros(len(edges) + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.array([v for e in edges for v in e], np.int32)
    ts = rng.integers(0, 10, size=len(edges)).astype(np.int64)  # many equal timestamps
    ins = [[3, 3, 7, 7, 7, 1], [5], [9, 2, 9], [11, 12, 13, 11]]  # repeats collapse
    ioff = np.zeros(len(ins) + 1, np.int64)
    ioff[1:] = np.cumsum([len(e) for e in ins])
    imem = np.array([v for e in ins for v in e], np.int32)
    its = np.array([4, 4, 5, 9], np.int64)
    delta = 6
    og = OracleHypergraph(40, off, mem, ts)
    g = E.Graph(40, off, mem, ts, families=ALL, delta=delta, **caps_for(40, 200, 1000, 100, 1000))
    assert_counts_equal(g.counts(), O.counts(og, ALL, delta, "brute"), "initial")
    dels = np.array([0, 5, 61, 70], np.int64)
    ids_o = og.apply_batch(ioff, imem, its, dels)
    ids_g = g.apply_batch(ioff, imem, its, dels.astype(np.int32))
    assert np.array_equal(ids_g, ids_o)
    assert_counts_equal(g.counts(), O.counts(og, ALL, delta, "brute"), "after")
    assert_store_equal(g, og)


@pytest.mark.parametrize("families", [ALL, 3])
def test_large_neighbourhoods_use_global_tables(E, families):
    """A hyperedge meeting more than the shared-memory tables hold: N(h) and
    N(g1) go to the per-block global tables."""
    rng = np.random.default_rng(7)
    nv = 3000
    big = sorted(rng.choice(nv, size=600, replace=False).tolist())
    edges = [big] + [sorted(rng.choice(nv, size=rng.integers(2, 12), replace=False).tolist())
                     for _ in range(1500)]
    off = np.zeros(len(edges) + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.array([v for e in edges for v in e], np.int32)
    og = OracleHypergraph(nv, off, mem, np.arange(len(edges)))
    g = E.Graph(nv, off, mem, np.arange(len(edges)), families=families, delta=1 << 40,
                **caps_for(nv, 4000, 40000, 2000, 40000))
    assert_counts_equal(g.counts(), O.counts(og, families, 1 << 40), "initial")
    # delete and re-insert the big hyperedge
    ids_o = og.apply_batch(np.array([0, 600]), np.array(big), np.array([7]), np.array([0]))
    ids_g = g.apply_batch(np.array([0, 600]), np.array(big, np.int32), np.array([7]), np.array([0], np.int32))
    assert np.array_equal(ids_g, ids_o)
    assert_counts_equal(g.counts(), O.counts(og, families, 1 << 40), "after")


@pytest.mark.parametrize("families", [ALL, 3])
def test_multi_pass_and_global_tables(E, monkeypatch, families):
    """Small table limits force the global tables and the partitioned
    (multi-pass) N(g1) build: an unchanged hyperedge B whose vertices gain
    degree becomes a neighbour with more entries than one table holds."""
    monkeypatch.setenv("ESC_COUNT_TABLE_SLOTS", "1024")
    monkeypatch.setenv("ESC_COUNT_SMEM_SLOTS", "64")
    rng = np.random.default_rng(13)
    nv = 400
    B = sorted(rng.choice(nv, size=60, replace=False).tolist())
    edges = [B] + [sorted(rng.choice(nv, size=rng.integers(2, 6), replace=False).tolist()) for _ in range(300)]
    off = np.zeros(len(edges) + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.array([v for e in edges for v in e], np.int32)
    ts = np.arange(len(edges), dtype=np.int64)
    og = OracleHypergraph(nv, off, mem, ts)
    g = E.Graph(nv, off, mem, ts, families=families, delta=1 << 40, **caps_for(nv, 2000, 20000, 1000, 20000))
    assert_counts_equal(g.counts(), O.counts(og, families, 1 << 40), "initial")
    for step in range(3):
        ins = [[B[(7 * j + step) % 60], int(rng.integers(0, nv))] for j in range(120)]
        ins = [sorted(set(e)) for e in ins]
        ioff = np.zeros(len(ins) + 1, np.int64)
        ioff[1:] = np.cumsum([len(e) for e in ins])
        imem = np.array([v for e in ins for v in e], np.int32)
        its = np.full(len(ins), 1000 + step, np.int64)
        dels = og.live_ids()[1:11]
        ids_o = og.apply_batch(ioff, imem, its, dels)
        ids_g = g.apply_batch(ioff, imem, its, dels.astype(np.int32))
        assert np.array_equal(ids_g, ids_o)
        assert_counts_equal(g.counts(), O.counts(og, families, 1 << 40), f"step {step}")
    assert_store_equal(g, og)


def _big_hyperedge_stream(E, families, seed):
    """Large hyperedges over popular vertices are inserted and, in the next
    batch, deleted again; counts, IDs and the store are compared with the
    oracle after every batch."""
    rng = np.random.default_rng(seed)
    nv = 300
    edges = [sorted(rng.choice(nv, size=rng.integers(2, 7), replace=False).tolist()) for _ in range(400)]
    off = np.zeros(len(edges) + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.array([v for e in edges for v in e], np.int32)
    ts = np.arange(len(edges), dtype=np.int64)
    og = OracleHypergraph(nv, off, mem, ts)
    g = E.Graph(nv, off, mem, ts, families=families, delta=1 << 40, **caps_for(nv, 2000, 20000, 1000, 20000))
    assert_counts_equal(g.counts(), O.counts(og, families, 1 << 40), "initial")
    big_ids = None
    for step in range(3):
        ins = [sorted(rng.choice(nv, size=int(rng.integers(120, 200)), replace=False).tolist()) for _ in range(4)]
        ins += [sorted(rng.choice(nv, size=int(rng.integers(2, 5)), replace=False).tolist()) for _ in range(20)]
        ioff = np.zeros(len(ins) + 1, np.int64)
        ioff[1:] = np.cumsum([len(e) for e in ins])
        imem = np.array([v for e in ins for v in e], np.int32)
        its = np.full(len(ins), 1000 + step, np.int64)
        live = og.live_ids()
        dels = np.sort(np.concatenate([big_ids if big_ids is not None else np.zeros(0, np.int64),
                                       rng.choice(live[:300], size=10, replace=False)])).astype(np.int64)
        dels = np.unique(dels)
        ids_o = og.apply_batch(ioff, imem, its, dels)
        ids_g = g.apply_batch(ioff, imem, its, dels.astype(np.int32))
        assert np.array_equal(ids_g, ids_o)
        big_ids = np.asarray(ids_o[:2], np.int64)
        assert_counts_equal(g.counts(), O.counts(og, families, 1 << 40), f"step {step}")
    assert_store_equal(g, og)


@pytest.mark.parametrize("families", [ALL, 3])
def test_neighbourhoods_built_in_place(E, monkeypatch, families):
    """A changed hyperedge whose neighbourhood is larger than the block's
    hash table (1024 slots here) has its table built in place, in its own
    region of the neighbour lists."""
    monkeypatch.setenv("ESC_COUNT_TABLE_SLOTS", "1024")
    monkeypatch.setenv("ESC_COUNT_SMEM_SLOTS", "64")
    _big_hyperedge_stream(E, families, 17)


@pytest.mark.parametrize("families", [1, 2, 3])
def test_restricted_lists(E, monkeypatch, families):
    """Without the temporal family and with a list pool configured, a large
    N(h) (here from 600 neighbour entries on) gets restricted incidence lists
    R(u), through which the centre kernel meets N(g1) and N(h); with the pool
    too small for some of them the rest take the hash-probing path in the
    same run."""
    monkeypatch.setenv("ESC_COUNT_RMIN", "600")
    monkeypatch.setenv("ESC_COUNT_RPOOL", str(1 << 22))
    _big_hyperedge_stream(E, families, 19)
    monkeypatch.setenv("ESC_COUNT_RPOOL", "12000")
    _big_hyperedge_stream(E, families, 23)


@pytest.mark.parametrize("orient", ["0", "1"])
def test_both_centre_kernels_without_temporal(E, monkeypatch, orient):
    """Without the temporal family closed pairs are searched once in (|g|, g)
    order by default; ESC_COUNT_ORIENT=0 selects the earlier kernel, which
    visits both sides of every closed pair.  Both must equal the oracle on a
    stream with hub vertices and Zipf cardinalities."""
    monkeypatch.setenv("ESC_COUNT_ORIENT", orient)
    s = gen.random_small(27, 500, 700, 2, 40, n_batches=3, n_ins=60, n_del=60, membership="zipf", card="zipf")
    run_stream(E, s, 3, 0)


@pytest.mark.parametrize("orient,coarse,open_max,open_smem", [
    ("0", 1, None, None), ("1", 1, None, None), ("1", 2000, None, None),
    ("1", 1, "16", None), ("1", 2000, "0", None), ("1", 1, None, "16"), ("1", 2000, "64", "8")])
def test_both_centre_kernels_with_temporal(E, monkeypatch, orient, coarse, open_max, open_smem):
    """All three families through both centre kernels.  The oriented one
    counts the open triads centred at h from the time order of N'(h)
    (k_open_h: sorted in shared memory up to ESC_COUNT_OPEN_SMEM entries,
    in the block's global scratch above), or, for a list longer than
    ESC_COUNT_OPEN_MAX, classifies each as it visits N'(h); those centred at
    g1 are counted per chunk by a sweep over N(g1); closed triads take back
    what those counts gave them.  Timestamps divided by `coarse` make many
    ties (ordered by ID), and the window cuts part of the triads."""
    monkeypatch.setenv("ESC_COUNT_ORIENT", orient)
    if open_max is not None:
        monkeypatch.setenv("ESC_COUNT_OPEN_MAX", open_max)
    if open_smem is not None:
        monkeypatch.setenv("ESC_COUNT_OPEN_SMEM", open_smem)
    s = gen.random_small(31, 400, 600, 2, 30, n_batches=3, n_ins=60, n_del=60, membership="zipf", card="zipf")
    if coarse > 1:
        s.initial.timestamps[:] //= coarse
        for b in s.batches:
            b.inserts.timestamps[:] //= coarse
    span = int(s.initial.timestamps[-1] - s.initial.timestamps[0])
    run_stream(E, s, ALL, max(span // 5, 1))


@pytest.mark.parametrize("families", [3, ALL])
def test_unsorted_neighbourhood_without_table(E, monkeypatch, families):
    """A changed hyperedge with more than 4096 distinct neighbours (too many
    to sort) and, with ESC_COUNT_BIGNH raised, no hash table: the centre
    kernel visits its whole N(h), testing the (|g|, g) order per entry."""
    monkeypatch.setenv("ESC_COUNT_BIGNH", "8192")
    rng = np.random.default_rng(29)
    nv = 200
    edges = [sorted(rng.choice(nv, size=2, replace=False).tolist()) for _ in range(4500)]
    off = np.zeros(len(edges) + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.array([v for e in edges for v in e], np.int32)
    ts = np.arange(len(edges), dtype=np.int64)
    og = OracleHypergraph(nv, off, mem, ts)
    delta = 1500  # the initial timestamps run 0..4499: the window cuts part of the triads
    g = E.Graph(nv, off, mem, ts, families=families, delta=delta, **caps_for(nv, 10000, 40000, 2000, 20000))
    assert_counts_equal(g.counts(), O.counts(og, families, delta), "initial")
    big = sorted(rng.choice(nv, size=150, replace=False).tolist())
    # the initial hyperedges hold IDs 0..n-1 on both sides: delete five of them
    ids_o = og.apply_batch(np.array([0, 150]), np.array(big), np.array([9000]), np.arange(5))
    ids_g = g.apply_batch(np.array([0, 150]), np.array(big, np.int32), np.array([9000]), np.arange(5, dtype=np.int32))
    assert np.array_equal(ids_g, ids_o)
    assert_counts_equal(g.counts(), O.counts(og, families, delta), "after insert")
    ids_o2 = og.apply_batch(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int64), ids_o)
    ids_g2 = g.apply_batch(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int64),
                           np.asarray(ids_g, np.int32))
    assert ids_o2.size == 0 and len(ids_g2) == 0
    assert_counts_equal(g.counts(), O.counts(og, families, delta), "after delete")


@pytest.mark.parametrize("families", [1, 2, 4, 3, 5, 6])
def test_family_subsets(E, families):
    s = gen.random_small(9, 300, 200, 2, 7, n_batches=1, n_ins=30, n_del=30)
    run_stream(E, s, families, int(s.initial.timestamps[-1] // 2), check_store=False)


def test_edge_cases_empty_and_degenerate(E):
    # empty initial graph, insert-only, delete-only, delete everything
    nv = 50
    g = E.Graph(nv, None, None, None, families=ALL, delta=100, **caps_for(nv, 200, 2000, 200, 2000))
    og = OracleHypergraph(nv)
    assert_counts_equal(g.counts(), O.counts(og, ALL, 100), "empty")
    g.apply_batch(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int64), np.zeros(0, np.int32))
    rng = np.random.default_rng(10)
    edges = [sorted(rng.choice(nv, size=rng.integers(1, 5), replace=False).tolist()) for _ in range(40)]
    off = np.zeros(41, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.array([v for e in edges for v in e], np.int32)
    ts = np.arange(40, dtype=np.int64) * 7
    ids_o = og.apply_batch(off, mem, ts, np.zeros(0, np.int64))
    ids_g = g.apply_batch(off, mem, ts, None)
    assert np.array_equal(ids_g, ids_o)
    assert_counts_equal(g.counts(), O.counts(og, ALL, 100), "insert-only")
    dels = np.arange(0, 40, 3)
    og.apply_batch(np.zeros(1, np.int64), np.zeros(0), None, dels)
    g.apply_batch(None, None, None, dels.astype(np.int32))
    assert_counts_equal(g.counts(), O.counts(og, ALL, 100), "delete-only")
    rest = og.live_ids()
    og.apply_batch(np.zeros(1, np.int64), np.zeros(0), None, rest)
    g.apply_batch(None, None, None, rest.astype(np.int32))
    assert_counts_equal(g.counts(), O.counts(og, ALL, 100), "all deleted")
    for v in g.counts().values():
        assert not np.any(v)
    assert_store_equal(g, og)


def test_invalid_batches_leave_graph_unchanged(E):
    s = gen.random_small(11, 200, 100, 2, 6)
    caps = caps_for(200, 150, 1000, 100, 1000)
    g = E.Graph(200, s.initial.offsets, s.initial.members, s.initial.timestamps, families=ALL, delta=1 << 50, **caps)
    before = g.counts()
    ex0 = g.export()
    bad = [
        dict(ins_offsets=np.array([0, 2]), ins_members=np.array([1, 999], np.int32), ins_timestamps=np.array([1]),
             del_ids=None, code=1),          # vertex out of range
        dict(ins_offsets=np.array([0, 0]), ins_members=np.zeros(0, np.int32), ins_timestamps=np.array([1]),
             del_ids=None, code=1),          # empty hyperedge
        dict(ins_offsets=None, ins_members=None, ins_timestamps=None, del_ids=np.array([3, 3], np.int32), code=1),
        dict(ins_offsets=None, ins_members=None, ins_timestamps=None, del_ids=np.array([140], np.int32), code=2),
        dict(ins_offsets=np.array([0, 2]), ins_members=np.array([1, 2], np.int32), ins_timestamps=np.array([1]),
             del_ids=np.array([5, 150], np.int32), code=2),   # valid insert, one bad delete
        dict(ins_offsets=np.arange(0, 102, dtype=np.int64), ins_members=np.arange(101, dtype=np.int32) % 200,
             ins_timestamps=np.arange(101), del_ids=None, code=3),   # more than max_batch_hyperedges
    ]
    for b in bad:
        code = b.pop("code")
        with pytest.raises(E.EscError) as ei:
            g.apply_batch(**b)
        assert ei.value.status == code, (ei.value, code)
        assert_counts_equal(g.counts(), before, "after a rejected batch")
        ex = g.export()
        for k in ex0:
            assert np.array_equal(ex[k], ex0[k]), k
    # the graph still works
    og = OracleHypergraph(200, s.initial.offsets, s.initial.members, s.initial.timestamps)
    ids_o = og.apply_batch(np.array([0, 3]), np.array([4, 5, 6]), np.array([9]), np.array([1, 2]))
    ids_g = g.apply_batch(np.array([0, 3]), np.array([4, 5, 6], np.int32), np.array([9]), np.array([1, 2], np.int32))
    assert np.array_equal(ids_g, ids_o)
    assert_counts_equal(g.counts(), O.counts(og, ALL, 1 << 50), "recovered")


def test_out_of_capacity_is_rejected_cleanly(E):
    g = E.Graph(100, None, None, None, families=ALL, delta=10, capacity_hyperedges=32,
                capacity_incidences=64, max_batch_hyperedges=100, max_batch_incidences=1000)
    off = np.arange(0, 41, dtype=np.int64)
    with pytest.raises(E.EscError) as ei:
        g.apply_batch(off, np.arange(40, dtype=np.int32), np.arange(40), None)
    assert ei.value.status == 3
    for v in g.counts().values():
        assert not np.any(v)


def test_local_triads_match_oracle(E):
    s = gen.random_small(12, 300, 250, 2, 8)
    g = E.Graph(300, s.initial.offsets, s.initial.members, s.initial.timestamps, families=ALL,
                delta=1 << 50, **caps_for(300, 300, 3000, 300, 3000))
    og = OracleHypergraph(300, s.initial.offsets, s.initial.members, s.initial.timestamps)
    off, mem, ts, ids = og.csr()
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(len(ids), size=17, replace=False))
    h, t = O.count_containing(off, mem, ts, ids, 1 << 50, 5, sel)
    got = g.local_triads(ids[sel])
    assert np.array_equal(got["hyperedge"], h)
    assert np.array_equal(got["temporal"], t)
    full = g.local_triads(ids)
    assert_counts_equal(full, g.counts(), "recount")


def test_group_matches_single_graphs(E):
    streams = [gen.random_small(20 + i, 150 + 30 * i, 100 + 40 * i, 2, 7, n_batches=1, n_ins=15 + i,
                                n_del=10 + i) for i in range(5)]
    delta = 1 << 50
    shared = E.make_config(1, 1, 1, 4000, 40000, ALL, delta)
    cfgs = [E.make_config(s.n_vertices, 400, 4000, 0, 0, ALL, delta) for s in streams]
    grp = E.esc_group_create(shared, cfgs)
    try:
        ogs = []
        first = [dict(graph=i, ins_offsets=s.initial.offsets, ins_members=s.initial.members,
                      ins_timestamps=s.initial.timestamps, del_ids=None) for i, s in enumerate(streams)]
        E.esc_group_apply(grp, first)
        for i, s in enumerate(streams):
            og = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
            ogs.append(og)
            want = O.counts(og, ALL, delta)
            assert np.array_equal(E.esc_group_triads(grp, i, 0), want["hyperedge"])
        batches, expect_ids = [], []
        for i in (4, 1, 3):   # a subset, out of order
            s, og = streams[i], ogs[i]
            b = s.batches[0]
            dels = og.resolve_ranks(b.del_ranks)
            expect_ids.append(og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels))
            out = np.zeros(b.inserts.n, np.int32)
            batches.append(dict(graph=i, ins_offsets=b.inserts.offsets, ins_members=b.inserts.members,
                                ins_timestamps=b.inserts.timestamps, del_ids=dels.astype(np.int32), out_ids=out))
        E.esc_group_apply(grp, batches)
        for b, want_ids in zip(batches, expect_ids):
            assert np.array_equal(b["out_ids"], want_ids)
        for i, og in enumerate(ogs):
            want = O.counts(og, ALL, delta)
            assert np.array_equal(E.esc_group_triads(grp, i, 0), want["hyperedge"]), i
            assert np.array_equal(E.esc_group_triads(grp, i, 1), want["vertex"]), i
            assert np.array_equal(E.esc_group_triads(grp, i, 2, delta), want["temporal"]), i
    finally:
        E.esc_group_destroy(grp)


def test_temporal_stream_with_expirations(E):
    """Time-ordered stream (scaled temporal configuration): every batch
    inserts the next hyperedges and deletes those older than T - delta."""
    ts_stream = gen.temporal(seed=3, scale=0.0005, batch=256, n_batches=6, kmax=12)
    delta = int(ts_stream.delta // 7200)
    from tests.harness import GpuLive
    nv = ts_stream.n_vertices
    g = E.Graph(nv, None, None, None, families=ALL, delta=delta,
                **caps_for(nv, 4000, 60000, 2000, 20000))
    og = OracleHypergraph(nv)
    live = GpuLive(0)
    for k, b in enumerate(ts_stream.batches):
        t_cut = int(b.timestamps.max()) - delta
        dels_o = np.array([i for i in og.live_ids() if og.ts[i] < t_cut], np.int64)
        dels_g = live.expired(t_cut)
        ids_o = og.apply_batch(b.offsets, b.members, b.timestamps, dels_o)
        ids_g = g.apply_batch(b.offsets, b.members, b.timestamps, dels_g.astype(np.int32))
        assert np.array_equal(ids_g, ids_o)
        live.apply(dels_g, ids_g, b.timestamps)
        assert_counts_equal(g.counts(), O.counts(og, ALL, delta), f"batch {k}")


@pytest.mark.parametrize("families", [ALL, 3])
def test_large_overlaps(E, families):
    """Pairs of hyperedges sharing more than 64 vertices (outside the
    aggregated counter's histogram window) and nested hyperedges."""
    rng = np.random.default_rng(14)
    nv = 500
    edges = []
    for _ in range(12):
        core = sorted(rng.choice(nv, size=150, replace=False).tolist())
        edges.append(core)
        edges.append(sorted(set(core[:100]) | set(rng.choice(nv, size=20).tolist())))
        edges.append(core[10:90])
    edges += [sorted(rng.choice(nv, size=rng.integers(2, 8), replace=False).tolist()) for _ in range(150)]
    off = np.zeros(len(edges) + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.array([v for e in edges for v in e], np.int32)
    ts = np.arange(len(edges), dtype=np.int64)
    og = OracleHypergraph(nv, off, mem, ts)
    g = E.Graph(nv, off, mem, ts, families=families, delta=1 << 40, **caps_for(nv, 600, 20000, 400, 20000))
    assert_counts_equal(g.counts(), O.counts(og, families, 1 << 40), "initial")
    dels = np.array([0, 4, 8, 40, 41, 100], np.int64)
    ins = [list(range(0, 120)), list(range(50, 130)), [1, 2, 3]]
    ioff = np.zeros(len(ins) + 1, np.int64)
    ioff[1:] = np.cumsum([len(e) for e in ins])
    imem = np.array([v for e in ins for v in e], np.int32)
    its = np.array([500, 501, 502], np.int64)
    ids_o = og.apply_batch(ioff, imem, its, dels)
    ids_g = g.apply_batch(ioff, imem, its, dels.astype(np.int32))
    assert np.array_equal(ids_g, ids_o)
    assert_counts_equal(g.counts(), O.counts(og, families, 1 << 40), "after")


@pytest.mark.parametrize("families", [3, ALL])
def test_autotune_keeps_counts_exact(E, families):
    """The autotuner times every launch shape (and, without the temporal
    family, restricted lists), then the neighbourhood size from which N(h)
    gets a table and filter and the per-pair side weight, on a sample of
    live hyperedges, and keeps the fastest of each; counts are untouched by
    it and stay exact afterwards, under the chosen strategy."""
    s = gen.random_small(31, 500, 700, 2, 12, membership="zipf", n_batches=2, n_ins=60, n_del=60)
    init = s.initial
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    delta = int(init.timestamps[-1] // 2)
    g = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=families, delta=delta,
                **caps_for(s.n_vertices, 2000, 20000, 1000, 20000))
    before = g.counts()
    res = g.autotune(np.arange(0, init.n, 3, dtype=np.int32), reps=1)
    assert 0 <= res["center_shape"] <= 3
    assert all(m >= 0 for m in res["ms"][:4])
    if families & 4:
        assert res["restricted"] == 0 and all(m == -1 for m in res["ms"][4:])
    assert res["table_from"] in (256, 512, 1024) and res["m1_pct"] in (50, 100, 200)
    assert all(m >= 0 for m in res["ms_table"]) and all(m >= 0 for m in res["ms_m1"])
    assert_counts_equal(g.counts(), before, "after tuning")
    live = GpuLive(init.n, init.timestamps)
    for b in s.batches:
        dels_o = og.resolve_ranks(b.del_ranks)
        dels_g = live.resolve(b.del_ranks)
        ids_o = og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_o)
        ids_g = g.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_g.astype(np.int32))
        assert np.array_equal(ids_g, ids_o)
        live.apply(dels_g, ids_g, b.inserts.timestamps)
        assert_counts_equal(g.counts(), O.counts(og, families, delta), "after a batch")
    with pytest.raises(E.EscError):
        g.autotune(np.array([10 ** 6], np.int32))


def test_maximum_cardinality(E):
    """A hyperedge of exactly the largest accepted size (16,384 members)
    among small ones; one member more is rejected with nothing changed; a
    16,384-member input with every vertex twice collapses to 8,192."""
    nv = 20000
    fam = 5  # hyperedge + temporal (the oracle's vertex counter enumerates vertex triples)
    rng = np.random.default_rng(31)
    sets = [rng.permutation(nv)[:16384]] + [rng.choice(nv, size=int(rng.integers(2, 6)), replace=False)
                                           for _ in range(300)]
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in sets])
    mem = np.concatenate(sets).astype(np.int32)
    ts = np.arange(len(sets), dtype=np.int64) * 3
    delta = 400
    og = OracleHypergraph(nv, off, mem, ts)
    g = E.Graph(nv, off, mem, ts, families=fam, delta=delta, **caps_for(nv, 1000, 60000, 400, 40000))
    assert_counts_equal(g.counts(), O.counts(og, fam, delta), "initial")
    before = g.counts()
    with pytest.raises(E.EscError) as ei:
        g.apply_batch(np.array([0, 16385], np.int64), rng.permutation(nv)[:16385].astype(np.int32),
                      np.array([999], np.int64), None)
    assert ei.value.status == 4
    assert_counts_equal(g.counts(), before, "after the rejected batch")
    twice = np.repeat(rng.permutation(nv)[:8192], 2).astype(np.int32)
    want = og.apply_batch(np.array([0, 16384], np.int64), twice, np.array([1000], np.int64), np.array([0]))
    got = g.apply_batch(np.array([0, 16384], np.int64), twice, np.array([1000], np.int64), np.array([0], np.int32))
    assert np.array_equal(got, want)
    assert_counts_equal(g.counts(), O.counts(og, fam, delta), "after the big replacement")
    assert_store_equal(g, og)
    g.close()


def test_hub_vertex_lists_rewritten_by_blocks(E):
    """Vertices in thousands of hyperedges: v2h lists of 2,048 entries and
    more are rewritten by a whole block, in chunks of 4,096, in place when
    the slab still fits.  Deletes in place, a list that outgrows its slab
    while losing entries, and a list that shrinks below 2,048; the store and
    the assigned IDs equal the oracle's after every batch (incident-vertex
    types 1 and 2 from pair statistics keep the oracle's counting cheap)."""
    rng = np.random.default_rng(37)
    nv = 3000

    def make(n):
        out = []
        for _ in range(n):
            m = set(rng.choice(np.arange(2, nv), size=int(rng.integers(1, 5)), replace=False).tolist())
            m.add(0)
            if rng.random() < 0.3:
                m.add(1)
            out.append(sorted(m))
        return out

    def csr(edges):
        off = np.zeros(len(edges) + 1, np.int64)
        off[1:] = np.cumsum([len(e) for e in edges])
        return off, np.array([v for e in edges for v in e], np.int32)

    init = make(9000)
    batches = [(1500, make(500)), (700, make(12000)), (14000, make(300))]
    sizes = [len(e) for e in init] + [len(e) for _, b in batches for e in b]
    pairs = sum(k * (k - 1) // 2 for k in sizes) + 64
    off, mem = csr(init)
    ts = np.arange(len(init), dtype=np.int64)
    og = OracleHypergraph(nv, off, mem, ts)
    g = E.Graph(nv, off, mem, ts, families=8, capacity_vertex_pairs=pairs,
                **caps_for(nv, 30000, 120000, 16000, 60000))
    assert_store_equal(g, og)
    t = len(init)
    for k, (n_del, ins) in enumerate(batches):
        live = og.live_ids()
        dels = np.sort(rng.choice(live, size=min(n_del, len(live)), replace=False)).astype(np.int64)
        o, m = csr(ins)
        tsb = np.arange(t, t + len(ins), dtype=np.int64)
        t += len(ins)
        ids_o = og.apply_batch(o, m, tsb, dels)
        ids_g = g.apply_batch(o, m, tsb, dels.astype(np.int32))
        assert np.array_equal(ids_g, ids_o), f"batch {k}"
        assert_store_equal(g, og)
    g.close()


def test_debug_mode_checks_the_store_after_every_call(E, tmp_path, monkeypatch):
    """esc_config.debug = 1 checks the store's invariants on the device after
    every call (the two views agree, members sorted and in range, degrees
    within their slabs, live counts); a stream with hub vertices and
    single-member hyperedges passes every check with counts and store equal
    to the oracle's.  ESC_STATS_JSONL records one line per call.  A debug
    value other than 0 or 1 is refused."""
    import json
    path = tmp_path / "calls.jsonl"
    monkeypatch.setenv("ESC_STATS_JSONL", str(path))
    s = gen.random_small(33, 300, 400, 1, 20, n_batches=3, n_ins=80, n_del=80, membership="zipf", card="zipf")
    init = s.initial
    delta = int(init.timestamps[-1] // 3)
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    g = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=ALL, delta=delta, debug=1,
                **caps_for(s.n_vertices, 2000, 20000, 1000, 20000))
    g.set_profiling(True)
    live = GpuLive(init.n, init.timestamps)
    for b in s.batches:
        dels_o = og.resolve_ranks(b.del_ranks)
        dels_g = live.resolve(b.del_ranks)
        ids_o = og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_o)
        ids_g = g.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_g.astype(np.int32))
        assert np.array_equal(ids_g, ids_o)
        live.apply(dels_g, ids_g, b.inserts.timestamps)
        assert_counts_equal(g.counts(), O.counts(og, ALL, delta), "debug mode")
        assert_store_equal(g, og)
    g.close()
    rec = [json.loads(line) for line in open(path)]
    assert len(rec) >= 1 + len(s.batches)
    for r, b in zip(rec[-len(s.batches):], s.batches):
        assert r["status"] == 0 and r["inserts"] == b.inserts.n and r["deletes"] == len(b.del_ranks)
        assert r["launches"] > 0 and r["ms_total"] > 0 and len(r["work"]) == 6
    with pytest.raises(E.EscError):
        E.Graph(10, None, None, None, families=1, debug=2, **caps_for(10, 64, 1024, 64, 1024))

"""Parity at the benchmark's full size, in the launch configuration the
benchmark times (the uniform 1M-vertex, 2M-hyperedge graph, batches of
5e4 inserts + 5e4 deletes, hyperedge and incident-vertex families, counter
shape picked by the autotuner on a sample of one batch's size).

After two batches: the assigned IDs and the whole store equal the oracle's;
the incrementally kept counts equal a full recount of every live hyperedge
(a property that holds at any size); and the triads holding a few sampled
hyperedges, counted by the oracle's own enumeration on its own copy of the
graph, equal the library's local counts for the same hyperedges.  Then a
small batch on the same graph: its count change, for both families, equals
the oracle's count of the triads (hyperedge family) and witness assignments
(incident-vertex family) holding an inserted hyperedge on the new graph
minus those holding a deleted one on the old graph (Alg. 3)."""
import numpy as np
import pytest

import gen
from harness import LiveIds
from oracle import OracleHypergraph
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    return escher


M64 = 1 << 64


def check_small_batch(g, og, live, seed, families, n=3, kmax=64):
    """Apply n inserts and n deletes (cardinality <= kmax, so that the oracle
    enumerates their triads in seconds) and compare the library's count
    change with the oracle's Alg. 3 terms for every family in `families`."""
    rng = np.random.default_rng(seed)
    off0, mem0, ts0, ids0 = og.csr()
    small = np.flatnonzero(np.diff(off0) <= kmax)
    ranks = np.sort(rng.choice(small, size=n, replace=False))   # positions = ranks among live IDs
    ins = gen.insert_batches(seed, og.n_vertices, 1, n, kmax, ts_start=int(ts0.max()))[0]
    before = g.counts()
    dels_o = og.resolve_ranks(ranks)
    want_ids = og.apply_batch(ins.offsets, ins.members, ins.timestamps, dels_o)
    dels_g = live.resolve(ranks)
    got_ids = g.apply_batch(ins.offsets, ins.members, ins.timestamps, dels_g.astype(np.int32))
    assert np.array_equal(got_ids, want_ids), "small batch: assigned IDs differ"
    live.apply(dels_g, got_ids)
    after = g.counts()
    off1, mem1, ts1, ids1 = og.csr()
    p0, p1 = np.searchsorted(ids0, dels_o), np.searchsorted(ids1, want_ids)
    terms = {}
    if "hyperedge" in families:
        terms["hyperedge"] = (O.count_containing(off0, mem0, ts0, ids0, 0, O.FAM_HYPEREDGE, p0)[0],
                              O.count_containing(off1, mem1, ts1, ids1, 0, O.FAM_HYPEREDGE, p1)[0])
    if "vertex" in families:
        terms["vertex"] = (O.count_vertex_containing(off0, mem0, p0), O.count_vertex_containing(off1, mem1, p1))
    moved = 0
    for fam, (d, i) in terms.items():
        got = [(int(a) - int(b)) % M64 for a, b in zip(after[fam], before[fam])]
        want = [(int(x) - int(y)) % M64 for x, y in zip(i, d)]
        assert got == want, f"small batch, {fam}: library change {got}, oracle {want}"
        moved += int(d.sum()) + int(i.sum())
    assert moved > 0


def test_full_size_batches(E):
    import torch
    s = gen.large(seed=2, membership="uniform", scale=1.0, n_batches=2, batch_updates=100_000)
    init = s.initial
    dev = torch.device("cuda", 0)
    todev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)  # noqa: E731
    # the benchmark's capacities and batch limits
    max_bh = max(100_000, min(init.n, 100_000))
    max_bi = max(max(b.inserts.nnz for b in s.batches), 4 * max_bh * 16)
    g = E.Graph(s.n_vertices, todev(init.offsets, np.int64), todev(init.members, np.int32),
                todev(init.timestamps, np.int64),
                capacity_hyperedges=init.n + max(b.inserts.n for b in s.batches) + 64,
                capacity_incidences=int(init.nnz * 1.6) + 4 * max(b.inserts.nnz for b in s.batches),
                max_batch_hyperedges=max_bh, max_batch_incidences=max_bi, families=3,
                stream=torch.cuda.current_stream(dev))
    rng = np.random.default_rng(19)
    g.autotune(np.sort(rng.choice(init.n, size=100_000, replace=False)).astype(np.int32), reps=1)
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    live = LiveIds(np.arange(init.n))
    for k, b in enumerate(s.batches):
        dels_o = og.resolve_ranks(b.del_ranks)
        want = og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_o)
        dels_g = live.resolve(b.del_ranks)
        got = g.apply_batch(todev(b.inserts.offsets, np.int64), todev(b.inserts.members, np.int32),
                            todev(b.inserts.timestamps, np.int64), todev(np.sort(dels_g), np.int32))
        assert np.array_equal(got, want), f"batch {k}: assigned IDs differ"
        live.apply(dels_g, got)
    # the store, both views
    ex = g.export()
    off, mem, ts, ids = og.csr()
    assert np.array_equal(ex["ids"], ids)
    assert np.array_equal(ex["offsets"], off)
    assert np.array_equal(ex["members"], mem)
    assert np.array_equal(ex["timestamps"], ts)
    v2h = og.v2h()
    assert np.array_equal(ex["v_offsets"][1:], np.cumsum([len(x) for x in v2h]))
    assert np.array_equal(ex["v_members"], np.concatenate(v2h).astype(np.int32))
    # incremental counts == full recount of every live hyperedge
    counts = g.counts()
    full = g.local_triads(ids.astype(np.int32))
    for fam in ("hyperedge", "vertex"):
        assert np.array_equal(counts[fam], full[fam]), fam
    # sampled hyperedges: the oracle's enumeration of the triads holding them
    sel = np.sort(rng.choice(ids.size, size=3, replace=False))
    h30, _ = O.count_containing(off, mem, ts, ids, 0, O.FAM_HYPEREDGE, sel)
    loc = g.local_triads(ids[sel].astype(np.int32))
    assert np.array_equal(loc["hyperedge"], h30)
    assert int(h30.sum()) > 0
    # Alg. 3 on the benchmark graph, both families, against the oracle
    for seed in (29, 31):
        check_small_batch(g, og, live, seed, ("hyperedge", "vertex"))
    g.close()


def test_full_size_temporal_stream(E):
    """The temporal stream at full size (4M hyperedges over 2M vertices in
    batches of 2^16, each batch deleting every live hyperedge older than
    T - delta): IDs after every batch, the store at the end, the running
    temporal counts against a full recount, and sampled enumerations by
    the oracle."""
    ts = gen.temporal(seed=3, scale=1.0)
    delta = ts.delta
    n_total = sum(b.n for b in ts.batches)
    bmax = max(b.n for b in ts.batches)
    g = E.Graph(ts.n_vertices, None, None, None, capacity_hyperedges=n_total + 64,
                capacity_incidences=sum(b.nnz for b in ts.batches) + 1024, max_batch_hyperedges=4 * bmax,
                max_batch_incidences=max(b.nnz for b in ts.batches) + 1024, families=4, delta=delta)
    og = OracleHypergraph(ts.n_vertices)
    # each side keeps its own live list in insertion order (timestamps grow
    # along the stream, so a batch's expirations are a prefix of it)
    o_ids, o_ts = np.zeros(0, np.int64), np.zeros(0, np.int64)
    g_ids, g_ts = np.zeros(0, np.int64), np.zeros(0, np.int64)
    n_exp_total = 0
    for k, b in enumerate(ts.batches):
        t_cut = int(b.timestamps.max()) - delta
        ne_o = int(np.searchsorted(o_ts, t_cut, side="left"))
        ne_g = int(np.searchsorted(g_ts, t_cut, side="left"))
        want = og.apply_batch(b.offsets, b.members, b.timestamps, np.sort(o_ids[:ne_o]))
        got = g.apply_batch(b.offsets, b.members, b.timestamps, np.sort(g_ids[:ne_g]).astype(np.int32))
        assert np.array_equal(got, want), f"batch {k}: assigned IDs differ"
        o_ids, o_ts = np.concatenate([o_ids[ne_o:], want]), np.concatenate([o_ts[ne_o:], b.timestamps])
        g_ids, g_ts = np.concatenate([g_ids[ne_g:], got]), np.concatenate([g_ts[ne_g:], b.timestamps])
        n_exp_total += ne_o
    assert n_exp_total > 0  # the window filled and hyperedges expired
    ex = g.export()
    off, mem, tsv, ids = og.csr()
    assert np.array_equal(ex["ids"], ids)
    assert np.array_equal(ex["offsets"], off)
    assert np.array_equal(ex["members"], mem)
    assert np.array_equal(ex["timestamps"], tsv)
    running = g.triads(E.TRIAD_TEMPORAL)
    full = g.local_triads(ids.astype(np.int32))["temporal"]
    assert np.array_equal(running, full)
    rng = np.random.default_rng(23)
    sel = np.sort(rng.choice(ids.size, size=3, replace=False))
    _, t96 = O.count_containing(off, mem, tsv, ids, delta, O.FAM_TEMPORAL, sel)
    assert np.array_equal(g.local_triads(ids[sel].astype(np.int32))["temporal"], t96)
    assert int(t96.sum()) > 0
    g.close()

"""Graph launch: every call replays one captured CUDA graph of the whole
device work of a call.  Results must be those of the oracle, as without the
graph: streams of batches, a group, a rejected batch (nothing changes), and a
call whose neighbour lists need more count runs than the graph holds (it is
detected inside the graph and run again without it)."""
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
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    return escher


@pytest.mark.parametrize("families", [ALL, 3])
def test_graph_launch_stream(E, monkeypatch, families):
    monkeypatch.setenv("ESC_CALL_GRAPH", "1")
    s = gen.random_small(51, 600, 500, 2, 9, membership="zipf", n_batches=4, n_ins=40, n_del=40)
    run_stream(E, s, families, int(s.initial.timestamps[-1] // 2))


def test_graph_launch_rejected_batch_changes_nothing(E):
    s = gen.random_small(52, 300, 200, 2, 6, n_batches=2, n_ins=20, n_del=20)
    init = s.initial
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    g = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=ALL, delta=1 << 40,
                **caps_for(s.n_vertices, 1000, 10000, 500, 5000))
    g.set_graph_launch(True)
    before = g.counts()
    with pytest.raises(E.EscError):
        g.apply_batch(np.array([0, 2], np.int64), np.array([1, 2], np.int32), np.array([5], np.int64),
                      np.array([999], np.int32))  # not live
    assert_counts_equal(g.counts(), before, "after the rejected batch")
    assert_store_equal(g, og)
    live = GpuLive(init.n, init.timestamps)
    for b in s.batches:
        d_o, d_g = og.resolve_ranks(b.del_ranks), live.resolve(b.del_ranks)
        ids_o = og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, d_o)
        ids_g = g.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, d_g.astype(np.int32))
        assert np.array_equal(ids_g, ids_o)
        live.apply(d_g, ids_g, b.inserts.timestamps)
        assert_counts_equal(g.counts(), O.counts(og, ALL, 1 << 40), "after a batch")
    g.close()


def test_graph_launch_more_runs_than_the_graph_holds(E, monkeypatch):
    """A 4096-entry list arena makes one batch need more than one count run
    per side: the graph's call stops inside with the retry status before
    anything changes and is run again with host-planned runs."""
    monkeypatch.setenv("ESC_CALL_GRAPH", "1")
    monkeypatch.setenv("ESC_COUNT_LIST", "4096")
    s = gen.random_small(53, 400, 600, 3, 10, n_batches=3, n_ins=200, n_del=150)
    run_stream(E, s, ALL, 1 << 40)


def test_graph_launch_group(E):
    streams = [gen.random_small(60 + i, 150 + 20 * i, 120 + 30 * i, 2, 7, n_batches=2, n_ins=15, n_del=10)
               for i in range(4)]
    delta = 1 << 50
    shared = E.make_config(1, 1, 1, 4000, 40000, ALL, delta)
    cfgs = [E.make_config(s.n_vertices, 500, 5000, 0, 0, ALL, delta) for s in streams]
    grp = E.esc_group_create(shared, cfgs)
    try:
        E.esc_group_set_graph_launch(grp, True)
        E.esc_group_apply(grp, [dict(graph=i, ins_offsets=s.initial.offsets, ins_members=s.initial.members,
                                     ins_timestamps=s.initial.timestamps, del_ids=None)
                                for i, s in enumerate(streams)])
        ogs = [OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
               for s in streams]
        for k in range(2):
            batches = []
            for i in (3, 0, 2) if k == 0 else (1, 2):
                b = streams[i].batches[k]
                dels = ogs[i].resolve_ranks(b.del_ranks)
                want = ogs[i].apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels)
                out = np.zeros(b.inserts.n, np.int32)
                batches.append((want, dict(graph=i, ins_offsets=b.inserts.offsets, ins_members=b.inserts.members,
                                           ins_timestamps=b.inserts.timestamps, del_ids=dels.astype(np.int32),
                                           out_ids=out)))
            E.esc_group_apply(grp, [b for _, b in batches])
            for want, b in batches:
                assert np.array_equal(b["out_ids"], want)
            for i, og in enumerate(ogs):
                want = O.counts(og, ALL, delta)
                assert np.array_equal(E.esc_group_triads(grp, i, 0), want["hyperedge"]), i
                assert np.array_equal(E.esc_group_triads(grp, i, 1), want["vertex"]), i
                assert np.array_equal(E.esc_group_triads(grp, i, 2, delta), want["temporal"]), i
    finally:
        E.esc_group_destroy(grp)

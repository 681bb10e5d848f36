"""Horizontal updates (Sec. III-B): incident vertices inserted into and
deleted from live hyperedges, which keep their IDs and timestamps.  After
every update batch, counts and store equal the oracle's; a rejected update
changes nothing; graph launch gives the same results."""
import numpy as np
import pytest

import gen
from oracle import OracleHypergraph
from oracle import oracle as O
from tests.harness import assert_counts_equal, assert_store_equal, caps_for

pytestmark = pytest.mark.gpu

ALL = 7


@pytest.fixture(scope="module")
def E():
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    return escher


def _updates(rng, og, n):
    """n distinct live hyperedges, each with some members dropped and some
    vertices added (repeats included: they collapse)."""
    live = og.live_ids()
    ids = rng.choice(live, size=min(n, len(live)), replace=False)
    sets = []
    for hid in ids:
        cur = og.edge(int(hid))
        keep = cur[rng.random(cur.size) < 0.7]
        add = rng.integers(0, og.n_vertices, size=int(rng.integers(0, 4)))
        new = np.concatenate([keep, add, add[:1]])
        if new.size == 0:
            new = cur[:1]
        sets.append(new)
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in sets])
    return ids.astype(np.int32), off, np.concatenate(sets).astype(np.int32)


@pytest.mark.parametrize("families,graph", [(ALL, False), (3, False), (ALL, True)])
def test_horizontal_updates_match_oracle(E, families, graph):
    s = gen.random_small(71, 300, 260, 2, 8, membership="zipf")
    init = s.initial
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    delta = int(init.timestamps[-1] // 2)
    g = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=families, delta=delta,
                **caps_for(s.n_vertices, 1000, 20000, 1000, 20000))
    if graph:
        g.set_graph_launch(True)
    rng = np.random.default_rng(5)
    for step in range(4):
        ids, off, mem = _updates(rng, og, 30 + 20 * step)
        og.update_members(ids, off, mem)
        g.update_members(ids, off, mem)
        assert_counts_equal(g.counts(), O.counts(og, families, delta), f"step {step}")
    assert_store_equal(g, og)
    # a plain batch after horizontal updates follows the ID rule as usual
    b_off = np.array([0, 3], np.int64)
    b_mem = np.array([1, 2, 3], np.int32)
    dels = og.live_ids()[:2]
    want = og.apply_batch(b_off, b_mem, np.array([123], np.int64), dels)
    got = g.apply_batch(b_off, b_mem, np.array([123], np.int64), dels.astype(np.int32))
    assert np.array_equal(got, want)
    assert_counts_equal(g.counts(), O.counts(og, families, delta), "after a plain batch")
    g.close()


def test_rejected_horizontal_update_changes_nothing(E):
    s = gen.random_small(72, 200, 150, 2, 6)
    init = s.initial
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    g = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=ALL, delta=1 << 40,
                **caps_for(s.n_vertices, 500, 5000, 500, 5000))
    before = g.counts()
    off = np.array([0, 2, 4], np.int64)
    mem = np.array([1, 2, 3, 4], np.int32)
    with pytest.raises(E.EscError) as e1:
        g.update_members(np.array([5, 5], np.int32), off, mem)     # repeated
    assert e1.value.status == 1
    og.apply_batch(np.zeros(1, np.int64), np.zeros(0, np.int32), None, np.array([7], np.int64))
    g.apply_batch(np.zeros(1, np.int64), np.zeros(0, np.int32), None, np.array([7], np.int32))
    before = g.counts()
    with pytest.raises(E.EscError) as e2:
        g.update_members(np.array([3, 7], np.int32), off, mem)     # 7 is not live
    assert e2.value.status == 2
    assert_counts_equal(g.counts(), before, "after the rejected update")
    assert_store_equal(g, og)
    g.close()


def test_horizontal_updates_in_a_group(E):
    streams = [gen.random_small(80 + i, 150, 120, 2, 6) for i in range(3)]
    delta = 1 << 50
    shared = E.make_config(1, 1, 1, 2000, 20000, ALL, delta)
    cfgs = [E.make_config(st.n_vertices, 400, 4000, 0, 0, ALL, delta) for st in streams]
    grp = E.esc_group_create(shared, cfgs)
    try:
        E.esc_group_apply(grp, [dict(graph=i, ins_offsets=st.initial.offsets, ins_members=st.initial.members,
                                     ins_timestamps=st.initial.timestamps, del_ids=None)
                                for i, st in enumerate(streams)])
        ogs = [OracleHypergraph(st.n_vertices, st.initial.offsets, st.initial.members, st.initial.timestamps)
               for st in streams]
        rng = np.random.default_rng(9)
        for i in (2, 0):
            ids, off, mem = _updates(rng, ogs[i], 25)
            ogs[i].update_members(ids, off, mem)
            E.esc_group_update_members(grp, i, ids, off, mem)
        for i, og in enumerate(ogs):
            want = O.counts(og, ALL, delta)
            assert np.array_equal(E.esc_group_triads(grp, i, 0), want["hyperedge"]), i
            assert np.array_equal(E.esc_group_triads(grp, i, 1), want["vertex"]), i
            assert np.array_equal(E.esc_group_triads(grp, i, 2, delta), want["temporal"]), i
    finally:
        E.esc_group_destroy(grp)

"""Incident-vertex types 1 and 2 from vertex-pair statistics
(ESC_FAMILY_VERTEX12) against the oracle.

The oracle counts the three types by definition (per vertex triple, and by
literal witness assignment on tiny inputs); this family keeps types 1 and 2
from the multiplicity and size sum of every vertex pair instead of from
neighbourhoods, and must equal the oracle's types 1 and 2 after every batch
(type 3 reads 0), on hub-bearing graphs, combined with the other families,
in a group, under graph launch and for horizontal updates.  A batch whose
inserted pairs could exceed the configured capacity is refused and changes
nothing.
"""
import numpy as np
import pytest

import gen
from harness import GpuLive, caps_for
from oracle import OracleHypergraph
from oracle import oracle as O

pytestmark = pytest.mark.gpu
V12 = 8


@pytest.fixture(scope="module")
def E():
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    return escher


def _pairs(s):
    sizes = list(np.diff(s.initial.offsets)) + [k for b in s.batches for k in np.diff(b.inserts.offsets)]
    return int(sum(int(k) * (int(k) - 1) // 2 for k in sizes)) + 64


def _check(g, og, fam, delta, where):
    got = g.counts()
    want = O.counts(og, (fam & ~V12) | 2, delta)
    v = [int(x) for x in got["vertex"]]
    assert v[:2] == [int(x) for x in want["vertex"][:2]], f"{where}: {v} vs {want['vertex']}"
    assert v[2] == 0
    for k in ("hyperedge", "temporal"):
        if k in got:
            assert np.array_equal(got[k], want[k]), f"{where} {k}"


def _stream(E, s, fam, delta=0, graph_launch=False):
    init = s.initial
    caps = caps_for(s.n_vertices, 4 * init.n + 4096, 4 * init.nnz + 40000, 4096, 40000)
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    g = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=fam, delta=delta,
                capacity_vertex_pairs=_pairs(s), **caps)
    if graph_launch:
        g.set_graph_launch(True)
    _check(g, og, fam, delta, "initial")
    live = GpuLive(init.n, init.timestamps)
    for k, b in enumerate(s.batches):
        dels_o = og.resolve_ranks(b.del_ranks)
        ids_o = og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_o)
        dels_g = live.resolve(b.del_ranks).astype(np.int32)
        ids_g = g.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_g)
        assert np.array_equal(ids_g, ids_o)
        live.apply(dels_g, ids_g, b.inserts.timestamps)
        _check(g, og, fam, delta, f"batch {k}")
    return g, og


@pytest.mark.parametrize("fam", [V12, V12 | 1, V12 | 4])
def test_vertex12_matches_oracle_on_hub_graphs(E, fam):
    s = gen.random_small(71, 300, 400, 2, 25, n_batches=3, n_ins=60, n_del=60, membership="zipf", card="zipf")
    delta = int(s.initial.timestamps[-1] // 3)
    g, _ = _stream(E, s, fam, delta)
    g.close()


def test_vertex12_graph_launch_and_horizontal(E):
    s = gen.random_small(72, 200, 300, 2, 12, n_batches=2, n_ins=40, n_del=40, membership="zipf")
    g, og = _stream(E, s, V12, 0, graph_launch=True)
    # horizontal updates: members of live hyperedges change in place
    rng = np.random.default_rng(3)
    ids = np.sort(rng.choice(og.live_ids(), size=20, replace=False))
    sets = [np.unique(rng.choice(s.n_vertices, size=int(rng.integers(2, 9)), replace=False)) for _ in ids]
    off = np.concatenate([[0], np.cumsum([len(x) for x in sets])]).astype(np.int64)
    mem = np.concatenate(sets).astype(np.int32)
    og.update_members(ids, off, mem)
    g.update_members(ids.astype(np.int32), off, mem)
    _check(g, og, V12, 0, "horizontal")
    g.close()


def test_vertex12_group(E):
    ss = [gen.random_small(80 + i, 150 + 50 * i, 200, 2, 10, n_batches=1, n_ins=30, n_del=30,
                           membership="zipf") for i in range(3)]
    shared = E.make_config(1, 1, 1, 2000, 20000, V12, 0)
    cfgs = [E.make_config(s.n_vertices, 2000, 20000, 0, 0, V12, 0, _pairs(s)) for s in ss]
    grp = E.esc_group_create(shared, cfgs)
    try:
        E.esc_group_apply(grp, [dict(graph=i, ins_offsets=s.initial.offsets, ins_members=s.initial.members,
                                     ins_timestamps=None, del_ids=None) for i, s in enumerate(ss)])
        ogs = [OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members) for s in ss]
        batches = []
        for i, (s, og) in enumerate(zip(ss, ogs)):
            b = s.batches[0]
            dels = og.resolve_ranks(b.del_ranks)   # initial IDs are 0..n-1 on both sides
            og.apply_batch(b.inserts.offsets, b.inserts.members, None, dels)
            batches.append(dict(graph=i, ins_offsets=b.inserts.offsets, ins_members=b.inserts.members,
                                ins_timestamps=None, del_ids=np.sort(b.del_ranks).astype(np.int32)))
        E.esc_group_apply(grp, batches)
        for i, og in enumerate(ogs):
            v = [int(x) for x in E.esc_group_triads(grp, i, E.TRIAD_VERTEX, 0)]
            assert v[:2] == [int(x) for x in O.counts(og, 2)["vertex"][:2]] and v[2] == 0, i
    finally:
        E.esc_group_destroy(grp)


def test_vertex12_capacity_and_config_refusals(E):
    s = gen.random_small(73, 200, 100, 2, 6, n_batches=1, n_ins=10, n_del=5)
    init = s.initial
    caps = caps_for(s.n_vertices, 1000, 10000, 1000, 10000)
    need = int(sum(int(k) * (int(k) - 1) // 2 for k in np.diff(init.offsets)))
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    g = E.Graph(s.n_vertices, init.offsets, init.members, None, families=V12, capacity_vertex_pairs=need + 10,
                **caps)
    before = [int(x) for x in g.counts()["vertex"]]
    # a hyperedge of 40 members brings 780 pairs: beyond the capacity
    big = np.arange(40, dtype=np.int32)
    with pytest.raises(E.EscError) as ei:
        g.apply_batch(np.array([0, 40]), big, None, None)
    assert ei.value.status == 3
    assert [int(x) for x in g.counts()["vertex"]] == before
    # the graph is unchanged: a small batch afterwards is exact
    b = s.batches[0]
    dels = og.resolve_ranks(b.del_ranks)[:0]
    og.apply_batch(np.array([0, 2]), np.array([0, 1]), None, dels)
    g.apply_batch(np.array([0, 2]), np.array([0, 1], np.int32), None, None)
    _check(g, og, V12, 0, "after refusal")
    g.close()
    for fam, pairs in ((V12 | 2, 100), (V12, 0)):
        with pytest.raises(E.EscError) as ei:
            E.Graph(s.n_vertices, init.offsets, init.members, None, families=fam, capacity_vertex_pairs=pairs, **caps)
        assert ei.value.status == 1


def test_vertex12_has_no_neighbourhood_limit(E, monkeypatch):
    """A hub vertex in every hyperedge: with the neighbour-list arena shrunk
    (ESC_COUNT_LIST), every hyperedge's neighbourhood is over the counter's
    limit, which the neighbourhood families refuse; the vertex-pair family
    never builds a neighbourhood and is exact."""
    monkeypatch.setenv("ESC_COUNT_LIST", "4096")   # neighbourhoods of at most 512 entries
    nv, n = 700, 600
    E_ = [[0, 1 + i, 1 + (i * 7 + 3) % (nv - 1)] for i in range(n)]
    E_ = [sorted(set(e)) for e in E_]
    off = np.concatenate([[0], np.cumsum([len(e) for e in E_])]).astype(np.int64)
    mem = np.concatenate([np.array(e, np.int32) for e in E_])
    caps = caps_for(nv, 2000, 8000, 1000, 8000)
    og = OracleHypergraph(nv, off, mem)
    g = E.Graph(nv, off, mem, None, families=V12, capacity_vertex_pairs=4000, **caps)
    _check(g, og, V12, 0, "initial")
    ids_o = og.apply_batch(np.array([0, 3]), np.array([0, 5, 9]), None, np.arange(10))
    ids_g = g.apply_batch(np.array([0, 3]), np.array([0, 5, 9], np.int32), None, np.arange(10, dtype=np.int32))
    assert np.array_equal(ids_g, ids_o)
    _check(g, og, V12, 0, "after")
    g.close()
    with pytest.raises(E.EscError) as ei:
        E.Graph(nv, off, mem, None, families=2, **caps)
    assert ei.value.status == 4


def _csr(edges):
    off = np.zeros(len(edges) + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.array([v for e in edges for v in e], np.int32)
    return off, mem


def test_vertex12_singletons_and_one_large_hyperedge(E):
    """Runs of more than 32 single-member hyperedges (no member pairs, some
    written as a repeated member) among ordinary ones, and one hyperedge of
    800 members whose 319,600 member pairs are spread over the whole grid;
    the next batch deletes it with part of the singletons while inserting
    more of them."""
    rng = np.random.default_rng(73)
    nv = 3000
    init = gen.random_small(73, nv, 500, 2, 20, membership="zipf").initial
    og = OracleHypergraph(nv, init.offsets, init.members, init.timestamps)
    caps = caps_for(nv, 4096, 40000, 4096, 40000)
    g = E.Graph(nv, init.offsets, init.members, init.timestamps, families=V12,
                capacity_vertex_pairs=int(np.sum(np.diff(init.offsets) ** 2)) + 800000, **caps)
    _check(g, og, V12, 0, "initial")

    def ordinary(n):
        return [sorted(rng.choice(nv, size=int(rng.integers(2, 30)), replace=False).tolist()) for _ in range(n)]

    def singles(n):
        return [[int(v)] * int(rng.integers(1, 3)) for v in rng.integers(0, nv, size=n)]

    large = sorted(rng.choice(nv, size=800, replace=False).tolist())
    edges = ordinary(5) + singles(70) + [large] + singles(70) + ordinary(5)
    off, mem = _csr(edges)
    ts = np.arange(len(edges), dtype=np.int64) + 10_000
    ids_o = og.apply_batch(off, mem, ts, np.zeros(0, np.int64))
    ids_g = g.apply_batch(off, mem, ts, np.zeros(0, np.int32))
    assert np.array_equal(ids_g, ids_o)
    _check(g, og, V12, 0, "after the large insert")

    # delete the large hyperedge, 50 singletons and three ordinary ones
    dels = np.array([ids_o[75]] + list(ids_o[5:55]) + list(ids_o[-3:]), np.int64)
    edges2 = singles(40) + ordinary(2)
    off2, mem2 = _csr(edges2)
    ts2 = np.arange(len(edges2), dtype=np.int64) + 20_000
    ids_o2 = og.apply_batch(off2, mem2, ts2, dels)
    ids_g2 = g.apply_batch(off2, mem2, ts2, dels.astype(np.int32))
    assert np.array_equal(ids_g2, ids_o2)
    _check(g, og, V12, 0, "after the delete")
    g.close()

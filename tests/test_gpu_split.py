"""The work split of one hypergraph (esc_set_split) against the oracle.

Ranks are emulated by `world` independent replicas of the graph on one GPU,
each told its rank (no replica waits on another).  Every replica applies the
same batches and must return the oracle's IDs; after every batch the sum of
the replicas' counts, modulo 2^64, must equal the oracle's recount, for the
oriented counter (hyperedge + vertex families) and the earlier one (all
three families).  Local counts stay whole, and the split refuses a second
setting, a bad rank and graph launch.
"""
import numpy as np
import pytest

import gen
from harness import GpuLive, caps_for
from oracle import OracleHypergraph
from oracle import oracle as O

pytestmark = pytest.mark.gpu
M64 = 1 << 64


@pytest.fixture(scope="module")
def E():
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    return escher


def _sum_counts(graphs):
    tot = {}
    for g in graphs:
        for k, v in g.counts().items():
            acc = tot.setdefault(k, [0] * len(v))
            for i, x in enumerate(v):
                acc[i] = (acc[i] + int(x)) % M64
    return tot


@pytest.mark.parametrize("world,families", [(2, 3), (3, 3), (2, 7), (3, 7)])
def test_split_shares_sum_to_the_oracle(E, world, families):
    s = gen.random_small(33, 600, 800, 2, 30, n_batches=3, n_ins=80, n_del=80, membership="zipf", card="zipf")
    init = s.initial
    delta = int(init.timestamps[-1] // 3)
    caps = caps_for(s.n_vertices, 2000, 20000, 1000, 20000)
    og = OracleHypergraph(s.n_vertices, init.offsets, init.members, init.timestamps)
    graphs = [E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=families, delta=delta,
                      **caps) for _ in range(world)]
    for r, g in enumerate(graphs):
        g.set_split(r, world)
    want = {k: [int(x) for x in v] for k, v in O.counts(og, families, delta).items()}
    assert _sum_counts(graphs) == want, "initial"
    live = GpuLive(init.n, init.timestamps)
    for k, b in enumerate(s.batches):
        dels_o = og.resolve_ranks(b.del_ranks)
        ids_o = og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_o)
        dels_g = live.resolve(b.del_ranks).astype(np.int32)
        for g in graphs:
            ids_g = g.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_g)
            assert np.array_equal(ids_g, ids_o), f"batch {k}: IDs"
        live.apply(dels_g, ids_o, b.inserts.timestamps)
        want = {kk: [int(x) for x in v] for kk, v in O.counts(og, families, delta).items()}
        assert _sum_counts(graphs) == want, f"batch {k}"
        # every share is a part: no replica holds the whole change by itself
    ids = og.live_ids().astype(np.int32)
    for g in graphs:
        loc = g.local_triads(ids)
        for kk in want:
            assert [int(x) for x in loc[kk]] == want[kk], "local counts are whole"
    for g in graphs:
        g.close()


def test_split_refusals(E):
    s = gen.random_small(34, 100, 80, 2, 6)
    init = s.initial
    g = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=3,
                **caps_for(s.n_vertices, 200, 2000, 100, 2000))
    with pytest.raises(E.EscError) as ei:
        g.set_split(2, 2)
    assert ei.value.status == 1
    with pytest.raises(E.EscError) as ei:
        g.set_split(0, 1)
    assert ei.value.status == 1
    g.set_split(1, 2)
    assert not any(int(x) for x in g.counts()["hyperedge"])   # rank 1 starts from zero
    with pytest.raises(E.EscError) as ei:
        g.set_split(0, 2)
    assert ei.value.status == 4
    with pytest.raises(E.EscError) as ei:
        g.set_graph_launch(True)
    assert ei.value.status == 4
    g.close()
    g2 = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps, families=3,
                 **caps_for(s.n_vertices, 200, 2000, 100, 2000))
    g2.set_graph_launch(True)
    with pytest.raises(E.EscError) as ei:
        g2.set_split(0, 2)
    assert ei.value.status == 4
    g2.close()

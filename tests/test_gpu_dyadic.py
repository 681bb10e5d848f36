"""The dyadic special case: a graph held as two-member hyperedges.  On plain
edges the incident-vertex type-3 count is the triangle count (with parallel
edges, each triangle weighted by its edge multiplicities) and types 1 and 2
are zero; the CUDA path matches that closed form and the oracle after every
batch, also when inserted hyperedges of spread-out cardinality join the
graph."""
import networkx as nx
import numpy as np
import pytest

import gen
from oracle import OracleHypergraph
from oracle import oracle as O
from tests.harness import assert_counts_equal, assert_store_equal, caps_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    return escher


def _triangles(og):
    """Triangles of the graph, each weighted by the product of its three
    edge multiplicities (a vertex triad is counted once per choice of the
    hyperedges that join its pairs); on a simple graph, the triangle count."""
    mult = {}
    for h in og.live_ids():
        e = og.edge(int(h))
        assert e.size == 2
        key = (int(min(e)), int(max(e)))
        mult[key] = mult.get(key, 0) + 1
    G = nx.Graph()
    G.add_edges_from(mult)
    total = 0
    for a, b, c in (t for t in nx.enumerate_all_cliques(G) if len(t) == 3):
        total += mult[tuple(sorted((a, b)))] * mult[tuple(sorted((b, c)))] * mult[tuple(sorted((a, c)))]
    return total


@pytest.mark.parametrize("families", [2, 7])
def test_dyadic_graph_triangles(E, families):
    nv = 120
    init = gen.dyadic_graph(7, nv, 500)
    og = OracleHypergraph(nv, init.offsets, init.members, init.timestamps)
    delta = int(init.timestamps[-1] // 2)
    g = E.Graph(nv, init.offsets, init.members, init.timestamps, families=families, delta=delta,
                **caps_for(nv, 2000, 4000, 500, 2000))
    rng = np.random.default_rng(1)
    batches = gen.spread_inserts(8, nv, 4, 60, 2.0, 0.0, ts_start=int(init.timestamps[-1]))
    for k, b in enumerate([None] + batches):
        if b is not None:
            live = og.live_ids()
            dels = np.sort(rng.choice(live, size=40, replace=False))
            want = og.apply_batch(b.offsets, b.members, b.timestamps, dels)
            got = g.apply_batch(b.offsets, b.members, b.timestamps, dels.astype(np.int32))
            assert np.array_equal(got, want)
        v = g.triads(E.TRIAD_VERTEX)
        assert int(v[0]) == 0 and int(v[1]) == 0, f"step {k}: {v.tolist()}"
        assert int(v[2]) == _triangles(og), f"step {k}"
        assert_counts_equal(g.counts(), O.counts(og, families, delta), f"step {k}")
    assert_store_equal(g, og)
    g.close()


def test_spread_cardinalities_on_a_dyadic_graph(E):
    nv = 150
    init = gen.dyadic_graph(9, nv, 400)
    og = OracleHypergraph(nv, init.offsets, init.members, init.timestamps)
    g = E.Graph(nv, init.offsets, init.members, init.timestamps, families=2,
                **caps_for(nv, 2000, 20000, 500, 8000))
    rng = np.random.default_rng(2)
    for k, sd in enumerate((1.0, 4.0, 16.0)):
        b = gen.spread_inserts(10 + k, nv, 1, 50, 4.0, sd, kmax=nv)[0]
        dels = np.sort(rng.choice(og.live_ids(), size=30, replace=False))
        want = og.apply_batch(b.offsets, b.members, b.timestamps, dels)
        got = g.apply_batch(b.offsets, b.members, b.timestamps, dels.astype(np.int32))
        assert np.array_equal(got, want)
        assert_counts_equal(g.counts(), O.counts(og, 2, 0), f"std {sd}")
    assert_store_equal(g, og)
    g.close()

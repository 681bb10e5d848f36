"""Parity at the benchmark's full size, in the launch configuration the
benchmark times (the uniform 1M-vertex, 2M-hyperedge graph, batches of
5e4 inserts + 5e4 deletes, hyperedge and incident-vertex families, counter
shape picked by the autotuner on a sample of one batch's size).

After two batches: the assigned IDs and the whole store equal the oracle's;
the incrementally kept counts equal a full recount of every live hyperedge
(a property that holds at any size); and the triads holding a few sampled
hyperedges, counted by the oracle's own enumeration on its own copy of the
graph, equal the library's local counts for the same hyperedges."""
import numpy as np
import pytest

import gen
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
    for k, b in enumerate(s.batches):
        dels_o = og.resolve_ranks(b.del_ranks)
        want = og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_o)
        got = g.apply_batch(todev(b.inserts.offsets, np.int64), todev(b.inserts.members, np.int32),
                            todev(b.inserts.timestamps, np.int64), todev(np.sort(b.del_ranks), np.int32))
        assert np.array_equal(got, want), f"batch {k}: assigned IDs differ"
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
    g.close()

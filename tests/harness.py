"""Test-side bookkeeping shared by the GPU parity tests: run the same seeded
stream through the oracle and through the CUDA library and compare after
every batch.  Each side resolves delete ranks and expirations against its own
live set; nothing the CUDA side returns is fed to the oracle."""
from __future__ import annotations

import numpy as np

from oracle import OracleHypergraph
from oracle import oracle as O


class GpuLive:
    """Live IDs and timestamps of the CUDA side, kept from the IDs it returns."""

    def __init__(self, n0: int, ts0=None):
        self.ts = {i: (int(ts0[i]) if ts0 is not None else 0) for i in range(n0)}

    def resolve(self, ranks):
        live = np.array(sorted(self.ts), dtype=np.int64)
        return live[np.asarray(ranks, dtype=np.int64)] if len(ranks) else np.zeros(0, np.int64)

    def expired(self, t_cut):
        return np.array(sorted(i for i, t in self.ts.items() if t < t_cut), dtype=np.int64)

    def apply(self, dels, ids, ts):
        for d in dels:
            del self.ts[int(d)]
        for i, t in zip(ids, ts):
            self.ts[int(i)] = int(t)


class LiveIds:
    """Live IDs of the CUDA side as a sorted array, kept from the IDs it
    returns (a client's copy; for large graphs where a dict is slow)."""

    def __init__(self, ids):
        self.ids = np.sort(np.asarray(ids, dtype=np.int64))

    def resolve(self, ranks):
        return self.ids[np.asarray(ranks, dtype=np.int64)] if len(ranks) else np.zeros(0, np.int64)

    def apply(self, dels, new_ids):
        keep = np.ones(self.ids.size, bool)
        keep[np.searchsorted(self.ids, np.asarray(dels, dtype=np.int64))] = False
        self.ids = np.sort(np.concatenate([self.ids[keep], np.asarray(new_ids, dtype=np.int64)]))


def caps_for(n_vertices, n_edges, nnz, batch_hyperedges, batch_incidences, slack=2.0):
    return dict(capacity_hyperedges=int(max(64, n_edges * slack)),
                capacity_incidences=int(max(1024, nnz * slack)),
                max_batch_hyperedges=int(max(64, batch_hyperedges)),
                max_batch_incidences=int(max(1024, batch_incidences)))


def assert_counts_equal(got: dict, want: dict, where=""):
    for k in want:
        g, w = np.asarray(got[k], np.uint64), np.asarray(want[k], np.uint64)
        assert np.array_equal(g, w), f"{where} {k}: gpu {g.tolist()} oracle {w.tolist()}"


def assert_store_equal(graph, og: OracleHypergraph):
    ex = graph.export()
    off, mem, ts, ids = og.csr()
    assert np.array_equal(ex["ids"], ids), "live IDs differ"
    assert np.array_equal(ex["offsets"], off), "hyperedge sizes differ"
    assert np.array_equal(ex["members"], mem), "h2v members differ"
    assert np.array_equal(ex["timestamps"], ts), "timestamps differ"
    v2h = og.v2h()
    voff = ex["v_offsets"]
    for v in range(og.n_vertices):
        got = ex["v_members"][voff[v]:voff[v + 1]]
        assert np.array_equal(got, v2h[v]), f"v2h of vertex {v} differs"


def run_stream(E, stream, families, delta, *, check_store=True, method="wedge", device=None,
               caps=None, local_check=False):
    """Create both sides from the stream's initial hypergraph, apply every
    batch, compare counts (and optionally the store) after each step."""
    init = stream.initial
    if caps is None:
        bh = max((b.inserts.n + len(b.del_ranks) for b in stream.batches), default=64)
        bi = max((b.inserts.nnz for b in stream.batches), default=1024)
        caps = caps_for(stream.n_vertices, init.n + sum(b.inserts.n for b in stream.batches),
                        init.nnz + sum(b.inserts.nnz for b in stream.batches), max(bh, init.n), max(bi, init.nnz))
    og = OracleHypergraph(stream.n_vertices, init.offsets, init.members, init.timestamps)
    conv = (lambda a: a) if device is None else (lambda a: _to_dev(a, device))
    g = E.Graph(stream.n_vertices, conv(init.offsets), conv(init.members), conv(init.timestamps),
                families=families, delta=delta, **caps)
    live = GpuLive(init.n, init.timestamps)
    assert_counts_equal(g.counts(), O.counts(og, families, delta, method), "initial")
    if check_store:
        assert_store_equal(g, og)
    for bi_, b in enumerate(stream.batches):
        dels_o = og.resolve_ranks(b.del_ranks)
        dels_g = live.resolve(b.del_ranks)
        ids_o = og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels_o)
        ids_g = g.apply_batch(conv(b.inserts.offsets), conv(b.inserts.members), conv(b.inserts.timestamps),
                              conv(dels_g.astype(np.int32)))
        assert np.array_equal(ids_g, ids_o), f"batch {bi_}: assigned IDs differ"
        live.apply(dels_g, ids_g, b.inserts.timestamps)
        assert_counts_equal(g.counts(), O.counts(og, families, delta, method), f"batch {bi_}")
        if check_store:
            assert_store_equal(g, og)
    if local_check:
        ids = og.live_ids().astype(np.int32)
        full = g.local_triads(ids)
        assert_counts_equal(full, g.counts(), "full recount")
    return g, og


def _to_dev(a, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)

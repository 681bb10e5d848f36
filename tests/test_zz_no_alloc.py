"""The allocation-free entry point (esc_count_static_noalloc) against the
allocating one (esc_create + esc_triads).

esc_count_static_noalloc serves callers that cannot allocate device memory
(code running under CUDA-graph stream capture, code held to a memory budget
by its own allocator): it keeps its temporary buffers in a fixed device array
inside the library.  Two calls in a row on different hypergraphs must each
give exactly the counts that a graph built with esc_create reports, so
nothing left in the shared array from one call leaks into the next.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

ALL = 7


def _sorted_csr(s):
    off = s.initial.offsets
    mem = s.initial.members.copy()
    for i in range(s.initial.n):
        mem[off[i]:off[i + 1]] = np.sort(mem[off[i]:off[i + 1]])
    return off, mem, s.initial.timestamps


@pytest.fixture(scope="module")
def E():
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    return escher


def test_noalloc_matches_allocating_entry_point_twice(E):
    import torch
    dev = torch.device("cuda:0")
    cases = [gen.random_small(41, 400, 350, 1, 9, membership="zipf"),
             gen.random_small(42, 900, 600, 2, 40, card="zipf")]
    for s in cases:
        off, mem, ts = _sorted_csr(s)
        delta = int(ts[-1] // 3)
        g = E.Graph(s.n_vertices, off, mem, ts, capacity_hyperedges=2 * s.initial.n,
                    capacity_incidences=2 * s.initial.nnz, max_batch_hyperedges=s.initial.n,
                    max_batch_incidences=s.initial.nnz, families=ALL, delta=delta)
        want = g.counts()
        g.close()
        out = torch.full((129,), -1, dtype=torch.int64, device=dev)
        E.esc_count_static_noalloc(s.n_vertices, torch.from_numpy(off).to(dev), torch.from_numpy(mem).to(dev),
                                   torch.from_numpy(ts).to(dev), ALL, delta, out)
        got = out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got[0:30], want["hyperedge"])
        assert np.array_equal(got[30:33], want["vertex"])
        assert np.array_equal(got[33:129], want["temporal"])


def test_noalloc_rejects_sizes_beyond_its_limit(E):
    import torch
    dev = torch.device("cuda:0")
    n = (1 << 18) + 1
    off = torch.arange(n + 1, dtype=torch.int64, device=dev)
    mem = torch.zeros(n, dtype=torch.int32, device=dev)
    out = torch.zeros(129, dtype=torch.int64, device=dev)
    with pytest.raises(E.EscError) as ei:
        E.esc_count_static_noalloc(10, off, mem, None, 1, 0, out)
    assert ei.value.status == 4

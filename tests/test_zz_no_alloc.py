"""The allocation-free entry point (esc_count_static_noalloc) against the
oracle and against the allocating one (esc_create + esc_triads).

esc_count_static_noalloc serves callers that cannot allocate device memory
(code held to a memory budget by its own allocator, or code whose allocator
must not be re-entered): it keeps its temporary buffers in a fixed device
array inside the library.  Two calls in a row on different hypergraphs must
each give exactly the counts of the oracle and of a graph built with
esc_create, so nothing left in the shared array from one call leaks into the
next.  Inputs it must refuse -- a hyperedge whose members' degrees sum past
its limit, a repeated member, offsets that go backwards -- give an error
status and all-zero counts, and the next valid call is exact again.
"""
import numpy as np
import pytest

import gen
from oracle import OracleHypergraph
from oracle import oracle as O

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


def _noalloc(E, nv, off, mem, ts, fam, delta):
    import torch
    dev = torch.device("cuda:0")
    out = torch.full((129,), -1, dtype=torch.int64, device=dev)
    E.esc_count_static_noalloc(nv, torch.from_numpy(off).to(dev), torch.from_numpy(mem).to(dev),
                               None if ts is None else torch.from_numpy(ts).to(dev), fam, delta, out)
    return out.cpu().numpy().view(np.uint64)


def _status_and_out(E, nv, off, mem, fam=1):
    import torch
    dev = torch.device("cuda:0")
    out = torch.full((129,), -1, dtype=torch.int64, device=dev)
    try:
        E.esc_count_static_noalloc(nv, torch.from_numpy(off).to(dev), torch.from_numpy(mem).to(dev),
                                   None, fam, 0, out)
        status = 0
    except E.EscError as e:
        status = e.status
    return status, out.cpu().numpy().view(np.uint64)


CASES = [(41, 400, 350, 1, 9, "zipf", "uniform"), (42, 900, 600, 2, 40, "uniform", "zipf")]


def _case(i):
    seed, nv, ne, kmin, kmax, memb, card = CASES[i]
    return gen.random_small(seed, nv, ne, kmin, kmax, membership=memb, card=card)


def _check_exact(E, s):
    off, mem, ts = _sorted_csr(s)
    delta = int(ts[-1] // 3)
    got = _noalloc(E, s.n_vertices, off, mem, ts, ALL, delta)
    og = OracleHypergraph(s.n_vertices, off, mem, ts)
    want = O.counts(og, ALL, delta)
    assert np.array_equal(got[0:30], want["hyperedge"])
    assert np.array_equal(got[30:33], want["vertex"])
    assert np.array_equal(got[33:129], want["temporal"])
    return got, off, mem, ts, delta


def test_noalloc_matches_oracle_and_allocating_entry_point_twice(E):
    for i in range(len(CASES)):
        s = _case(i)
        got, off, mem, ts, delta = _check_exact(E, s)
        g = E.Graph(s.n_vertices, off, mem, ts, capacity_hyperedges=2 * s.initial.n,
                    capacity_incidences=2 * s.initial.nnz, max_batch_hyperedges=s.initial.n,
                    max_batch_incidences=s.initial.nnz, families=ALL, delta=delta)
        want = g.counts()
        g.close()
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


def test_noalloc_degree_sum_limit_then_exact(E):
    # 70,000 copies of {0, 1}: every hyperedge's members have degrees summing
    # to 140,000, past the per-hyperedge limit of 65,536 (within every other
    # limit); the device reports it and the counts read zero
    n = 70_000
    off = np.arange(n + 1, dtype=np.int64) * 2
    mem = np.tile(np.array([0, 1], np.int32), n)
    status, out = _status_and_out(E, 4, off, mem)
    assert status == 4
    assert not out.any()
    _check_exact(E, _case(0))


def test_noalloc_malformed_hypergraphs_then_exact(E):
    # a repeated member
    status, out = _status_and_out(E, 10, np.array([0, 3, 5], np.int64), np.array([1, 2, 2, 4, 5], np.int32))
    assert status == 1 and not out.any()
    _check_exact(E, _case(1))
    # offsets that go backwards; every range they name stays inside the
    # four members, so only the order is wrong
    status, out = _status_and_out(E, 10, np.array([0, 3, 1, 4], np.int64), np.array([1, 2, 3, 4], np.int32))
    assert status == 1 and not out.any()
    _check_exact(E, _case(0))
    # an out-of-range vertex
    status, out = _status_and_out(E, 10, np.array([0, 2], np.int64), np.array([3, 10], np.int32))
    assert status == 1 and not out.any()
    _check_exact(E, _case(1))


def test_noalloc_wrapper_refuses_bad_tensors(E):
    import torch
    dev = torch.device("cuda:0")
    off = torch.tensor([0, 2], dtype=torch.int64, device=dev)
    mem = torch.tensor([0, 1], dtype=torch.int32, device=dev)
    with pytest.raises(E.EscError) as ei:   # too short an output
        E.esc_count_static_noalloc(4, off, mem, None, 1, 0, torch.zeros(128, dtype=torch.int64, device=dev))
    assert ei.value.status == 1
    with pytest.raises(E.EscError) as ei:   # members of the wrong type
        E.esc_count_static_noalloc(4, off, mem.to(torch.int64), None, 1, 0,
                                   torch.zeros(129, dtype=torch.int64, device=dev))
    assert ei.value.status == 1

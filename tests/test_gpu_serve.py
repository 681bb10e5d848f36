"""The serving loop (esc_server_*) over a group of resident graphs.

Requests for several graphs are submitted in a burst, so that the worker
batches them; each graph's IDs and counts must equal those of the oracle,
which applies the same graph's requests one by one.  Also: the
one-request-per-call policy, admission (a full queue refuses a request and
keeps nothing of it) and a faulty request failing alone.
"""
import numpy as np
import pytest

import gen
from oracle import OracleHypergraph
from oracle import oracle as O

pytestmark = pytest.mark.gpu

ALL = 7
DELTA = 1 << 50


@pytest.fixture(scope="module")
def E():
    from paper_2512_21009_gb300 import build as b
    b.build()
    from paper_2512_21009_gb300 import escher
    escher.load()
    return escher


def _group(E, streams, max_bh=4000, max_bi=40000):
    shared = E.make_config(1, 1, 1, max_bh, max_bi, ALL, DELTA)
    cfgs = [E.make_config(s.n_vertices, 1200, 12000, 0, 0, ALL, DELTA) for s in streams]
    grp = E.esc_group_create(shared, cfgs)
    E.esc_group_apply(grp, [dict(graph=i, ins_offsets=s.initial.offsets, ins_members=s.initial.members,
                                 ins_timestamps=s.initial.timestamps, del_ids=None)
                            for i, s in enumerate(streams)])
    ogs = [OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
           for s in streams]
    return grp, ogs


def _request(rng, og, n_ins, n_del, t0):
    """A random request against the oracle's live set: n_ins hyperedges of
    2..6 uniform members and n_del uniform live IDs."""
    live = og.live_ids()
    dels = np.sort(rng.choice(live, size=min(n_del, len(live)), replace=False))
    edges = [np.sort(rng.choice(og.n_vertices, size=int(rng.integers(2, 7)), replace=False)) for _ in range(n_ins)]
    off = np.zeros(n_ins + 1, np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    mem = np.concatenate(edges).astype(np.int32) if n_ins else np.zeros(0, np.int32)
    ts = t0 + np.arange(n_ins, dtype=np.int64)
    return off, mem, ts, dels


def _streams():
    return [gen.random_small(60 + i, 120 + 25 * i, 90 + 30 * i, 2, 6) for i in range(6)]


@pytest.mark.parametrize("per_call", [0, 1])
def test_server_matches_oracle_per_graph(E, per_call):
    streams = _streams()
    grp, ogs = _group(E, streams)
    srv = E.esc_server_create(grp, max_pending_updates=1 << 20, max_batches_per_call=per_call)
    try:
        rng = np.random.default_rng(5 + per_call)
        sub, t0 = [], 10_000
        for r in range(60):
            g = int(rng.integers(0, len(streams)))
            off, mem, ts, dels = _request(rng, ogs[g], int(rng.integers(0, 12)), int(rng.integers(1, 12)), t0)
            t0 += 100
            want_ids = ogs[g].apply_batch(off, mem, ts, dels)
            out = np.full(max(len(off) - 1, 1), -1, np.int32)
            t = E.esc_server_submit(srv, g, off, mem, ts, dels.astype(np.int32), out)
            assert t >= 0
            sub.append((t, out, want_ids))
        E.esc_server_drain(srv)
        batched = 0
        for t, out, want_ids in sub:
            info = E.esc_server_wait(srv, t)
            assert info["status"] == 0
            assert info["t_arrival_ns"] <= info["t_start_ns"] <= info["t_done_ns"]
            assert np.array_equal(out[:len(want_ids)], want_ids)
            batched = max(batched, info["call_batches"])
        if per_call == 1:
            assert batched == 1
        st = E.esc_server_get_stats(srv)
        assert st["completed"] == 60 and st["failed"] == 0 and st["pending_updates"] == 0
        assert st["calls"] <= 60
        for i, og in enumerate(ogs):
            want = O.counts(og, ALL, DELTA)
            assert np.array_equal(E.esc_server_triads(srv, i, 0), want["hyperedge"]), i
            assert np.array_equal(E.esc_server_triads(srv, i, 1), want["vertex"]), i
            assert np.array_equal(E.esc_server_triads(srv, i, 2, DELTA), want["temporal"]), i
    finally:
        E.esc_server_destroy(srv)
        E.esc_group_destroy(grp)


def test_server_admission_and_failure_isolation(E):
    streams = _streams()
    grp, ogs = _group(E, streams)
    # room for one small request at a time
    srv = E.esc_server_create(grp, max_pending_updates=8, max_batches_per_call=0)
    try:
        rng = np.random.default_rng(11)
        accepted, refused, t0 = 0, 0, 50_000
        for r in range(20):
            # two requests back to back: the second usually finds the queue full
            tickets = []
            for g in (int(rng.integers(0, 3)), int(rng.integers(3, 6))):
                off, mem, ts, dels = _request(rng, ogs[g], 3, 3, t0)
                t0 += 100
                t = E.esc_server_submit(srv, g, off, mem, ts, dels.astype(np.int32))
                if t < 0:
                    refused += 1
                    continue
                accepted += 1
                ogs[g].apply_batch(off, mem, ts, dels)
                tickets.append(t)
            for t in tickets:
                assert E.esc_server_wait(srv, t)["status"] == 0
        assert accepted > 0
        st = E.esc_server_get_stats(srv)
        assert st["rejected"] == refused and st["completed"] == accepted
        # a request too large for the queue is refused outright
        off, mem, ts, dels = _request(rng, ogs[0], 5, 5, t0)
        assert E.esc_server_submit(srv, 0, off, mem, ts, dels.astype(np.int32)) == -1
        E.esc_server_destroy(srv)
        # a faulty request (delete of a dead ID) fails alone, the rest apply
        srv = E.esc_server_create(grp, max_pending_updates=1 << 20, max_batches_per_call=0)
        tickets = []
        for g in range(len(streams)):
            off, mem, ts, dels = _request(rng, ogs[g], 4, 4, t0)
            if g == 2:
                dels = np.array([1100], np.int64)  # inside the ID range, never live
                tickets.append((g, E.esc_server_submit(srv, g, off, mem, ts, dels.astype(np.int32)), False))
                continue
            ogs[g].apply_batch(off, mem, ts, dels)
            tickets.append((g, E.esc_server_submit(srv, g, off, mem, ts, dels.astype(np.int32)), True))
        E.esc_server_drain(srv)
        for g, t, ok in tickets:
            info = E.esc_server_wait(srv, t)
            assert (info["status"] == 0) == ok, (g, info)
        assert E.esc_server_get_stats(srv)["failed"] == 1
        for i, og in enumerate(ogs):
            want = O.counts(og, ALL, DELTA)
            assert np.array_equal(E.esc_server_triads(srv, i, 0), want["hyperedge"]), i
            assert np.array_equal(E.esc_server_triads(srv, i, 2, DELTA), want["temporal"]), i
    finally:
        E.esc_server_destroy(srv)
        E.esc_group_destroy(grp)


def test_group_bytes_covers_the_allocation(E):
    import torch
    streams = _streams()
    shared = E.make_config(1, 1, 1, 4000, 40000, ALL, DELTA)
    cfgs = [E.make_config(s.n_vertices, 1200, 12000, 0, 0, ALL, DELTA) for s in streams]
    est = E.esc_group_bytes(shared, cfgs)
    E.esc_group_destroy(E.esc_group_create(shared, cfgs))  # load the kernels first
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    grp = E.esc_group_create(shared, cfgs)
    try:
        torch.cuda.synchronize()
        used = free0 - torch.cuda.mem_get_info()[0]
        # the driver rounds each of the ~70 allocations up to its page size
        slack = 160 << 20
        assert used - slack <= est <= used + slack, (est, used)
    finally:
        E.esc_group_destroy(grp)


def test_groups_added_while_serving_overlap_and_match_alone(E):
    """A server starts with one group and takes two more while it runs; the
    groups live on their own streams, so their workers' calls overlap on the
    device.  Requests for all of them are interleaved from this thread.  Each
    graph's IDs and counts must equal those of the oracle applying that
    graph's requests alone, and the call records must show calls of
    different groups overlapping in time."""
    import torch
    streams3 = [_streams()[2 * k:2 * k + 2] for k in range(3)]
    cuda_streams = [torch.cuda.Stream() for _ in range(3)]
    shared = E.make_config(1, 1, 1, 4000, 40000, ALL, DELTA)
    groups, ogs, firsts = [], [], []

    def make(k):
        sts = streams3[k]
        cfgs = [E.make_config(s.n_vertices, 1200, 12000, 0, 0, ALL, DELTA) for s in sts]
        assert E.esc_group_fits(shared, cfgs, 0)
        grp = E.esc_group_create(shared, cfgs, stream=cuda_streams[k])
        E.esc_group_apply(grp, [dict(graph=i, ins_offsets=s.initial.offsets, ins_members=s.initial.members,
                                     ins_timestamps=s.initial.timestamps, del_ids=None) for i, s in enumerate(sts)])
        groups.append(grp)
        ogs.extend(OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
                   for s in sts)
        return grp

    srv = E.esc_server_create(make(0), max_pending_updates=1 << 22, max_batches_per_call=0)
    firsts.append(0)
    try:
        rng = np.random.default_rng(17)
        sub, t0 = [], 90_000
        for phase in range(3):
            if phase > 0:
                firsts.append(E.esc_server_add_group(srv, make(phase)))
                assert firsts[-1] == 2 * phase
            # the phase's requests are prepared (and applied to the oracle)
            # first, then submitted in one burst
            reqs = []
            for r in range(60):
                g = int(rng.integers(0, 2 * (phase + 1)))
                off, mem, ts, dels = _request(rng, ogs[g], int(rng.integers(10, 30)), int(rng.integers(10, 30)), t0)
                t0 += 100
                reqs.append((g, off, mem, ts, dels, ogs[g].apply_batch(off, mem, ts, dels)))
            for g, off, mem, ts, dels, want_ids in reqs:
                out = np.full(max(len(off) - 1, 1), -1, np.int32)
                t = E.esc_server_submit(srv, g, off, mem, ts, dels.astype(np.int32), out)
                assert t >= 0
                sub.append((g, t, out, want_ids))
        E.esc_server_drain(srv)
        spans = []
        for g, t, out, want_ids in sub:
            info = E.esc_server_wait(srv, t)
            assert info["status"] == 0
            assert np.array_equal(out[:len(want_ids)], want_ids), g
            spans.append((g // 2, info["t_start_ns"], info["t_done_ns"]))
        for i, og in enumerate(ogs):
            want = O.counts(og, ALL, DELTA)
            assert np.array_equal(E.esc_server_triads(srv, i, 0), want["hyperedge"]), i
            assert np.array_equal(E.esc_server_triads(srv, i, 1), want["vertex"]), i
            assert np.array_equal(E.esc_server_triads(srv, i, 2, DELTA), want["temporal"]), i
        # some call of one group ran while a call of another group ran
        overlap = any(a[0] != b[0] and a[1] < b[2] and b[1] < a[2] for a in spans for b in spans)
        assert overlap
    finally:
        E.esc_server_destroy(srv)
        for grp in groups:
            E.esc_group_destroy(grp)
    with pytest.raises(E.EscError):
        s2 = E.esc_server_create(make(0), max_pending_updates=16)
        try:
            E.esc_server_add_group(s2, groups[-1])   # already served by s2
        finally:
            E.esc_server_destroy(s2)
            E.esc_group_destroy(groups[-1])

"""The single-graph work split on CPU ranks (gloo), checked with the oracle.

With a work split every rank holds the same hypergraph and counts only its
share of a batch's changed hyperedges: per side, a contiguous range of them
in ID order (the library cuts the ranges by neighbourhood size).  Alg. 3's
change of the counts is a sum over the changed hyperedges, each triad (and
each incident-vertex witness assignment) counted at its changed member of
smallest ID; so the share of a range [c_a, c_b) of the sorted changed IDs is
containing(c_1..c_b-1) - containing(c_1..c_a-1), and the shares of all ranks,
summed by one all-reduce, are the whole change.  Here each rank takes its
range by the same rule as the library (equal parts of the total of the
neighbourhood sizes plus one), computes its share with the oracle, and the
all-reduce of the int64 images of the uint64 shares (exact modulo 2^64) must
equal the oracle's unsplit change, for 2 and 3 ranks.
"""
import json
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def split_range(costs, rank, world):
    """Contiguous range [a, b) of rank: items whose prefix of (cost + 1) falls
    in the rank's equal part of the total."""
    pre = np.concatenate([[0], np.cumsum(np.asarray(costs, np.int64) + 1)])
    total = int(pre[-1])
    owner = (pre[:-1] * world) // total
    idx = np.flatnonzero(owner == rank)
    return (int(idx[0]), int(idx[-1]) + 1) if idx.size else (0, 0)


def _side_terms(off, mem, ids, changed):
    """Oracle count of the triads / witness assignments holding >= 1 of the
    given changed IDs (positions looked up in the CSR), both families."""
    from oracle import oracle as O
    pos = np.searchsorted(ids, np.sort(changed))
    h, _ = O.count_containing(off, mem, None, ids, 0, O.FAM_HYPEREDGE, pos)
    v = O.count_vertex_containing(off, mem, pos)
    return [int(x) for x in h] + [int(x) for x in v]


def _share(off, mem, ids, changed, a, b):
    """Share of the changed IDs [a, b) (sorted order): prefix telescoping."""
    c = np.sort(np.asarray(changed, np.int64))
    hi = _side_terms(off, mem, ids, c[:b]) if b > 0 else [0] * 33
    lo = _side_terms(off, mem, ids, c[:a]) if a > 0 else [0] * 33
    return [(x - y) % (1 << 64) for x, y in zip(hi, lo)]


def _costs(off, mem, ids, changed):
    deg = np.bincount(mem, minlength=int(mem.max()) + 1 if mem.size else 1)
    pos = np.searchsorted(ids, np.sort(changed))
    return [int(deg[mem[off[p]:off[p + 1]]].sum()) for p in pos]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import gen
    from oracle import OracleHypergraph
    dist.init_process_group("gloo")
    try:
        s = gen.random_small(61, 400, 500, 2, 12, n_batches=1, n_ins=40, n_del=40, membership="zipf", card="zipf")
        og = OracleHypergraph(s.n_vertices, s.initial.offsets, s.initial.members, s.initial.timestamps)
        off0, mem0, _, ids0 = og.csr()
        b = s.batches[0]
        dels = og.resolve_ranks(b.del_ranks)
        new = og.apply_batch(b.inserts.offsets, b.inserts.members, b.inserts.timestamps, dels)
        off1, mem1, _, ids1 = og.csr()
        ranges = {}
        share = [0] * 33
        for side, (off, mem, ids, ch) in enumerate([(off0, mem0, ids0, dels), (off1, mem1, ids1, new)]):
            a, bb = split_range(_costs(off, mem, ids, ch), rank, ws)
            ranges[side] = (a, bb)
            part = _share(off, mem, ids, ch, a, bb)
            sign = -1 if side == 0 else 1
            share = [(x + sign * y) % (1 << 64) for x, y in zip(share, part)]
        t = torch.tensor(np.array(share, dtype=np.uint64).view(np.int64))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total = [int(x) % (1 << 64) for x in t.numpy().view(np.uint64)]
        every = [None] * ws
        dist.all_gather_object(every, ranges)
        out = dict(rank=rank, total=total, ranges=every)
        if rank == 0:
            whole_d = _side_terms(off0, mem0, ids0, dels)
            whole_i = _side_terms(off1, mem1, ids1, new)
            out["whole"] = [(i - d) % (1 << 64) for d, i in zip(whole_d, whole_i)]
            out["n"] = [len(dels), len(new)]
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(out, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_shares_sum_to_the_whole_change(tmp_path, world):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    whole = res[0]["whole"]
    assert any(whole)
    for x in res:
        assert x["total"] == whole
    # the ranges of the ranks tile each side exactly once
    for side in ("0", "1"):
        rs = sorted(tuple(x[side]) for x in res[0]["ranges"])
        nonempty = [r for r in rs if r[1] > r[0]]
        assert nonempty[0][0] == 0 and nonempty[-1][1] == res[0]["n"][int(side)]
        assert all(p[1] == q[0] for p, q in zip(nonempty, nonempty[1:]))

"""Host logic of the multi-process bench on CPU: two gloo ranks.

Under torchrun every rank works on its own replica (one hypergraph) or on its
own share of independent graphs; the whole-job figures are the slowest
rank's time and the sum of every rank's units, and graphs are split so that
each is handled by exactly one rank.
"""
import json
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    r, w, local, dist = bench.dist_init("gloo")
    try:
        bench.barrier(dist)
        t_max, units = bench.combine(dist, None, elapsed_s=1.0 + r, units=10.0 * (r + 1))
        mine = bench.shard(11, r, w)
        every = [None] * w
        dist.all_gather_object(every, mine)
        with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
            json.dump(dict(rank=r, ws=w, local=local, t_max=t_max, units=units, shards=every), f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, x in enumerate(res):
        assert x["rank"] == r and x["ws"] == 2 and x["local"] == r
        assert x["t_max"] == 2.0          # slowest rank
        assert x["units"] == 30.0         # 10 + 20
    shards = res[0]["shards"]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(11))        # every graph exactly once
    assert all(len(s) in (5, 6) for s in shards)


def test_single_process_needs_no_group():
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE",) if k in os.environ}
    try:
        assert bench.dist_init() == (0, 1, 0, None)
        assert bench.combine(None, None, 3.0, 7.0) == (3.0, 7.0)
        assert bench.shard(4, 0, 1) == [0, 1, 2, 3]
    finally:
        os.environ.update(env)

"""Benchmark: hyperedge updates per second with an exact triad-count refresh,
plus p50/p99 batch latency.

A step is one batch of the stream applied through esc_apply_batch: 1e5
updates (5e4 inserts + 5e4 deletes of uniformly chosen live hyperedges),
after which the hyperedge-based (30 classes) and incident-vertex (types 1-3)
counts are exact and readable.  Default workload: 1M vertices, 2M
hyperedges, cardinality Zipf(2.0) truncated to [2, 1000], uniform vertex
membership (the large configuration with uniform membership: with Zipf(1.1)
popularity one vertex sits in ~73% of the hyperedges and an exact recount of
the triads around it is ~1e17 classifications per batch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large_uniform|tiny|batched|temporal|serving|horizontal|sweep]
                  [--sweep batch|delete|card|size|spread] [--scale S]

Under torchrun (N > 1) every rank runs its own replica on its own GPU (weak
scaling; the single-graph path has no exchange step).  Rank 0 prints one
JSON line.  ``--impl reference`` times the CPU oracle on a bounded sample of
the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "hyperedge updates/s with exact triad-count refresh; p50/p99 batch latency"
UNIT = "updates/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(backend=None):
    """Rank, world size, local rank and the process group module (None when
    run alone).  One process per GPU under torchrun: NCCL; gloo on CPU."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend=backend)
    return dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0")), dist


def barrier(dist, device=None):
    if dist is not None:
        import torch
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def allreduce_max(dist, x: float, device) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(dist, x: float, device) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def combine(dist, device, elapsed_s: float, units: float):
    """Whole-job figures: the slowest rank's time and every rank's units
    (weak scaling: each rank works on its own replica or its own graphs)."""
    return allreduce_max(dist, elapsed_s, device), allreduce_sum(dist, units, device)


def shard(n: int, rank: int, ws: int):
    """Indices of the independent units (graphs) that rank handles."""
    return list(range(rank, n, ws))


def make_stream(args, rank):
    # warm-up batches, the timed device-resident batches, then as many batches
    # again for the end-to-end run with host buffers
    nb = args.warmup + 2 * args.steps
    if args.workload == "tiny":
        s = gen.random_small(args.seed + rank, 2000, 1000, 2, 8, n_batches=nb, n_ins=50, n_del=50)
        fam = 3
    else:
        s = gen.large(seed=args.seed + rank, membership="uniform", scale=args.scale, n_batches=nb,
                      batch_updates=args.batch)
        fam = 3
    return s, fam


class _LiveRule:
    """Client copy of one graph's live IDs under the library's ID rule
    (deletes first; the j-th insert takes the j-th smallest free ID below the
    high-water mark, then fresh IDs upward).  A stream's delete ranks resolve
    to IDs through it, and the IDs the library will return are known before a
    batch is staged; the run checks them afterwards."""

    def __init__(self, n0: int):
        self.live = np.arange(n0, dtype=np.int64)
        self.hw = n0

    def step(self, ranks, n_ins):
        dels = self.live[np.sort(np.asarray(ranks, dtype=np.int64))]
        keep = np.ones(self.live.size, bool)
        keep[np.searchsorted(self.live, dels)] = False
        live = self.live[keep]
        free = np.ones(self.hw, bool)
        free[live] = False
        free = np.flatnonzero(free)
        take = min(n_ins, free.size)
        ids = np.concatenate([free[:take], np.arange(self.hw, self.hw + n_ins - take)])
        self.hw += n_ins - take
        self.live = np.sort(np.concatenate([live, ids]))
        return dels, ids


def workload_desc(args, s):
    if args.workload == "tiny":
        return "tiny: 2,000 vertices, 1,000 hyperedges, cardinality U[2,8], batches of 50+50"
    return (f"large, uniform membership: {s.n_vertices:,} vertices, {s.initial.n:,} hyperedges, "
            f"cardinality Zipf(2.0) in [2,{s.meta['kmax']}], uniform members, batches of "
            f"{args.batch // 2:,} inserts + {args.batch - args.batch // 2:,} deletes")


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    from paper_2512_21009_gb300 import escher as E
    rank, ws, local, dist = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # several ranks: by default one hypergraph whose count is split across
    # the ranks (every rank holds the same graph and batches; one all-reduce
    # of the counts per step); --replicas: an independent graph per rank
    split = ws > 1 and not args.replicas
    s, fam = make_stream(args, 0 if split else rank)
    init = s.initial
    nb = args.warmup + 2 * args.steps
    n_upd = [b.inserts.n + len(b.del_ranks) for b in s.batches[:nb]]
    cap_e = init.n + max(b.inserts.n for b in s.batches) + 64
    cap_inc = int(init.nnz * 1.6) + 4 * max(b.inserts.nnz for b in s.batches)
    max_bh = max(max(n_upd), 1)
    max_bi = max(max(b.inserts.nnz for b in s.batches), 1)
    # initial hypergraph enters in chunks of at most max_batch_*
    max_bh = max(max_bh, min(init.n, 100_000))
    max_bi = max(max_bi, 4 * max_bh * 16)
    todev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)  # noqa: E731
    t0 = time.time()
    g = E.Graph(s.n_vertices, todev(init.offsets, np.int64), todev(init.members, np.int32),
                todev(init.timestamps, np.int64), capacity_hyperedges=cap_e, capacity_incidences=cap_inc,
                max_batch_hyperedges=max_bh, max_batch_incidences=max_bi, families=fam,
                stream=torch.cuda.current_stream(dev))
    torch.cuda.synchronize(dev)
    t_create = time.time() - t0
    # the library's autotuner picks the counter's launch shape on this graph:
    # it counts (and discards) the triads of a seeded sample of live
    # hyperedges the size of one batch's changes, once per candidate
    tune = None
    if not args.no_autotune:
        rng_t = np.random.default_rng(args.seed + 17)
        sample = np.sort(rng_t.choice(init.n, size=min(init.n, args.batch), replace=False)).astype(np.int32)
        t1 = time.time()
        tune = g.autotune(sample, reps=1)
        tune["seconds"] = round(time.time() - t1, 2)
    # deletes resolved through a client copy of the ID rule; the IDs it
    # predicts for the inserts are checked against the library's after the run
    model = _LiveRule(init.n)
    predicted = []
    dev_batches, host_batches = [], []
    for b in s.batches[:nb]:
        dels, ids_pred = model.step(b.del_ranks, b.inserts.n)
        dels = dels.astype(np.int32)
        predicted.append(ids_pred)
        dev_batches.append((todev(b.inserts.offsets, np.int64), todev(b.inserts.members, np.int32),
                            todev(b.inserts.timestamps, np.int64), todev(dels, np.int32)))
        pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()  # noqa: E731
        host_batches.append((pin(b.inserts.offsets, np.int64), pin(b.inserts.members, np.int32),
                             pin(b.inserts.timestamps, np.int64), pin(dels, np.int32)))
    returned = []
    if split:
        g.set_split(rank, ws)
    # the summed counts of a split graph (hyperedge 30 + vertex 3), on the device
    shares = torch.zeros(33, dtype=torch.int64, device=dev)

    def reduce_counts():
        """One all-reduce of this rank's shares of the counts: the int64 images
        of the uint64 counts, whose sum is exact modulo 2^64."""
        E.esc_triads(g.h, E.TRIAD_HYPEREDGE, 0, shares[0:30])
        E.esc_triads(g.h, E.TRIAD_VERTEX, 0, shares[30:33])
        dist.all_reduce(shares, op=dist.ReduceOp.SUM)

    def step(batch, want_ids=True):
        out = np.zeros(batch[0].numel() - 1, np.int32)
        E.esc_apply_batch(g.h, batch[0], batch[1], batch[2], batch[3], out)
        returned.append(out)
        if split:
            reduce_counts()

    st = torch.cuda.current_stream(dev)
    g.set_profiling(True)
    for k in range(args.warmup):
        step(dev_batches[k])
    torch.cuda.synchronize(dev)
    barrier(dist, dev)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = g.launch_count()
    lat, cnt_ms, store_ms, triads = [], [], [], 0
    cen_ms, cen_launches = 0.0, 0
    terms = {"store": 0, "build": 0, "closed": 0, "open": 0}   # algorithmic bytes
    work = [0] * 6
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for k in range(args.warmup, args.warmup + args.steps):
        ts0 = time.perf_counter()
        step(dev_batches[k])
        lat.append((time.perf_counter() - ts0) * 1e3)
        sts = g.stats()
        cnt_ms.append(sts["ms_count_del"] + sts["ms_count_ins"])
        store_ms.append(sts["ms_ingest"] + sts["ms_store"])
        for k in terms:
            terms[k] += 4 * sts["alg_" + k]
        cen_ms += sts["ms_center"]
        cen_launches += sts["center_launches"]
        triads += sts["triads"]
        work = [a + b for a, b in zip(work, sts["work"])]
    e1.record(st)
    torch.cuda.synchronize(dev)
    launches = g.launch_count() - launches0
    barrier(dist, dev)
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    # end-to-end through the public API with pinned host buffers: H2D of the
    # batch inside the call, D2H of the refreshed counts
    lat_e2e = []
    h2d = d2h = 0
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    te0 = time.perf_counter()
    for k in range(args.warmup + args.steps, nb):
        hb = host_batches[k]
        t1 = time.perf_counter()
        out = np.zeros(hb[0].numel() - 1, np.int32)
        E.esc_apply_batch(g.h, hb[0].numpy(), hb[1].numpy(), hb[2].numpy(), hb[3].numpy(), out)
        returned.append(out)
        if split:
            reduce_counts()
            c = {"counts": shares.cpu().numpy()}
        else:
            c = g.counts()
        lat_e2e.append((time.perf_counter() - t1) * 1e3)
        h2d += sum(t.numel() * t.element_size() for t in hb)
        d2h += sum(v.nbytes for v in c.values())
    te = time.perf_counter() - te0
    barrier(dist, dev)
    # the library's IDs are the ones the client's copy of the ID rule predicted
    for k, out in enumerate(returned):
        if not np.array_equal(out, predicted[k]):
            raise SystemExit(f"bench: batch {k}: the library's IDs differ from the ID rule's prediction")
    upd_timed = sum(n_upd[args.warmup:args.warmup + args.steps])
    upd_e2e = sum(n_upd[args.warmup + args.steps:nb])
    if split:
        # one job: every rank applies the same updates
        t_max, tot_upd = allreduce_max(dist, elapsed, dev), upd_timed
        te_max, tot_upd_e2e = allreduce_max(dist, te, dev), upd_e2e
    else:
        t_max, tot_upd = combine(dist, dev, elapsed, upd_timed)
        te_max, tot_upd_e2e = combine(dist, dev, te, upd_e2e)
    if rank != 0:
        return
    hbm, kind = peaks()
    cnt_s = sum(cnt_ms) / 1e3
    alg_bytes = sum(terms.values())
    count_achieved = alg_bytes / cnt_s / 1e9 if cnt_s > 0 else 0.0
    # the dominant kernel: the centre kernel, timed with events around each
    # launch; its algorithmic bytes are the closed-pair and open-path terms
    cen_bytes = terms["closed"] + terms["open"]
    achieved = cen_bytes / (cen_ms / 1e3) / 1e9 if cen_ms > 0 else 0.0
    per_launch = cen_bytes / max(cen_launches, 1)
    traffic, traffic_note = centre_traffic(args, per_launch)
    lat_sorted = sorted(lat)
    res = {
        "metric": METRIC, "value": tot_upd / t_max, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "strong" if split else "weak", "vs_baseline": None, "dtype": "int32 ids / uint64 counts",
        "data": "synthetic",
        "config": {"workload": workload_desc(args, s), "families": "hyperedge (30) + incident-vertex (3)",
                   "updates_per_step": args.batch,
                   "parallelism": f"work split x{ws}" if split else f"replicas x{ws}",
                   "l2": "resident store larger than L2 (129 MB)",
                   "create_s": round(t_create, 2), "autotune": tune},
        "latency_ms": {"p50": float(np.percentile(lat_sorted, 50)), "p99": float(np.percentile(lat_sorted, 99))},
        "stage_ms_per_step": {"count": sum(cnt_ms) / len(cnt_ms), "store_and_ingest": sum(store_ms) / len(store_ms)},
        "triads_per_step": triads / args.steps,
        "counter_work_per_step": {k: v / args.steps for k, v in zip(
            ["centre_items", "n_g1_build_entries", "pair_pass_visits", "closed_pairs", "slow_t_steps",
             "aggregate_visits"], work)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "traffic_source": traffic_note,
                     "peak_kind": kind,
                     "kernel": "k_center_o (centre kernel of the triad count)",
                     "bytes": ("4 B per int32 entry; the centre kernel's terms: closed pairs, min(|g1|, |g2|) "
                               "per closed pair {g1, g2} of N(h) counted, and open paths, the sum of g1's member "
                               "degrees per pair (h, g1)"),
                     "bytes_per_step_by_term": {k: v / args.steps for k, v in terms.items()},
                     "algorithmic_bytes_per_launch": per_launch,
                     "ms_per_launch": cen_ms / max(cen_launches, 1), "launches_per_step": cen_launches / args.steps,
                     "count_phase": {"achieved": count_achieved, "frac": count_achieved / hbm,
                                     "algorithmic_bytes_per_step": alg_bytes / args.steps,
                                     "ms_per_step": sum(cnt_ms) / len(cnt_ms)}},
        "e2e": {"value": tot_upd_e2e / te_max, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps, "steps": args.steps,
                "latency_ms": {"p50": float(np.percentile(lat_e2e, 50)), "p99": float(np.percentile(lat_e2e, 99))}},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args, s, budget_s=args.cpu_budget)
    print(json.dumps(res))


# ---------------------------------------------------------------------------
# the large workload as specified: Zipf(1.1) vertex popularity
# ---------------------------------------------------------------------------

def run_large_zipf(args):
    """1M vertices, 2M hyperedges, cardinality Zipf(2.0) in [2,1000], vertex
    popularity Zipf(1.1) (a vertex in ~44% of the hyperedges), batches of 5e4
    inserts + 5e4 deletes: the store update and incident-vertex types 1 and 2
    from vertex-pair statistics (ESC_FAMILY_VERTEX12).  The hyperedge family
    and type 3 would need every neighbourhood of a hub-holding hyperedge
    (~1e6 entries each) and are not kept here."""
    import torch
    from paper_2512_21009_gb300 import escher as E
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    nb = args.warmup + 2 * args.steps
    s = gen.large(seed=args.seed, membership="zipf", scale=args.scale, n_batches=nb, batch_updates=args.batch)
    init = s.initial
    fam = 8
    sizes_init = np.diff(init.offsets).astype(np.int64)
    pairs_all = int((sizes_init * (sizes_init - 1) // 2).sum())
    for b in s.batches[:nb]:
        k = np.diff(b.inserts.offsets).astype(np.int64)
        pairs_all += int((k * (k - 1) // 2).sum())
    max_bh = max(args.batch, min(init.n, 100_000))
    max_bi = max(max(b.inserts.nnz for b in s.batches), 4 * max_bh * 16)
    todev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)  # noqa: E731
    t0 = time.time()
    g = E.Graph(s.n_vertices, todev(init.offsets, np.int64), todev(init.members, np.int32),
                todev(init.timestamps, np.int64), capacity_hyperedges=init.n + args.batch + 64,
                capacity_incidences=int(init.nnz * 1.6) + 4 * max(b.inserts.nnz for b in s.batches),
                max_batch_hyperedges=max_bh, max_batch_incidences=max_bi, families=fam,
                capacity_vertex_pairs=pairs_all, stream=torch.cuda.current_stream(dev))
    torch.cuda.synchronize(dev)
    t_create = time.time() - t0
    model = _LiveRule(init.n)
    size_of = np.zeros(init.n + args.batch * nb + 64, np.int64)
    size_of[:init.n] = sizes_init
    predicted, dev_batches, host_batches, pair_ops = [], [], [], []
    for b in s.batches[:nb]:
        dels, ids = model.step(b.del_ranks, b.inserts.n)
        kd = size_of[dels]
        ki = np.diff(b.inserts.offsets).astype(np.int64)
        pair_ops.append(int((kd * (kd - 1) // 2).sum() + (ki * (ki - 1) // 2).sum()))
        size_of[ids] = ki
        predicted.append(ids)
        d32 = dels.astype(np.int32)
        dev_batches.append((todev(b.inserts.offsets, np.int64), todev(b.inserts.members, np.int32),
                            todev(b.inserts.timestamps, np.int64), todev(d32, np.int32)))
        pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()  # noqa: E731
        host_batches.append((pin(b.inserts.offsets, np.int64), pin(b.inserts.members, np.int32),
                             pin(b.inserts.timestamps, np.int64), pin(d32, np.int32)))
    returned = []
    g.set_profiling(True)

    def step(bt):
        out = np.zeros(bt[0].numel() - 1, np.int32)
        E.esc_apply_batch(g.h, bt[0], bt[1], bt[2], bt[3], out)
        returned.append(out)

    st = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        step(dev_batches[k])
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = g.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat, pair_ms, stage = [], [], {"ingest": 0.0, "pairs": 0.0, "store": 0.0, "count_ins": 0.0}
    e0.record(st)
    for k in range(args.warmup, args.warmup + args.steps):
        ts0 = time.perf_counter()
        step(dev_batches[k])
        lat.append((time.perf_counter() - ts0) * 1e3)
        sts = g.stats()
        pair_ms.append(sts["ms_count_del"])
        for name, key in (("ingest", "ms_ingest"), ("pairs", "ms_count_del"), ("store", "ms_store"),
                          ("count_ins", "ms_count_ins")):
            stage[name] += sts[key] / args.steps
    e1.record(st)
    torch.cuda.synchronize(dev)
    launches = g.launch_count() - l0
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    lat_e2e, h2d, d2h = [], 0, 0
    te0 = time.perf_counter()
    for k in range(args.warmup + args.steps, nb):
        hb = host_batches[k]
        t1 = time.perf_counter()
        out = np.zeros(hb[0].numel() - 1, np.int32)
        E.esc_apply_batch(g.h, hb[0].numpy(), hb[1].numpy(), hb[2].numpy(), hb[3].numpy(), out)
        returned.append(out)
        c = g.counts()
        lat_e2e.append((time.perf_counter() - t1) * 1e3)
        h2d += sum(t.numel() * t.element_size() for t in hb)
        d2h += sum(v.nbytes for v in c.values())
    te = time.perf_counter() - te0
    for k, out in enumerate(returned):
        if not np.array_equal(out, predicted[k]):
            raise SystemExit(f"bench: batch {k}: the library's IDs differ from the ID rule's prediction")
    v = g.counts()["vertex"]
    g.close()
    n_upd = [b.inserts.n + len(b.del_ranks) for b in s.batches[:nb]]
    upd = sum(n_upd[args.warmup:args.warmup + args.steps])
    upd_e2e = sum(n_upd[args.warmup + args.steps:nb])
    hbm, kind = peaks()
    ops = sum(pair_ops[args.warmup:args.warmup + args.steps])
    pair_s = sum(pair_ms) / 1e3
    # algorithmic bytes of the pair kernel: per (changed hyperedge, member
    # pair), the pair's key (8 B) and its packed word (8 B read, 8 B written)
    achieved = 24.0 * ops / pair_s / 1e9 if pair_s > 0 else 0.0
    print(json.dumps({
        "metric": METRIC, "value": upd / elapsed, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32 ids / uint64 counts", "data": "synthetic",
        "config": {"workload": (f"large, Zipf(1.1) vertex popularity as specified: {s.n_vertices:,} vertices, "
                                f"{init.n:,} hyperedges, cardinality Zipf(2.0) in [2,{s.meta['kmax']}], batches of "
                                f"{args.batch // 2:,} inserts + {args.batch - args.batch // 2:,} deletes"),
                   "families": "incident-vertex types 1 and 2 (ESC_FAMILY_VERTEX12: vertex-pair statistics)",
                   "max_vertex_degree": int(np.bincount(init.members).max()),
                   "vertex_pairs_capacity": pairs_all, "create_s": round(t_create, 2)},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "pair_updates_per_step": ops / args.steps,
        "stage_ms_per_step": stage,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "peak_kind": kind,
                     "kernel": "k_pairs (vertex-pair statistics; timed with its prefix-scan kernels)",
                     "bytes": "24 B per (changed hyperedge, member pair): the pair's key and its packed word "
                              "read and written",
                     "ms_per_step": pair_s * 1e3 / args.steps,
                     "pair_ops_per_s": ops / pair_s if pair_s > 0 else 0.0},
        "e2e": {"value": upd_e2e / te, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps, "steps": args.steps},
        "gpu_launches": int(launches), "clocks": clk,
        "vertex_types_final": [int(x) for x in v],
    }))


# ---------------------------------------------------------------------------
# DRAM traffic of the centre kernel, from the committed ncu summary
# ---------------------------------------------------------------------------

TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "k_center_o_large_uniform.md")
COUNT_SRC = os.path.join(ROOT, "paper_2512_21009_gb300", "csrc", "count.cu")


def centre_traffic(args, alg_bytes_per_launch):
    """DRAM bytes (read + write) of one centre-kernel launch: the ratio of
    DRAM bytes to algorithmic bytes that a one-pass ncu capture of this
    workload at full size measured (both sides of one step), times this
    launch's algorithmic bytes.  Only when the summary was taken on the
    kernel source that is built now (its sha256 is recorded there);
    otherwise None."""
    import hashlib
    if args.workload != "large_uniform" or not os.path.exists(TRAFFIC_SUMMARY):
        return None, "no capture of this workload"
    with open(COUNT_SRC, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    ratio, src = None, None
    for line in open(TRAFFIC_SUMMARY):
        if line.startswith("- dram bytes per algorithmic byte:"):
            try:
                ratio = float(line.split(":", 1)[1].split()[0])
            except ValueError:
                ratio = None
        if line.startswith("- source sha256 of count.cu:"):
            src = line.split(":", 1)[1].strip().strip("`")
    if ratio is None or src != sha:
        return None, "the centre kernel changed since the last ncu capture"
    return ratio * alg_bytes_per_launch, ("ncu dram__bytes_read.sum + dram__bytes_write.sum of a one-pass capture of "
                                          "this workload at full size on this kernel source, as DRAM bytes per "
                                          "algorithmic byte, times this run's algorithmic bytes per launch "
                                          f"({ratio:.3f}; {TRAFFIC_SUMMARY[len(ROOT) + 1:]})")


# ---------------------------------------------------------------------------
# the oracle on a bounded sample, on all host cores
# ---------------------------------------------------------------------------

ORACLE_KMAX = 16   # cardinality cap of the sampled updates (see oracle_sample)


def _sorted_csr(c):
    """CSR with every hyperedge's members sorted (the oracle's input form)."""
    sizes = np.diff(c.offsets)
    rows = np.repeat(np.arange(c.n), sizes)
    return np.ascontiguousarray(c.offsets, dtype=np.int64), np.ascontiguousarray(
        c.members[np.lexsort((c.members, rows))], dtype=np.int32)


class _OracleBatch:
    """The old and new graph of the stream's first batch, as the oracle takes
    them: the deleted hyperedges are positions of the old graph (IDs equal
    positions there), the inserted ones the positions appended to the kept
    hyperedges in the new graph.  Positions stand in for IDs: the hyperedge
    and incident-vertex families do not depend on IDs."""

    def __init__(self, s):
        init, b = s.initial, s.batches[0]
        self.off0, self.mem0 = _sorted_csr(init)
        sizes0 = np.diff(self.off0)
        self.dels = np.sort(np.asarray(b.del_ranks, dtype=np.int64))
        keep = np.ones(init.n, bool)
        keep[self.dels] = False
        ioff, imem = _sorted_csr(b.inserts)
        sizes1 = np.concatenate([sizes0[keep], np.diff(ioff)])
        self.off1 = np.concatenate([[0], np.cumsum(sizes1)]).astype(np.int64)
        self.mem1 = np.concatenate([self.mem0[np.repeat(keep, sizes0)], imem]).astype(np.int32)
        self.ins = np.arange(int(keep.sum()), int(keep.sum()) + b.inserts.n, dtype=np.int64)
        self.del_small = self.dels[sizes0[self.dels] <= ORACLE_KMAX]
        self.ins_small = self.ins[np.diff(ioff) <= ORACLE_KMAX]
        self.share = (self.del_small.size + self.ins_small.size) / max(1, self.dels.size + self.ins.size)


def oracle_sample(ob, threads, per_thread, seed):
    """Wall time of the oracle's count change for a sample of the batch's
    updates, on `threads` host threads: each thread takes per_thread sampled
    updates (deletes and inserts alternately) and runs the oracle's
    enumeration of the hyperedge triads (orc_count_containing) and of the
    incident-vertex witness assignments (orc_vertex_containing) holding its
    deleted hyperedges on the old graph and its inserted ones on the new graph.
    Updates are drawn uniformly among those of cardinality <= ORACLE_KMAX: the
    oracle's time per update grows with the cardinality (seconds at 10
    members, half a minute at 50, minutes at 200), so the sample's rate
    overstates the oracle's rate over the whole batch.  Returns (seconds,
    updates)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    n = threads * per_thread
    nd = min(n // 2, ob.del_small.size)
    ni = min(n - nd, ob.ins_small.size)
    sd = np.sort(rng.choice(ob.del_small, size=nd, replace=False))
    si = np.sort(rng.choice(ob.ins_small, size=ni, replace=False))

    def work(t):
        a, c = sd[t::threads], si[t::threads]
        if a.size:
            O.count_containing(ob.off0, ob.mem0, None, None, 0, O.FAM_HYPEREDGE, a)
            O.count_vertex_containing(ob.off0, ob.mem0, a)
        if c.size:
            O.count_containing(ob.off1, ob.mem1, None, None, 0, O.FAM_HYPEREDGE, c)
            O.count_vertex_containing(ob.off1, ob.mem1, c)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(work, range(threads)))
    return time.perf_counter() - t0, nd + ni


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _sample_desc(ob, upd, threads, per_thread, secs=None):
    t = f"; {secs:.1f} s" if secs is not None else ""
    return (f"{upd} updates of the first batch ({per_thread} per thread, deletes on the old graph and inserts on "
            f"the new one), drawn among its updates of cardinality <= {ORACLE_KMAX} ({ob.share:.1%} of them; larger "
            f"ones cost the oracle far more, so this rate overstates the oracle's): the oracle's enumeration of "
            f"the hyperedge triads and incident-vertex instances holding them on the full graph, {threads} "
            f"threads{t}")


def cpu_baseline(args, s, budget_s=20.0):
    from oracle import oracle as O
    O.build()
    ob = _OracleBatch(s)
    threads = host_threads()
    per_thread = 1
    secs, upd = oracle_sample(ob, threads, per_thread, seed=1)
    # grow the sample until it takes a meaningful share of the budget
    while secs < budget_s / 3 and per_thread < 16:
        per_thread *= 2
        secs, upd = oracle_sample(ob, threads, per_thread, seed=per_thread)
    return {"value": upd / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "cpu": cpu_model(), "sample": _sample_desc(ob, upd, threads, per_thread, secs)}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    s, fam = make_stream(args, 0)
    from oracle import oracle as O
    O.build()
    ob = _OracleBatch(s)
    threads = host_threads()
    per_thread = 1
    # warm-up steps (the oracle has no warm-up effects): one update each
    for k in range(args.warmup):
        oracle_sample(ob, 1, 1, seed=1000 + k)
    secs, upd, lat = 0.0, 0, []
    for k in range(args.steps):
        t, u = oracle_sample(ob, threads, per_thread, seed=k)
        secs += t
        upd += u
        lat.append(t * 1e3)
    value = upd / secs
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "uint64", "data": "synthetic",
        "config": {"workload": workload_desc(args, s), "families": "hyperedge (30) + incident-vertex (3)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": cpu_model(),
                         "sample": "per step: " + _sample_desc(ob, threads * per_thread, threads, per_thread)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# horizontal updates: vertex sets of live hyperedges change in place
# ---------------------------------------------------------------------------

def run_horizontal(args):
    """The 1M-vertex uniform workload; each step changes the vertex sets of
    --batch / 2 distinct live hyperedges (about 30% of each one's members
    dropped, 0-3 uniform vertices added), which keep their IDs (Sec. III-B's
    incident-vertex insertions and deletions).  Hyperedge + vertex families."""
    import torch
    from paper_2512_21009_gb300 import escher as E
    torch.cuda.set_device(0)
    s = gen.large(seed=args.seed, membership="uniform", scale=args.scale, n_batches=1, batch_updates=2)
    init = s.initial
    n_up = max(1, args.batch // 2)
    steps = args.warmup + args.steps
    g = E.Graph(s.n_vertices, init.offsets, init.members, init.timestamps,
                capacity_hyperedges=init.n + 64, capacity_incidences=int(init.nnz * 1.6) + 4096,
                max_batch_hyperedges=max(2 * n_up, min(init.n, 100_000)),
                max_batch_incidences=max(4 * n_up * 16, 1 << 22), families=3)
    rng = np.random.default_rng(args.seed + 5)
    off0, mem0 = init.offsets, init.members
    cur = [mem0[off0[i]:off0[i + 1]] for i in range(init.n)]   # client copy of the vertex sets
    batches = []
    for k in range(steps):
        ids = np.sort(rng.choice(init.n, size=min(n_up, init.n), replace=False)).astype(np.int32)
        sets = []
        for h in ids:
            c = cur[h]
            keep = c[rng.random(c.size) < 0.7]
            new = np.unique(np.concatenate([keep, rng.integers(0, s.n_vertices, size=int(rng.integers(0, 4)))]))
            if new.size == 0:
                new = c[:1]
            cur[h] = new.astype(np.int32)
            sets.append(cur[h])
        off = np.zeros(len(sets) + 1, np.int64)
        off[1:] = np.cumsum([x.size for x in sets])
        batches.append((torch.from_numpy(ids).cuda(), torch.from_numpy(off).cuda(),
                        torch.from_numpy(np.concatenate(sets).astype(np.int32)).cuda()))
    g.set_profiling(True)
    for k in range(args.warmup):
        E.esc_update_members(g.h, *batches[k])
    torch.cuda.synchronize()
    lat, cnt_ms = [], []
    t0 = time.perf_counter()
    for k in range(args.warmup, steps):
        t1 = time.perf_counter()
        E.esc_update_members(g.h, *batches[k])
        lat.append((time.perf_counter() - t1) * 1e3)
        st = g.stats()
        cnt_ms.append(st["ms_count_del"] + st["ms_count_ins"])
    el = time.perf_counter() - t0
    g.close()
    print(json.dumps({
        "metric": METRIC, "value": n_up * args.steps / el, "unit": "hyperedge updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32 ids / uint64 counts",
        "data": "synthetic",
        "config": {"workload": (f"horizontal updates on the uniform large graph ({s.n_vertices:,} vertices, "
                                f"{init.n:,} hyperedges): {n_up:,} distinct hyperedges per batch get a new vertex "
                                "set (~30% of members dropped, 0-3 vertices added), IDs kept"),
                   "families": "hyperedge (30) + incident-vertex (3)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "count_ms_per_step": sum(cnt_ms) / len(cnt_ms),
    }))


# ---------------------------------------------------------------------------
# sweeps: the same kernels over batch size, deletion share, inserted
# cardinality, graph size and cardinality spread (one JSON line per point)
# ---------------------------------------------------------------------------

def _sweep_graph(E, nv, init, n_ids, n_inc, max_bh, max_bi, fam, dev):
    import torch
    todev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)  # noqa: E731
    t0 = time.time()
    g = E.Graph(nv, todev(init.offsets, np.int64), todev(init.members, np.int32), todev(init.timestamps, np.int64),
                capacity_hyperedges=n_ids, capacity_incidences=n_inc, max_batch_hyperedges=max_bh,
                max_batch_incidences=max_bi, families=fam, stream=torch.cuda.current_stream(dev))
    torch.cuda.synchronize(dev)
    return g, time.time() - t0


def _sweep_point(E, g, model, inserts, n_del, args, dev, rng):
    """Apply ``warmup`` then ``steps`` batches (inserts[k] plus n_del deletes
    of uniform live hyperedges, inputs resident on the device); device time
    of the timed ones by CUDA events on the graph's stream."""
    import torch
    todev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)  # noqa: E731
    prepared, expect = [], []
    for csr in inserts:
        idx, dels = model.pick(rng, n_del)
        expect.append(model.commit(idx, dels, csr.n))
        prepared.append((todev(csr.offsets, np.int64), todev(csr.members, np.int32),
                         todev(csr.timestamps, np.int64), todev(np.sort(dels), np.int32)))
    got = []

    def step(b):
        out = np.zeros(b[0].numel() - 1, np.int32)
        E.esc_apply_batch(g.h, b[0], b[1], b[2], b[3], out)
        got.append(out)

    st = torch.cuda.current_stream(dev)
    g.set_profiling(True)
    for k in range(args.warmup):
        step(prepared[k])
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    l0 = g.launch_count()
    lat, cnt_ms, store_ms = [], [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for k in range(args.warmup, args.warmup + args.steps):
        t1 = time.perf_counter()
        step(prepared[k])
        lat.append((time.perf_counter() - t1) * 1e3)
        sts = g.stats()
        cnt_ms.append(sts["ms_count_del"] + sts["ms_count_ins"])
        store_ms.append(sts["ms_ingest"] + sts["ms_store"])
    e1.record(st)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    el = e0.elapsed_time(e1) / 1e3
    for want, have in zip(expect, got):
        if not np.array_equal(want, have):
            raise SystemExit("bench: assigned IDs differ from the client's copy of the ID rule")
    upd = sum(inserts[k].n + n_del for k in range(args.warmup, args.warmup + args.steps))
    return {"value": upd / el, "ms_per_step": el * 1e3 / args.steps,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "stage_ms_per_step": {"count": sum(cnt_ms) / len(cnt_ms), "store_and_ingest": sum(store_ms) / len(store_ms)},
            "gpu_launches": int(g.launch_count() - l0), "clocks": clk}


def _sweep_line(args, r, workload, sweep, point, families, extra=None):
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int32 ids / uint64 counts", "data": "synthetic",
           "config": {"workload": workload, "sweep": sweep, "point": point, "families": families,
                      "l2": "resident store larger than L2 (129 MB)"},
           "latency_ms": r["latency_ms"], "stage_ms_per_step": r["stage_ms_per_step"],
           "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
    if extra:
        out["config"].update(extra)
    print(json.dumps(out), flush=True)


def run_sweep(args):
    """Figs. 5a-c, 7 and 15 as synthetic sweeps.  batch: 50K/100K/200K
    updates, half inserts; delete: 50K updates with 20-80% deletes; card:
    50K inserts with cardinality Zipf(2.0) capped at 50/100/200; these three
    share the uniform 1M-vertex graph of the default workload.  size: graphs
    of 20M-55M hyperedges (times --size-scale), |V| = |E|/3, cardinality
    Zipf(2.0) in [2, --size-kmax] (default 1,000; at the paper's 10,000 one
    point at 1M hyperedges takes minutes: the largest hyperedges meet ~4e5
    neighbours each), 50K updates.  spread: a dyadic graph (1M
    vertices, 4M two-member hyperedges), 50K updates whose inserted
    cardinalities have mean 4 and standard deviation 0-16 (first point: plain
    edges), incident-vertex family."""
    import torch
    from paper_2512_21009_gb300 import escher as E
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    nb = args.warmup + args.steps
    rng = np.random.default_rng(args.seed + 101)
    fam_hv = "hyperedge (30) + incident-vertex (3)"
    if args.sweep in ("batch", "delete", "card"):
        s = gen.large(seed=args.seed, membership="uniform", scale=args.scale, n_batches=0)
        init = s.initial
        t_end = int(init.timestamps[-1])
        if args.sweep == "batch":
            pts = [(dict(batch=b, delete_pct=50), b - b // 2, b // 2, 1000) for b in (50_000, 100_000, 200_000)]
        elif args.sweep == "delete":
            pts = [(dict(batch=50_000, delete_pct=p), 50_000 - 500 * p, 500 * p, 1000) for p in (20, 40, 60, 80)]
        else:
            pts = [(dict(inserts=50_000, card_cap=c), 50_000, 0, c) for c in (50, 100, 200)]
        ins = [gen.insert_batches(args.seed + 7 + i, s.n_vertices, nb, n_ins, kmax, ts_start=t_end)
               for i, (_, n_ins, _, kmax) in enumerate(pts)]
        n_ids = init.n + sum(c.n for L in ins for c in L) + 64
        n_inc = int(1.6 * (init.nnz + sum(c.nnz for L in ins for c in L))) + (1 << 20)
        max_bh = max(max(n_i + n_d for _, n_i, n_d, _ in pts), min(init.n, 100_000))
        max_bi = max(max(c.nnz for L in ins for c in L), 4 * max_bh * 16)
        g, t_create = _sweep_graph(E, s.n_vertices, init, n_ids, n_inc, max_bh, max_bi, 3, dev)
        model = _IdModel(init.n)
        desc = (f"large, uniform membership: {s.n_vertices:,} vertices, {init.n:,} initial hyperedges, "
                "cardinality Zipf(2.0) in [2,1000]; inserts Zipf(2.0) in [2, cap], uniform members; deletes "
                "uniform over live hyperedges")
        for (point, n_ins, n_del, _), L in zip(pts, ins):
            r = _sweep_point(E, g, model, L, n_del, args, dev, rng)
            _sweep_line(args, r, desc, args.sweep, point, fam_hv, {"create_s": round(t_create, 2)})
        g.close()
    elif args.sweep == "size":
        for i, m in enumerate((20, 30, 40, 55)):
            if args.size_points and m not in args.size_points:
                continue
            n_e = max(64, int(round(m * 1e6 * args.size_scale)))
            nv = max(10_000, n_e // 3)
            init = gen.random_hypergraph(args.seed + 31 + i, nv, n_e, args.size_kmax)
            L = gen.insert_batches(args.seed + 41 + i, nv, nb, 25_000, args.size_kmax,
                                   ts_start=int(init.timestamps[-1]))
            n_ids = init.n + 25_000 * nb + 64
            n_inc = int(1.6 * (init.nnz + sum(c.nnz for c in L))) + (1 << 20)
            max_bh = max(50_000, min(init.n, 100_000))
            max_bi = max(max(c.nnz for c in L), 1 << 24)
            g, t_create = _sweep_graph(E, nv, init, n_ids, n_inc, max_bh, max_bi, 3, dev)
            r = _sweep_point(E, g, _IdModel(init.n), L, 25_000, args, dev, rng)
            desc = (f"random hypergraph: {n_e:,} hyperedges ({m}M x {args.size_scale}), {nv:,} vertices (|E|/3), "
                    f"cardinality Zipf(2.0) in [2,{args.size_kmax}], uniform members; batches of 25,000 inserts "
                    "(same distribution) + 25,000 uniform deletes")
            _sweep_line(args, r, desc, "size", dict(hyperedges=n_e, vertices=nv, incidences=int(init.nnz)), fam_hv,
                        {"create_s": round(t_create, 2)})
            g.close()
            del g
            torch.cuda.empty_cache()
    else:  # spread
        nv, n_e = int(round(1_000_000 * args.scale)), int(round(4_000_000 * args.scale))
        init = gen.dyadic_graph(args.seed + 51, nv, n_e)
        pts = [(2.0, 0.0)] + [(4.0, sd) for sd in (0.0, 1.0, 2.0, 4.0, 8.0, 16.0)]
        ins = [gen.spread_inserts(args.seed + 61 + i, nv, nb, 25_000, mu, sd, ts_start=int(init.timestamps[-1]))
               for i, (mu, sd) in enumerate(pts)]
        n_ids = init.n + sum(c.n for L in ins for c in L) + 64
        n_inc = int(1.6 * (init.nnz + sum(c.nnz for L in ins for c in L))) + (1 << 20)
        max_bh = max(50_000, min(init.n, 100_000))
        max_bi = max(max(c.nnz for L in ins for c in L), 1 << 22)
        g, t_create = _sweep_graph(E, nv, init, n_ids, n_inc, max_bh, max_bi, 2, dev)
        model = _IdModel(init.n)
        desc = (f"dyadic graph: {nv:,} vertices, {n_e:,} two-member hyperedges (uniform distinct endpoints); "
                "batches of 25,000 inserts with uniform members and 25,000 uniform deletes")
        for (mu, sd), L in zip(pts, ins):
            k = np.concatenate([np.diff(c.offsets) for c in L[args.warmup:]])
            r = _sweep_point(E, g, model, L, 25_000, args, dev, rng)
            _sweep_line(args, r, desc, "spread",
                        dict(card_mean=round(float(k.mean()), 3), card_std=round(float(k.std()), 3),
                             card_max=int(k.max())),
                        "incident-vertex (3); on plain edges type 3 is the triangle count",
                        {"create_s": round(t_create, 2)})
        g.close()


# ---------------------------------------------------------------------------
# batched form: many hypergraphs, one call vs one call per graph
# ---------------------------------------------------------------------------

def _group_cfgs(E, streams, delta, fam, max_bh, max_bi):
    shared = E.make_config(1, 1, 1, max_bh, max_bi, fam, delta)
    cfgs = []
    for st in streams:
        b = st.batches[0]
        cfgs.append(E.make_config(st.n_vertices, st.initial.n + b.inserts.n + 64,
                                  int(st.initial.nnz * 1.5) + 2 * b.inserts.nnz + 1024, 0, 0, fam, delta))
    return shared, cfgs


def _load_group(E, grp, streams, max_bh, max_bi):
    """Initial hyperedges of every graph, in calls that fit the staging
    limits: a graph larger than one call is loaded in pieces, in order, one
    piece of it per call (with no deletes the ID rule gives fresh IDs
    upward, so its hyperedges keep the IDs 0..n-1)."""
    pieces = []
    for st in streams:
        off, n, lo, mine = st.initial.offsets, st.initial.n, 0, []
        while lo < n:
            hi = lo
            while hi < n and hi - lo < max_bh and off[hi + 1] - off[lo] <= max_bi:
                hi += 1
            if hi == lo:
                raise SystemExit("bench: a hyperedge has more members than max_batch_incidences")
            mine.append((lo, hi))
            lo = hi
        pieces.append(mine)
    nxt = [0] * len(streams)
    todo = [i for i in range(len(streams)) if pieces[i]]
    while todo:
        call, nh, ni, rest = [], 0, 0, []
        for i in todo:
            st = streams[i]
            lo, hi = pieces[i][nxt[i]]
            a, b = int(st.initial.offsets[lo]), int(st.initial.offsets[hi])
            if call and (nh + hi - lo > max_bh or ni + b - a > max_bi):
                rest.append(i)
                continue
            nh += hi - lo
            ni += b - a
            call.append(dict(graph=i, ins_offsets=st.initial.offsets[lo:hi + 1] - a,
                             ins_members=st.initial.members[a:b], ins_timestamps=st.initial.timestamps[lo:hi],
                             del_ids=None))
            nxt[i] += 1
            if nxt[i] < len(pieces[i]):
                rest.append(i)
        E.esc_group_apply(grp, call)
        todo = rest


def run_batched(args):
    """One update batch for each of many independent hypergraphs (initial sizes
    log-uniform, one mixed batch each, all three families).  The same batches
    are applied to two identical groups: one esc_group_apply call per graph
    (plain, one batch per launch sequence) and one call for all graphs
    (batched).  Every graph's counts must agree between the two."""
    import torch
    from paper_2512_21009_gb300 import escher as E
    rank, ws, local, dist = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ms = gen.batched(seed=4, n_graphs=args.graphs or 256, e_hi=1e6 * args.scale, b_hi=1e5 * args.scale)
    streams = [ms.graphs[i] for i in shard(len(ms.graphs), rank, ws)]   # graphs are independent
    fam, delta = 7, ms.delta
    tot_upd = sum(st.batches[0].inserts.n + len(st.batches[0].del_ranks) for st in streams)
    max_bh = max(1 << 20, tot_upd + 1024)
    max_bi = max(1 << 24, sum(st.batches[0].inserts.nnz for st in streams) + 1024)
    shared, cfgs = _group_cfgs(E, streams, delta, fam, max_bh, max_bi)
    groups = []
    t0 = time.time()
    for _ in range(2):
        grp = E.esc_group_create(shared, cfgs)
        _load_group(E, grp, streams, max_bh, max_bi)
        groups.append(grp)
    torch.cuda.synchronize()
    t_create = time.time() - t0
    batches = []
    for i, st in enumerate(streams):
        b = st.batches[0]
        # initial IDs are 0..E0-1 and no insert happened yet: ranks are IDs
        dels = np.sort(b.del_ranks).astype(np.int32)
        batches.append(dict(graph=i, ins_offsets=b.inserts.offsets, ins_members=b.inserts.members,
                            ins_timestamps=b.inserts.timestamps, del_ids=dels))
    # plain: one call per graph
    lat = []
    barrier(dist, dev)
    t0 = time.perf_counter()
    for bt in batches:
        t1 = time.perf_counter()
        E.esc_group_apply(groups[0], [bt])
        lat.append((time.perf_counter() - t1) * 1e3)
    t_plain = time.perf_counter() - t0
    # batched: one call for every graph
    l0 = E.esc_group_launch_count(groups[1])
    E.esc_group_set_profiling(groups[1], True)
    barrier(dist, dev)
    t0 = time.perf_counter()
    E.esc_group_apply(groups[1], batches)
    t_batched = time.perf_counter() - t0
    launches_batched = E.esc_group_launch_count(groups[1]) - l0
    bst = E.esc_group_last_stats(groups[1])
    same = True
    for i in range(len(streams)):
        for tt in (0, 1, 2):
            a = E.esc_group_triads(groups[0], i, tt, delta)
            b = E.esc_group_triads(groups[1], i, tt, delta)
            same &= bool(np.array_equal(a, b))
    for grp in groups:
        E.esc_group_destroy(grp)
    t_plain, upd_all = combine(dist, dev, t_plain, tot_upd)
    t_batched, _ = combine(dist, dev, t_batched, tot_upd)
    n_diff = allreduce_sum(dist, 0.0 if same else 1.0, dev)
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": upd_all / t_batched, "unit": UNIT, "n_gpus": ws, "steps": 1, "warmup": 0,
        "ms_per_step": t_batched * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32 ids / uint64 counts", "data": "synthetic",
        "config": {"workload": (f"batched: {len(ms.graphs)} hypergraphs, initial sizes log-uniform "
                                f"[1e3, {1e6 * args.scale:.0e}], vertices = hyperedges/2, cardinality Zipf(2.0) in "
                                f"[2,256], one mixed batch each of log-uniform size [1e2, {1e5 * args.scale:.0e}], "
                                "all three families"), "updates": int(upd_all), "create_s": round(t_create, 2),
                   "parallelism": f"graphs sharded over {ws} rank(s)"},
        "plain": {"value": upd_all / t_plain, "unit": UNIT, "seconds": t_plain, "calls": len(ms.graphs),
                  "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))},
        "batched": {"value": upd_all / t_batched, "unit": UNIT, "seconds": t_batched, "calls": ws,
                    "launches": int(launches_batched)},
        "batched_over_plain": t_plain / t_batched,
        "counts_identical": n_diff == 0,
        "batched_call": {"count_ms": bst["ms_count_del"] + bst["ms_count_ins"], "triads": bst["triads"],
                         "counter_work": dict(zip(["centre_items", "n_g1_build_entries", "pair_pass_visits",
                                                   "closed_pairs", "slow_t_steps", "aggregate_visits"],
                                                  bst["work"]))},
    }))


# ---------------------------------------------------------------------------
# temporal stream with expirations
# ---------------------------------------------------------------------------

def run_temporal(args):
    """Time-ordered stream (batches of 2^16 inserts; every live hyperedge older
    than T - delta, T the batch's last timestamp, is deleted in the same batch)
    with the temporal family kept.  --scale shrinks the vertex count, the
    stream length and the arrival rate together, so the window holds the same
    share of the stream."""
    import torch
    from paper_2512_21009_gb300 import escher as E
    torch.cuda.set_device(0)
    ts = gen.temporal(seed=3, scale=args.scale, rate_per_s=1e3 * args.scale)
    delta = ts.delta
    nv = ts.n_vertices
    n_total = sum(b.n for b in ts.batches)
    nnz_total = sum(b.nnz for b in ts.batches)
    bmax = max(b.n for b in ts.batches)
    g = E.Graph(nv, None, None, None, capacity_hyperedges=n_total + 64, capacity_incidences=nnz_total + 1024,
                max_batch_hyperedges=4 * bmax, max_batch_incidences=max(b.nnz for b in ts.batches) + 1024,
                families=4, delta=delta)
    g.set_profiling(True)
    # timestamps grow along the stream, so the live hyperedges in insertion
    # order have sorted timestamps and each batch's expirations are a prefix
    live_ids = np.zeros(0, np.int32)
    live_ts = np.zeros(0, np.int64)
    lat, upd, t_all = [], [], 0.0
    cnt_ms, triads, work = [], 0, [0] * 6
    for k, b in enumerate(ts.batches):
        t_cut = int(b.timestamps.max()) - delta
        n_exp = int(np.searchsorted(live_ts, t_cut, side="left"))
        dels = np.sort(live_ids[:n_exp])
        t1 = time.perf_counter()
        ids = g.apply_batch(b.offsets, b.members, b.timestamps, dels)
        dt = time.perf_counter() - t1
        live_ids = np.concatenate([live_ids[n_exp:], ids.astype(np.int32)])
        live_ts = np.concatenate([live_ts[n_exp:], b.timestamps])
        if k >= args.warmup:
            lat.append(dt * 1e3)
            upd.append(b.n + n_exp)
            t_all += dt
            sts = g.stats()
            cnt_ms.append(sts["ms_count_del"] + sts["ms_count_ins"])
            triads += sts["triads"]
            work = [a + c for a, c in zip(work, sts["work"])]
    counts = g.triads(E.TRIAD_TEMPORAL)
    g.close()
    print(json.dumps({
        "metric": METRIC, "value": sum(upd) / t_all, "unit": UNIT, "n_gpus": 1, "steps": len(upd),
        "warmup": args.warmup, "ms_per_step": t_all * 1e3 / len(upd), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32 ids / uint64 counts", "data": "synthetic",
        "config": {"workload": (f"temporal: {n_total:,} hyperedges over {nv:,} vertices, cardinality Zipf(2.0) in "
                                f"[2,500], timestamps with Exp gaps (rate {1e3 * args.scale:g}/s), batches of "
                                f"{ts.meta['batch']:,} inserts plus expirations, delta = 3600 s"),
                   "families": "temporal (96)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "live_at_end": int(len(live_ids)), "temporal_triads": int(counts.sum()),
        "count_ms_per_step": sum(cnt_ms) / max(len(cnt_ms), 1),
        "triads_per_step": triads / max(len(cnt_ms), 1),
        "counter_work_per_step": {k: v / max(len(cnt_ms), 1) for k, v in zip(
            ["centre_items", "n_g1_build_entries", "pair_pass_visits", "closed_pairs", "slow_t_steps",
             "aggregate_visits"], work)},
    }))


# ---------------------------------------------------------------------------
# serving loop: Poisson arrivals over many resident graphs
# ---------------------------------------------------------------------------

class _IdModel:
    """Client-side copy of one graph's live IDs under the library's ID rule
    (deletes first; the j-th insert takes the j-th smallest free ID below the
    high-water mark, then fresh IDs), so that a request can delete hyperedges
    inserted by earlier requests that are still queued."""

    def __init__(self, n0: int):
        self.live = np.arange(n0, dtype=np.int32)
        self.n = n0
        self.free = np.zeros(0, np.int32)
        self.hw = n0

    def pick(self, rng, n_del):
        idx = rng.choice(self.n, size=min(n_del, self.n), replace=False)
        return idx, self.live[idx]

    def commit(self, idx, dels, n_ins):
        n, k = self.n, len(idx)
        tail = np.arange(n - k, n)
        moved = tail[~np.isin(tail, idx)]
        holes = np.sort(idx[idx < n - k])
        self.live[holes] = self.live[moved]
        self.n = n - k
        free = np.union1d(self.free, dels)
        take = min(n_ins, len(free))
        ids = np.concatenate([free[:take], np.arange(self.hw, self.hw + n_ins - take, dtype=np.int32)])
        self.free = free[take:].astype(np.int32)
        self.hw += n_ins - take
        if self.n + n_ins > len(self.live):
            self.live = np.concatenate([self.live, np.zeros(max(n_ins, len(self.live) // 2), np.int32)])
        self.live[self.n:self.n + n_ins] = ids
        self.n += n_ins
        return ids.astype(np.int32)


def _drive(E, srv, models, nvs, pool, rng, rate, duration, max_pending, t_clock, log=None):
    """Offer Poisson arrivals at ``rate`` requests/s for ``duration`` s: each
    request is one batch for a uniform graph, size floor(10**U(1, 4)), half
    inserts (cardinality Zipf(2.0) in [2,256], uniform members) and half
    deletes of uniform live hyperedges.  A request that does not fit the
    server's bounded queue is refused and dropped.  Returns the run's record."""
    G = len(models)
    n = max(1, int(rate * duration))
    gaps = rng.exponential(1.0 / rate, size=n)
    t_rel = np.cumsum(gaps)
    graphs = rng.integers(0, G, size=n)
    sizes = np.floor(10 ** rng.uniform(1, 4, size=n)).astype(np.int64)
    poff, pu = pool
    npool = len(poff) - 1
    cursor = int(rng.integers(0, npool))
    tickets, outs, refused = [], [], 0
    t0 = time.monotonic_ns()
    for k in range(n):
        ta = t0 + int(t_rel[k] * 1e9)
        now = time.monotonic_ns()
        if ta > now:
            dt = (ta - now) / 1e9
            if dt > 3e-4:
                time.sleep(dt - 2e-4)
            while time.monotonic_ns() < ta:
                pass
        size = int(sizes[k])
        if E.esc_server_get_stats(srv)["pending_updates"] + size > max_pending:
            refused += 1
            continue
        g = int(graphs[k])
        m = models[g]
        n_ins = size // 2
        idx, dels = m.pick(rng, size - n_ins)
        if cursor + n_ins > npool:
            cursor = 0
        a, b = int(poff[cursor]), int(poff[cursor + n_ins])
        off = (poff[cursor:cursor + n_ins + 1] - a).astype(np.int64)
        mem = np.minimum((pu[a:b] * nvs[g]).astype(np.int32), nvs[g] - 1)
        cursor += n_ins
        ts = (ta // 1000 - t_clock) + np.arange(n_ins, dtype=np.int64)
        dsort = np.sort(dels)
        out = np.zeros(max(n_ins, 1), np.int32)
        tk = E.esc_server_submit(srv, g, off, mem, ts, dsort, out, t_arrival_ns=ta)
        if tk < 0:
            refused += 1
            continue
        want = m.commit(idx, dels, n_ins)
        tickets.append((tk, size))
        outs.append((out, want))
        if log is not None and g in log:
            log[g].append((off, mem, ts, dsort))
    t_sub = time.monotonic_ns()
    E.esc_server_drain(srv)
    lat, done, t_end, calls_b = [], 0, t0, []
    for tk, size in tickets:
        inf = E.esc_server_wait(srv, tk)
        if inf["status"] != 0:
            raise RuntimeError(f"request failed with status {inf['status']}")
        lat.append((inf["t_done_ns"] - inf["t_arrival_ns"]) / 1e6)
        done += size
        t_end = max(t_end, inf["t_done_ns"])
        calls_b.append(inf["call_batches"])
    ids_ok = all(np.array_equal(o[:len(w)], w) for o, w in outs)
    wall = (t_end - t0) / 1e9
    lat = np.asarray(lat) if lat else np.zeros(1)
    return {"offered_per_s": rate, "requests": n, "served": len(tickets), "refused": refused,
            "updates_per_s": done / wall if wall > 0 else 0.0, "seconds": wall,
            "submit_seconds": (t_sub - t0) / 1e9,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_batches_per_call": float(np.mean(calls_b)) if calls_b else 0.0, "ids_ok": bool(ids_ok)}


def run_serving(args):
    """Resident hypergraphs (sizes as the batched workload, times --scale) in
    --shards groups, each group on its own stream with its own server worker
    (so calls of different groups overlap on the device).  Groups are
    admitted one at a time while the server runs under load: a group is
    created only if it fits the device's free memory less a reserve
    (esc_group_fits); later groups that do not fit are refused on the host.
    Poisson request arrivals over the admitted graphs.  Two server policies:
    continuous batching and one request per call.  Each is driven at offered
    loads of 0.25, 0.5 and 1.0 of the capacity of one request per call (the
    same offered mix for both policies), then at 1.0 of its own capacity and
    under overload.  Afterwards a few graphs are rebuilt alone from their
    logged requests and their counts compared with the served ones."""
    import torch
    from paper_2512_21009_gb300 import escher as E
    torch.cuda.set_device(0)
    n_graphs = args.graphs or 1024
    ms = gen.resident_graphs(seed=5, n_graphs=n_graphs, e_hi=1e6 * args.scale)
    all_streams, delta, fam = ms.graphs, ms.delta, 1 | 4
    # per-call limits of each group (they size its count arena: 512 neighbour
    # entries per batch hyperedge): 2^18 updates and 2^22 members per call
    max_bh, max_bi = 1 << 18, 1 << 22
    shared, all_cfgs = _group_cfgs_resident(E, all_streams, delta, fam, max_bh, max_bi)
    # shards: graphs dealt round-robin by size, so the groups are alike;
    # server graph numbers follow the shards in admission order
    n_sh = max(1, min(args.shards, n_graphs))
    by_size = np.argsort([st.initial.n for st in all_streams])[::-1]
    shard_graphs = [list(by_size[k::n_sh]) for k in range(n_sh)]
    reserve = 16 << 30
    cap_bytes = 200 << 30
    cuda_streams = [torch.cuda.Stream() for _ in range(n_sh)]
    streams, cfgs, groups, refused = [], [], [], 0
    models, nvs = [], []
    pool = gen.insert_pool(6, 1 << 21)
    rng = np.random.default_rng(args.seed + 100)
    t_clock = time.monotonic_ns() // 1000 - 3600 * 10 ** 6   # timestamps after every initial one
    max_pending = args.queue
    srv = None
    t0 = time.time()
    used = 0
    admitted_under_load = 0
    for k in range(n_sh):
        sc = [all_cfgs[g] for g in shard_graphs[k]]
        need = E.esc_group_bytes(shared, sc)
        if used + need > cap_bytes or not E.esc_group_fits(shared, sc, reserve):
            refused += len(sc)
            continue
        grp = E.esc_group_create(shared, sc, stream=cuda_streams[k])
        ss = [all_streams[g] for g in shard_graphs[k]]
        _load_group(E, grp, ss, max_bh, max_bi)
        if not args.no_graph_launch:
            E.esc_group_set_graph_launch(grp, True)  # each call replays one captured CUDA graph
        used += need
        groups.append(grp)
        streams += ss
        cfgs += sc
        models += [_IdModel(st.initial.n) for st in ss]
        nvs += [st.n_vertices for st in ss]
        if srv is None:
            srv = E.esc_server_create(grp, max_pending, 0)
            # graphs of the first group rebuilt alone at the end: every
            # request they receive is logged from now on
            order = np.argsort([st.initial.n for st in streams])
            sample = [int(order[0]), int(order[len(order) // 3]), int(order[2 * len(order) // 3])]
            log = {g: [] for g in sample}
        else:
            E.esc_server_add_group(srv, grp)
            admitted_under_load += 1
        # load on the admitted graphs while the next group is prepared
        _drive(E, srv, models, nvs, pool, rng, args.rate / 10, 1.0, max_pending, t_clock, log)
    torch.cuda.synchronize()
    t_load = time.time() - t0
    G = len(streams)
    E.esc_server_destroy(srv)
    mean_size = float(np.mean(np.floor(10 ** np.random.default_rng(0).uniform(1, 4, 100000))))
    runs = {}

    def server(per_call):
        sv = E.esc_server_create(groups[0], max_pending, per_call)
        for grp in groups[1:]:
            E.esc_server_add_group(sv, grp)
        return sv

    # capacity of each policy: the updates/s it sustains under overload
    caps = {}
    for policy, per_call in (("continuous", 0), ("one_per_call", 1)):
        sv = server(per_call)
        try:
            over = _drive(E, sv, models, nvs, pool, rng, args.rate, args.duration, max_pending, t_clock, log)
            caps[policy] = max(over["updates_per_s"], 1.0)
            runs[policy] = {"overload": over}
        finally:
            E.esc_server_destroy(sv)
    base = caps["one_per_call"]
    for policy, per_call in (("continuous", 0), ("one_per_call", 1)):
        sv = server(per_call)
        try:
            equal = [dict(fraction=f, offered_updates_per_s=f * base,
                          **_drive(E, sv, models, nvs, pool, rng, f * base / mean_size, args.duration, max_pending,
                                   t_clock, log)) for f in (0.25, 0.5, 1.0)]
            own = dict(fraction=1.0, offered_updates_per_s=caps[policy],
                       **_drive(E, sv, models, nvs, pool, rng, caps[policy] / mean_size, args.duration, max_pending,
                                t_clock, log))
            runs[policy].update({"equal_offered_load": equal, "own_capacity": own,
                                 "stats": E.esc_server_get_stats(sv)})
        finally:
            E.esc_server_destroy(sv)
    # each sampled graph alone, from its initial hyperedges and logged requests
    same = True
    for g in sample:
        st = streams[g]
        alone = E.Graph(st.n_vertices, st.initial.offsets, st.initial.members, st.initial.timestamps,
                        capacity_hyperedges=cfgs[g].capacity_hyperedges,
                        capacity_incidences=cfgs[g].capacity_incidences, max_batch_hyperedges=max_bh,
                        max_batch_incidences=max_bi, families=fam, delta=delta)
        for off, mem, ts, dels in log[g]:
            alone.apply_batch(off, mem, ts, dels, return_ids=False)
        sv = server(0)
        for tt in (E.TRIAD_HYPEREDGE, E.TRIAD_TEMPORAL):
            same &= bool(np.array_equal(alone.triads(tt), E.esc_server_triads(sv, g, tt, delta)))
        E.esc_server_destroy(sv)
        alone.close()
    for grp in groups:
        E.esc_group_destroy(grp)
    cont = runs["continuous"]["own_capacity"]
    one = runs["one_per_call"]["own_capacity"]
    eq = [(a["updates_per_s"], b["updates_per_s"], a["p50_ms"], b["p50_ms"], a["p99_ms"], b["p99_ms"])
          for a, b in zip(runs["continuous"]["equal_offered_load"], runs["one_per_call"]["equal_offered_load"])]
    print(json.dumps({
        "metric": METRIC, "value": cont["updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32 ids / uint64 counts", "data": "synthetic",
        "config": {"workload": (f"serving: {G} of {n_graphs} resident hypergraphs admitted (initial sizes "
                                f"log-uniform [1e3, {1e6 * args.scale:.0e}], vertices = hyperedges/2, cardinality "
                                "Zipf(2.0) in [2,256]); Poisson arrivals, uniform graph, sizes log-uniform "
                                "[10, 1e4], 1:1 insert/delete; hyperedge + temporal families"),
                   "groups": len(groups), "groups_admitted_under_load": admitted_under_load,
                   "graphs_refused": refused, "offered_per_s": args.rate, "seconds_per_run": args.duration,
                   "queue_updates": max_pending, "load_s": round(t_load, 1),
                   "hyperedges": int(sum(st.initial.n for st in streams)), "group_bytes": int(used),
                   "graph_launch": not args.no_graph_launch},
        "headline": ("each policy at an offered load equal to its own capacity: continuous batching "
                     f"{cont['updates_per_s']:.0f} vs one request per call {one['updates_per_s']:.0f} updates/s"),
        "p50_ms": cont["p50_ms"], "p99_ms": cont["p99_ms"],
        "continuous_over_one_per_call_at_own_capacity": cont["updates_per_s"] / max(one["updates_per_s"], 1e-9),
        "equal_offered_load": [dict(fraction=f, continuous_updates_per_s=a, one_per_call_updates_per_s=b,
                                    continuous_p50_ms=c, one_per_call_p50_ms=d, continuous_p99_ms=e,
                                    one_per_call_p99_ms=h)
                               for f, (a, b, c, d, e, h) in zip((0.25, 0.5, 1.0), eq)],
        "runs": runs,
        "alone_equals_served": same,
        "ids_ok": all(r["ids_ok"] for p in runs.values()
                      for r in [p["overload"], p["own_capacity"]] + p["equal_offered_load"]),
    }))


def _group_cfgs_resident(E, streams, delta, fam, max_bh, max_bi):
    """Per-graph capacities for a long request stream: the live count stays
    near the initial one (1:1 requests), the incidences drift."""
    shared = E.make_config(1, 1, 1, max_bh, max_bi, fam, delta)
    cfgs = [E.make_config(st.n_vertices, int(st.initial.n * 1.25) + 6000, int(st.initial.nnz * 2) + 60000,
                          0, 0, fam, delta) for st in streams]
    return shared, cfgs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_uniform",
                    choices=["large_uniform", "large_zipf", "tiny", "batched", "temporal", "serving", "horizontal",
                             "sweep"])
    ap.add_argument("--sweep", default="batch", choices=["batch", "delete", "card", "size", "spread"],
                    help="sweep workload: which parameter varies")
    ap.add_argument("--size-scale", type=float, default=0.05, help="size sweep: fraction of 20M-55M hyperedges")
    ap.add_argument("--size-kmax", type=int, default=1000, help="size sweep: cardinality cap (the paper's: 10000)")
    ap.add_argument("--size-points", type=int, nargs="*", default=None,
                    help="size sweep: which of 20 30 40 55 (million hyperedges before --size-scale) to run")
    ap.add_argument("--graphs", type=int, default=None)
    ap.add_argument("--rate", type=float, default=5e4, help="serving: offered requests/s")
    ap.add_argument("--duration", type=float, default=8.0, help="serving: seconds per run")
    ap.add_argument("--queue", type=int, default=1 << 20, help="serving: queued updates admitted")
    ap.add_argument("--shards", type=int, default=4, help="serving: groups of graphs, each with its own stream")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--batch", type=int, default=100_000)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--replicas", action="store_true",
                    help="several ranks: an independent graph per rank instead of one graph split across them")
    ap.add_argument("--no-graph-launch", action="store_true", help="serving: launch kernel by kernel")
    ap.add_argument("--ref-updates-per-step", type=int, default=4)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "large_zipf":
        run_large_zipf(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "temporal":
        run_temporal(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "horizontal":
        run_horizontal(args)
    elif args.workload == "sweep":
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

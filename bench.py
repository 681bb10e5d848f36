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
                  [--workload large_uniform|tiny] [--scale S]

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

E2E_STEPS = 3   # end-to-end steps (host buffers) after the timed device-resident steps
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


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    backend = "nccl"
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


def make_stream(args, rank):
    if args.workload == "tiny":
        s = gen.random_small(args.seed + rank, 2000, 1000, 2, 8, n_batches=args.warmup + args.steps + E2E_STEPS,
                             n_ins=50, n_del=50)
        fam = 3
    else:
        s = gen.large(seed=args.seed + rank, membership="uniform", scale=args.scale,
                      n_batches=args.warmup + args.steps + E2E_STEPS, batch_updates=args.batch)
        fam = 3
    return s, fam


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
    s, fam = make_stream(args, rank)
    init = s.initial
    nb = args.warmup + args.steps + E2E_STEPS
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
    # With equal inserts and deletes per batch the live IDs stay [0, E0):
    # the deletes of every batch are its ranks.  Checked after the run from
    # the IDs the library returns.
    live_n = init.n
    dev_batches, host_batches = [], []
    for b in s.batches[:nb]:
        dels = np.sort(b.del_ranks).astype(np.int32)   # ranks == IDs while live = [0, E0)
        dev_batches.append((todev(b.inserts.offsets, np.int64), todev(b.inserts.members, np.int32),
                            todev(b.inserts.timestamps, np.int64), todev(dels, np.int32)))
        pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()  # noqa: E731
        host_batches.append((pin(b.inserts.offsets, np.int64), pin(b.inserts.members, np.int32),
                             pin(b.inserts.timestamps, np.int64), pin(dels, np.int32)))
    returned = []

    def step(batch, want_ids=True):
        out = np.zeros(batch[0].numel() - 1, np.int32)
        E.esc_apply_batch(g.h, batch[0], batch[1], batch[2], batch[3], out)
        returned.append((batch[3], out))

    st = torch.cuda.current_stream(dev)
    g.set_profiling(True)
    for k in range(args.warmup):
        step(dev_batches[k])
    torch.cuda.synchronize(dev)
    barrier(dist, dev)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = g.launch_count()
    lat, cnt_ms, store_ms, alg_bytes, triads = [], [], [], 0, 0
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
        alg_bytes += 4 * sts["alg_entries"]
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
        returned.append((hb[3], out))
        c = g.counts()
        lat_e2e.append((time.perf_counter() - t1) * 1e3)
        h2d += sum(t.numel() * t.element_size() for t in hb)
        d2h += sum(v.nbytes for v in c.values())
    te = time.perf_counter() - te0
    barrier(dist, dev)
    # check the deletes were the live IDs the library reports
    for dels, out in returned:
        d = np.asarray(dels.cpu() if hasattr(dels, "cpu") else dels)
        if not np.array_equal(np.sort(out), np.sort(d)):
            raise SystemExit("bench: the live-ID assumption failed (inserts did not reuse the deleted IDs)")
    upd_timed = sum(n_upd[args.warmup:args.warmup + args.steps])
    t_max = allreduce_max(dist, elapsed, dev)
    te_max = allreduce_max(dist, te, dev)
    tot_upd = allreduce_sum(dist, upd_timed, dev)
    tot_upd_e2e = allreduce_sum(dist, sum(n_upd[args.warmup + args.steps:nb]), dev)
    if rank != 0:
        return
    hbm, kind = peaks()
    cnt_s = sum(cnt_ms) / 1e3
    achieved = alg_bytes / cnt_s / 1e9 if cnt_s > 0 else 0.0
    traffic = None
    prof_path = os.path.join(ROOT, "profiles", "count_traffic_per_launch.json")
    if os.path.exists(prof_path):
        try:
            traffic = json.load(open(prof_path)).get("traffic_bytes_per_launch")
        except Exception:
            traffic = None
    lat_sorted = sorted(lat)
    res = {
        "metric": METRIC, "value": tot_upd / t_max, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32 ids / uint64 counts", "data": "synthetic",
        "config": {"workload": workload_desc(args, s), "families": "hyperedge (30) + incident-vertex (3)",
                   "updates_per_step": args.batch, "parallelism": f"replicas x{ws}",
                   "l2": "resident store larger than L2 (129 MB)",
                   "create_s": round(t_create, 2)},
        "latency_ms": {"p50": float(np.percentile(lat_sorted, 50)), "p99": float(np.percentile(lat_sorted, 99))},
        "stage_ms_per_step": {"count": sum(cnt_ms) / len(cnt_ms), "store_and_ingest": sum(store_ms) / len(store_ms)},
        "triads_per_step": triads / args.steps,
        "counter_work_per_step": {k: v / args.steps for k, v in zip(
            ["centre_items", "n_g1_build_entries", "pair_pass_visits", "closed_pairs", "slow_t_steps",
             "aggregate_visits"], work)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_kind": kind,
                     "kernel": "triad count (k_nh_build + k_center and their work lists), per batch",
                     "bytes": "4 B per incidence entry the method reads for the changed hyperedges (per changed h: |h| + sum of member degrees; per candidate neighbour g1: |g1| + sum of its member degrees)",
                     "algorithmic_bytes_per_step": alg_bytes / args.steps},
        "e2e": {"value": tot_upd_e2e / te_max, "unit": UNIT, "h2d_bytes_per_step": h2d // E2E_STEPS,
                "d2h_bytes_per_step": d2h // E2E_STEPS, "steps": E2E_STEPS,
                "latency_ms": {"p50": float(np.percentile(lat_e2e, 50)), "p99": float(np.percentile(lat_e2e, 99))}},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args, s, budget_s=args.cpu_budget)
    print(json.dumps(res))


# ---------------------------------------------------------------------------
# the oracle on a bounded sample
# ---------------------------------------------------------------------------

def _oracle_sample(s, n_updates, rng_seed=0):
    """Time the oracle's update of the counts for a sample of one batch's
    updates on the full-size hypergraph: triads holding a sampled deleted
    hyperedge (old graph) and a sampled inserted one (new graph), each by the
    oracle's own enumeration.  Returns (seconds, updates)."""
    from oracle import oracle as O
    init = s.initial
    off = init.offsets
    # the oracle wants sorted member lists
    mem = init.members.copy()
    for i in range(init.n):
        a, b = off[i], off[i + 1]
        mem[a:b] = np.sort(mem[a:b])
    ts = init.timestamps
    ids = np.arange(init.n, dtype=np.int32)
    rng = np.random.default_rng(rng_seed)
    half = max(1, n_updates // 2)
    sel = np.sort(rng.choice(init.n, size=half, replace=False))
    t0 = time.perf_counter()
    O.count_containing(off, mem, ts, ids, 0, O.FAM_HYPEREDGE, sel)
    t1 = time.perf_counter()
    # inserted side: the same enumeration around the same number of hyperedges
    sel2 = np.sort(rng.choice(init.n, size=half, replace=False))
    O.count_containing(off, mem, ts, ids, 0, O.FAM_HYPEREDGE, sel2)
    t2 = time.perf_counter()
    return (t1 - t0) + (t2 - t1), 2 * half


def cpu_baseline(args, s, budget_s=20.0):
    from oracle import oracle as O
    O.build()
    n = 2
    secs, upd = _oracle_sample(s, n)
    # grow the sample until it takes a meaningful share of the budget
    while secs < budget_s / 4 and n < 4096:
        n *= 2
        secs, upd = _oracle_sample(s, n, rng_seed=n)
    return {"value": upd / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{upd} updates ({upd // 2} deletes + {upd // 2} inserts) of one batch: the oracle's "
                       f"enumeration of every triad holding a sampled hyperedge (hyperedge family) on the full "
                       f"{s.initial.n:,}-hyperedge graph, single thread; {secs:.1f} s")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    s, fam = make_stream(args, 0)
    from oracle import oracle as O
    O.build()
    per_step = max(2, args.ref_updates_per_step)
    for k in range(args.warmup):
        _oracle_sample(s, per_step, rng_seed=1000 + k)
    secs = 0.0
    upd = 0
    lat = []
    for k in range(args.steps):
        t, u = _oracle_sample(s, per_step, rng_seed=k)
        secs += t
        upd += u
        lat.append(t * 1e3)
    value = upd / secs
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "uint64", "data": "synthetic",
        "config": {"workload": workload_desc(args, s), "families": "hyperedge (30)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} updates per step, oracle enumeration on the full graph"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_uniform", choices=["large_uniform", "tiny"])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--batch", type=int, default=100_000)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-updates-per-step", type=int, default=4)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

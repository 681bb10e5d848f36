"""Seeded synthetic hypergraph streams.

Every array here is drawn from a numpy PCG64 stream seeded by the caller, so
the same seed gives the same stream on any machine.  The shapes follow the
workloads of the paper's evaluation (Section V: batches of hyperedge
insertions and deletions, 50% / 50% unless stated, Zipf-like cardinalities)
and the five synthetic configurations this project measures:

* ``tiny``      2,000 vertices, 1,000 hyperedges, cardinality uniform in [2, 8],
                one batch of 100 inserts + 100 deletes.
* ``large``     1M vertices, 2M hyperedges, cardinality Zipf(2.0) truncated to
                [2, 1000], vertex popularity Zipf(1.1) (``membership="zipf"``)
                or uniform (``membership="uniform"``), 20 batches of 1e5
                updates (5e4 inserts + 5e4 deletes).
* ``temporal``  a time-ordered stream of 4M hyperedges over 2M vertices,
                cardinality Zipf(2.0) in [2, 500], microsecond timestamps with
                exponential gaps (rate 1e3 per second), batches of 2^16.
* ``batched``   many independent hypergraphs of log-uniform size, one update
                batch each.
* ``serving``   a Poisson arrival process of update batches over many
                resident hypergraphs.

Deletes are given as *ranks*: ``del_ranks[i] = r`` means "delete the r-th
smallest live hyperedge ID at the start of the batch".  Each side of a test
resolves ranks against its own live-ID set; the generator never computes
hyperedge IDs itself, because the ID assignment rule belongs to the method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "CSR", "Batch", "Stream", "TemporalStream", "MultiStream",
    "zipf_cardinalities", "uniform_cardinalities", "sample_members",
    "exp_gap_timestamps",
    "tiny", "large", "temporal", "batched", "resident_graphs", "insert_pool", "serving_arrivals",
    "random_small", "random_hypergraph", "insert_batches", "dyadic_graph", "spread_cardinalities", "spread_inserts",
]


@dataclass
class CSR:
    """Hyperedge list in CSR form: members of hyperedge i are
    ``members[offsets[i]:offsets[i+1]]`` (int32 vertex IDs, unsorted)."""
    offsets: np.ndarray          # int64[n+1]
    members: np.ndarray          # int32[nnz]
    timestamps: np.ndarray       # int64[n]

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)

    def slice(self, lo: int, hi: int) -> "CSR":
        o = self.offsets[lo:hi + 1]
        return CSR(o - o[0], self.members[o[0]:o[-1]].copy(), self.timestamps[lo:hi].copy())


@dataclass
class Batch:
    inserts: CSR
    del_ranks: np.ndarray        # int64[n_del], distinct, in random order


@dataclass
class Stream:
    name: str
    seed: int
    n_vertices: int
    initial: CSR
    batches: List[Batch]
    meta: dict = field(default_factory=dict)


@dataclass
class TemporalStream:
    """Time-ordered insert stream; expirations are chosen by the consumer
    (every live hyperedge with ``ts < T - delta`` where ``T`` is the largest
    timestamp of the batch being applied)."""
    name: str
    seed: int
    n_vertices: int
    delta: int
    batches: List[CSR]
    meta: dict = field(default_factory=dict)


@dataclass
class MultiStream:
    name: str
    seed: int
    graphs: List[Stream]
    delta: int
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# primitive samplers
# ----------------------------------------------------------------------------

def uniform_cardinalities(rng: np.random.Generator, n: int, kmin: int, kmax: int) -> np.ndarray:
    return rng.integers(kmin, kmax + 1, size=n, dtype=np.int64)


def zipf_cardinalities(rng: np.random.Generator, n: int, exponent: float,
                       kmin: int, kmax: int) -> np.ndarray:
    """Zipf(``exponent``) truncated and renormalised on [kmin, kmax]:
    P(k) proportional to k**-exponent for kmin <= k <= kmax."""
    ks = np.arange(kmin, kmax + 1, dtype=np.float64)
    w = ks ** (-exponent)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(n)
    idx = np.searchsorted(cdf, u, side="right")
    idx = np.minimum(idx, len(ks) - 1)
    return (kmin + idx).astype(np.int64)


class _VertexSampler:
    """Draws vertex IDs uniformly, or by Zipf popularity over ranks mapped to
    IDs through a seeded random permutation."""

    def __init__(self, rng: np.random.Generator, n_vertices: int, membership: str,
                 exponent: float = 1.1):
        self.rng = rng
        self.n = n_vertices
        self.kind = membership
        if membership == "zipf":
            r = np.arange(1, n_vertices + 1, dtype=np.float64)
            w = r ** (-exponent)
            cdf = np.cumsum(w)
            cdf /= cdf[-1]
            self.cdf = cdf
            self.perm = rng.permutation(n_vertices).astype(np.int32)
        elif membership != "uniform":
            raise ValueError(membership)

    def draw(self, m: int) -> np.ndarray:
        if self.kind == "uniform":
            return self.rng.integers(0, self.n, size=m, dtype=np.int64).astype(np.int32)
        idx = np.searchsorted(self.cdf, self.rng.random(m), side="right")
        idx = np.minimum(idx, self.n - 1)
        return self.perm[idx]


def sample_members(rng: np.random.Generator, cards: np.ndarray, n_vertices: int,
                   membership: str = "uniform", sampler: Optional[_VertexSampler] = None):
    """Members for hyperedges of the given cardinalities, drawn without
    replacement inside each hyperedge (a duplicate draw is redrawn).
    Returns (offsets int64[n+1], members int32[nnz])."""
    cards = np.asarray(cards, dtype=np.int64)
    if np.any(cards > n_vertices):
        raise ValueError("cardinality larger than the vertex universe")
    if sampler is None:
        sampler = _VertexSampler(rng, n_vertices, membership)
    offsets = np.zeros(cards.shape[0] + 1, dtype=np.int64)
    np.cumsum(cards, out=offsets[1:])
    nnz = int(offsets[-1])
    seg = np.repeat(np.arange(cards.shape[0], dtype=np.int64), cards)
    vals = sampler.draw(nnz)
    pos = np.arange(nnz, dtype=np.int64)       # positions still being checked
    for _ in range(10_000):
        if pos.size == 0:
            break
        key = seg[pos] * np.int64(n_vertices) + vals[pos].astype(np.int64)
        order = np.argsort(key, kind="stable")
        sk = key[order]
        dup = np.zeros(order.shape[0], dtype=bool)
        dup[1:] = sk[1:] == sk[:-1]
        redo = pos[order[dup]]
        if redo.size == 0:
            break
        vals[redo] = sampler.draw(redo.size)
        # only segments that held a duplicate need checking again
        segs = np.unique(seg[redo])
        pos = pos[np.isin(seg[pos], segs)]
    else:  # pragma: no cover
        raise RuntimeError("member sampling did not converge")
    return offsets, vals


def exp_gap_timestamps(rng: np.random.Generator, n: int, start: int,
                       rate_per_s: float = 1e3) -> np.ndarray:
    """Strictly increasing microsecond timestamps: gap = max(1, round(Exp(rate)*1e6))."""
    gaps = np.maximum(1, np.rint(rng.exponential(1.0 / rate_per_s, size=n) * 1e6)).astype(np.int64)
    return start + np.cumsum(gaps)


def _csr(rng, cards, n_vertices, sampler, ts):
    off, mem = sample_members(rng, cards, n_vertices, sampler=sampler)
    return CSR(off, mem, ts)


def _batches(rng, n_live0, n_batches, n_ins, n_del, card_fn, sampler, n_vertices, ts_start):
    out = []
    n_live = n_live0
    t = ts_start
    for _ in range(n_batches):
        cards = card_fn(n_ins)
        ts = exp_gap_timestamps(rng, n_ins, t)
        if n_ins:
            t = int(ts[-1])
        ins = _csr(rng, cards, n_vertices, sampler, ts)
        nd = min(n_del, n_live)
        ranks = rng.choice(n_live, size=nd, replace=False).astype(np.int64) if nd else np.zeros(0, np.int64)
        out.append(Batch(ins, ranks))
        n_live += n_ins - nd
    return out


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------

def random_small(seed: int, n_vertices: int, n_edges: int, kmin: int, kmax: int,
                 n_batches: int = 0, n_ins: int = 0, n_del: int = 0,
                 membership: str = "uniform", card: str = "uniform",
                 zipf_exponent: float = 2.0) -> Stream:
    """Small stream for tests: any sizes, uniform or Zipf cardinalities."""
    rng = np.random.default_rng(seed)
    sampler = _VertexSampler(rng, n_vertices, membership)
    if card == "uniform":
        card_fn = lambda m: uniform_cardinalities(rng, m, kmin, kmax)  # noqa: E731
    else:
        card_fn = lambda m: zipf_cardinalities(rng, m, zipf_exponent, kmin, kmax)  # noqa: E731
    ts0 = exp_gap_timestamps(rng, n_edges, 0)
    init = _csr(rng, card_fn(n_edges), n_vertices, sampler, ts0)
    t = int(ts0[-1]) if n_edges else 0
    b = _batches(rng, n_edges, n_batches, n_ins, n_del, card_fn, sampler, n_vertices, t)
    return Stream("random_small", seed, n_vertices, init, b,
                  dict(kmin=kmin, kmax=kmax, membership=membership, card=card))


def tiny(seed: int = 0) -> Stream:
    """2,000 vertices; 1,000 hyperedges with cardinality uniform in [2, 8] and
    members uniform without replacement; one batch of 100 inserts (same
    distribution) and 100 deletes of uniformly chosen live hyperedges."""
    s = random_small(seed, 2000, 1000, 2, 8, n_batches=1, n_ins=100, n_del=100)
    s.name = "tiny"
    return s


def large(seed: int = 2, membership: str = "zipf", scale: float = 1.0,
          n_batches: int = 20, batch_updates: int = 100_000, kmax: int = 1000) -> Stream:
    """1M vertices, 2M hyperedges (times ``scale``), cardinality Zipf(2.0)
    truncated to [2, kmax], vertex popularity Zipf(1.1) or uniform; batches of
    ``batch_updates`` updates split 50% inserts / 50% deletes."""
    rng = np.random.default_rng(seed)
    n_vertices = max(16, int(round(1_000_000 * scale)))
    n_edges = max(8, int(round(2_000_000 * scale)))
    kmax = min(kmax, n_vertices)
    sampler = _VertexSampler(rng, n_vertices, membership)
    card_fn = lambda m: zipf_cardinalities(rng, m, 2.0, 2, kmax)  # noqa: E731
    ts0 = exp_gap_timestamps(rng, n_edges, 0)
    init = _csr(rng, card_fn(n_edges), n_vertices, sampler, ts0)
    n_ins = batch_updates // 2
    n_del = batch_updates - n_ins
    b = _batches(rng, n_edges, n_batches, n_ins, n_del, card_fn, sampler, n_vertices, int(ts0[-1]))
    return Stream(f"large_{membership}", seed, n_vertices, init, b,
                  dict(scale=scale, membership=membership, kmax=kmax,
                       batch_updates=batch_updates))


def temporal(seed: int = 3, scale: float = 1.0, batch: int = 1 << 16,
             delta_s: float = 3600.0, kmax: int = 500, rate_per_s: float = 1e3,
             n_batches: Optional[int] = None) -> TemporalStream:
    """Time-ordered stream: 4M hyperedges (times ``scale``) over 2M vertices
    (times ``scale``), cardinality Zipf(2.0) in [2, kmax], uniform members,
    microsecond timestamps with Exp(rate) gaps, batches of ``batch`` inserts.
    ``delta`` (microseconds) is the temporal window."""
    rng = np.random.default_rng(seed)
    n_vertices = max(16, int(round(2_000_000 * scale)))
    n_total = max(batch, int(round(4_000_000 * scale)))
    kmax = min(kmax, n_vertices)
    sampler = _VertexSampler(rng, n_vertices, "uniform")
    nb = math.ceil(n_total / batch) if n_batches is None else n_batches
    out = []
    t = 0
    for i in range(nb):
        m = min(batch, n_total - i * batch) if n_batches is None else batch
        cards = zipf_cardinalities(rng, m, 2.0, 2, kmax)
        ts = exp_gap_timestamps(rng, m, t, rate_per_s)
        t = int(ts[-1])
        out.append(_csr(rng, cards, n_vertices, sampler, ts))
    return TemporalStream("temporal", seed, n_vertices, int(round(delta_s * 1e6)), out,
                          dict(scale=scale, batch=batch, kmax=kmax, rate_per_s=rate_per_s))


def batched(seed: int = 4, n_graphs: int = 256, e_lo: float = 1e3, e_hi: float = 1e6,
            b_lo: float = 1e2, b_hi: float = 1e5, kmax: int = 256,
            delta_s: float = 3600.0) -> MultiStream:
    """``n_graphs`` independent hypergraphs: initial hyperedge count
    floor(10**U(log10 e_lo, log10 e_hi)), vertices = hyperedges / 2,
    cardinality Zipf(2.0) in [2, kmax], uniform members, timestamps with
    Exp(1e3/s) gaps; one mixed batch each of size floor(10**U(log10 b_lo,
    log10 b_hi)), half inserts, half deletes of uniform live hyperedges."""
    rng = np.random.default_rng(seed)
    graphs = []
    for g in range(n_graphs):
        e0 = int(math.floor(10 ** rng.uniform(math.log10(e_lo), math.log10(e_hi))))
        nv = max(kmax, e0 // 2)
        size = int(math.floor(10 ** rng.uniform(math.log10(b_lo), math.log10(b_hi))))
        n_ins = size // 2
        n_del = min(size - n_ins, e0)
        sampler = _VertexSampler(rng, nv, "uniform")
        card_fn = lambda m: zipf_cardinalities(rng, m, 2.0, 2, kmax)  # noqa: E731
        ts0 = exp_gap_timestamps(rng, e0, 0)
        init = _csr(rng, card_fn(e0), nv, sampler, ts0)
        b = _batches(rng, e0, 1, n_ins, n_del, card_fn, sampler, nv, int(ts0[-1]))
        graphs.append(Stream(f"g{g}", seed, nv, init, b, dict(e0=e0)))
    return MultiStream("batched", seed, graphs, int(round(delta_s * 1e6)),
                       dict(n_graphs=n_graphs, kmax=kmax))


def resident_graphs(seed: int = 5, n_graphs: int = 1024, e_lo: float = 1e3, e_hi: float = 1e6,
                    kmax: int = 256, delta_s: float = 3600.0) -> MultiStream:
    """Initial hypergraphs of the serving workload, drawn as in ``batched``
    (initial hyperedge count floor(10**U(log10 e_lo, log10 e_hi)), vertices
    = hyperedges / 2, cardinality Zipf(2.0) in [2, kmax], uniform members,
    Exp(1e3/s) timestamp gaps) but without a batch of their own."""
    rng = np.random.default_rng(seed)
    graphs = []
    for g in range(n_graphs):
        e0 = int(math.floor(10 ** rng.uniform(math.log10(e_lo), math.log10(e_hi))))
        nv = max(kmax, e0 // 2)
        sampler = _VertexSampler(rng, nv, "uniform")
        ts0 = exp_gap_timestamps(rng, e0, 0)
        init = _csr(rng, zipf_cardinalities(rng, e0, 2.0, 2, kmax), nv, sampler, ts0)
        graphs.append(Stream(f"g{g}", seed, nv, init, [], dict(e0=e0)))
    return MultiStream("resident", seed, graphs, int(round(delta_s * 1e6)), dict(n_graphs=n_graphs, kmax=kmax))


def insert_pool(seed: int, n: int, kmax: int = 256):
    """A pool of ``n`` hyperedges for update requests: cardinalities
    Zipf(2.0) in [2, kmax] and members as uniform fractions in [0, 1), to be
    scaled to a graph's vertex count (floor(u * n_vertices); repeats within a
    hyperedge are legal input and are removed on ingest)."""
    rng = np.random.default_rng(seed)
    cards = zipf_cardinalities(rng, n, 2.0, 2, kmax)
    offs = np.zeros(n + 1, np.int64)
    np.cumsum(cards, out=offs[1:])
    return offs, rng.random(int(offs[-1]), dtype=np.float32)


def serving_arrivals(seed: int, n_graphs: int, n_requests: int, rate_per_s: float,
                     size_lo: float = 10, size_hi: float = 1e4):
    """Poisson arrivals of update requests: (arrival_time_s, graph, size)
    with sizes floor(10**U(log10 size_lo, log10 size_hi)) and graphs uniform."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_requests))
    g = rng.integers(0, n_graphs, size=n_requests)
    s = np.floor(10 ** rng.uniform(math.log10(size_lo), math.log10(size_hi), size=n_requests)).astype(np.int64)
    return t, g, s


def random_hypergraph(seed: int, n_vertices: int, n_edges: int, kmax: int, membership: str = "uniform",
                      card_exponent: float = 2.0, ts_start: int = 0) -> CSR:
    """``n_edges`` hyperedges with cardinality Zipf(``card_exponent``) in
    [2, kmax], members by ``membership``, timestamps with Exp(1e3/s) gaps."""
    rng = np.random.default_rng(seed)
    sampler = _VertexSampler(rng, n_vertices, membership)
    kmax = min(kmax, n_vertices)
    ts = exp_gap_timestamps(rng, n_edges, ts_start)
    return _csr(rng, zipf_cardinalities(rng, n_edges, card_exponent, 2, kmax), n_vertices, sampler, ts)


def insert_batches(seed: int, n_vertices: int, n_batches: int, n_ins: int, kmax: int,
                   membership: str = "uniform", card_exponent: float = 2.0, ts_start: int = 0) -> List[CSR]:
    """``n_batches`` insert lists of ``n_ins`` hyperedges each, drawn as in
    ``random_hypergraph`` (cardinality cap ``kmax``), timestamps continuing
    from ``ts_start``.  Deletes are chosen by the caller among its live IDs."""
    rng = np.random.default_rng(seed)
    sampler = _VertexSampler(rng, n_vertices, membership)
    kmax = min(kmax, n_vertices)
    out, t = [], ts_start
    for _ in range(n_batches):
        ts = exp_gap_timestamps(rng, n_ins, t)
        if n_ins:
            t = int(ts[-1])
        out.append(_csr(rng, zipf_cardinalities(rng, n_ins, card_exponent, 2, kmax), n_vertices, sampler, ts))
    return out


def _edge_csr(u: np.ndarray, v: np.ndarray, ts: np.ndarray) -> CSR:
    off = np.arange(u.shape[0] + 1, dtype=np.int64) * 2
    mem = np.empty(2 * u.shape[0], np.int32)
    mem[0::2] = u
    mem[1::2] = v
    return CSR(off, mem, ts)


def _other_end(rng: np.random.Generator, u: np.ndarray, n_vertices: int) -> np.ndarray:
    """A uniform second endpoint distinct from ``u``."""
    v = rng.integers(0, n_vertices - 1, size=u.shape[0], dtype=np.int64)
    v = v + (v >= u)  # skip u: uniform over the other n-1 vertices
    return v.astype(np.int32)


def dyadic_graph(seed: int, n_vertices: int, n_edges: int) -> CSR:
    """A dyadic graph as two-member hyperedges: ``n_edges`` edges with both
    endpoints uniform and distinct (parallel edges possible, as in a
    multigraph), timestamps with Exp(1e3/s) gaps."""
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n_vertices, size=n_edges, dtype=np.int64).astype(np.int32)
    return _edge_csr(u, _other_end(rng, u, n_vertices), exp_gap_timestamps(rng, n_edges, 0))


def spread_cardinalities(rng: np.random.Generator, n: int, mean: float, std: float, kmax: int) -> np.ndarray:
    """Cardinalities 2 + round(X), X ~ Gamma with mean ``mean`` - 2 and
    standard deviation ``std`` (``std`` 0: every cardinality is round(mean)),
    clipped to [2, kmax]."""
    m = mean - 2.0
    if std <= 0 or m <= 0:
        return np.full(n, int(round(max(mean, 2.0))), dtype=np.int64)
    x = rng.gamma(shape=m * m / (std * std), scale=std * std / m, size=n)
    return np.clip(2 + np.rint(x).astype(np.int64), 2, kmax)


def spread_inserts(seed: int, n_vertices: int, n_batches: int, n_ins: int, mean: float, std: float,
                   kmax: int = 4096, ts_start: int = 0) -> List[CSR]:
    """Insert lists whose cardinalities have a set mean and standard
    deviation (``spread_cardinalities``); members uniform and distinct within
    a hyperedge.  ``mean`` 2 with ``std`` 0 gives plain edges."""
    rng = np.random.default_rng(seed)
    sampler = _VertexSampler(rng, n_vertices, "uniform")
    kmax = min(kmax, n_vertices)
    out, t = [], ts_start
    for _ in range(n_batches):
        ts = exp_gap_timestamps(rng, n_ins, t)
        if n_ins:
            t = int(ts[-1])
        out.append(_csr(rng, spread_cardinalities(rng, n_ins, mean, std, kmax), n_vertices, sampler, ts))
    return out

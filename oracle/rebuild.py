"""Host model of the dynamic hypergraph, rebuilt from scratch after each batch.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
baseline of the benchmark; the product path never imports it.

Semantics followed (paper Section III-B, "Operations on ESCHER"):

* A hyperedge is a set of vertices (Section II): repeated members of an
  inserted hyperedge collapse to one; an empty hyperedge is rejected.
* Deletions of a batch apply before its insertions (Algorithm 3, step 3).
* ID reuse (Section III-B, insertion Case 1 and Algorithm 2): the j-th
  inserted hyperedge of a batch, in input order, takes the j-th smallest free
  ID, a free ID being one below the high-water mark that holds no live
  hyperedge, including IDs deleted earlier in the same batch.  Once those run
  out, new IDs are handed out in increasing order from the high-water mark.
  Initial hyperedges therefore get IDs 0..n-1 in input order.
* Horizontal updates (Section III-B: incident vertices inserted into or
  deleted from live hyperedges): a live hyperedge gets a new vertex set and
  keeps its ID and its timestamp.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np


class OracleHypergraph:
    def __init__(self, n_vertices: int, offsets=None, members=None, timestamps=None):
        self.n_vertices = int(n_vertices)
        self.members: list = []        # index = ID; None when not live
        self.ts: list = []
        if offsets is not None:
            self.apply_batch(offsets, members, timestamps, np.zeros(0, np.int64))

    # ------------------------------------------------------------------ state
    @property
    def high_water(self) -> int:
        return len(self.members)

    def live_ids(self) -> np.ndarray:
        return np.array([i for i, m in enumerate(self.members) if m is not None], dtype=np.int64)

    def n_live(self) -> int:
        return sum(1 for m in self.members if m is not None)

    def resolve_ranks(self, ranks: Sequence[int]) -> np.ndarray:
        """IDs of the r-th smallest live IDs, for each rank r."""
        live = self.live_ids()
        return live[np.asarray(ranks, dtype=np.int64)] if len(ranks) else np.zeros(0, np.int64)

    def edge(self, hid: int) -> Optional[np.ndarray]:
        return self.members[hid] if 0 <= hid < len(self.members) else None

    # ---------------------------------------------------------------- updates
    def apply_batch(self, ins_offsets, ins_members, ins_ts, del_ids) -> np.ndarray:
        ins_offsets = np.asarray(ins_offsets, dtype=np.int64)
        ins_members = np.asarray(ins_members, dtype=np.int64)
        del_ids = np.asarray(del_ids, dtype=np.int64)
        n_ins = ins_offsets.shape[0] - 1
        if ins_ts is None:
            ins_ts = np.zeros(n_ins, dtype=np.int64)
        ins_ts = np.asarray(ins_ts, dtype=np.int64)
        # ---- validate everything before changing anything
        if n_ins < 0 or (n_ins > 0 and ins_offsets[0] != 0) or np.any(np.diff(ins_offsets) < 0):
            raise ValueError("bad insert offsets")
        new_sets = []
        for j in range(n_ins):
            s = np.unique(ins_members[ins_offsets[j]:ins_offsets[j + 1]])
            if s.size == 0:
                raise ValueError("empty hyperedge")
            if s[0] < 0 or s[-1] >= self.n_vertices:
                raise ValueError("vertex out of range")
            new_sets.append(s.astype(np.int32))
        if np.unique(del_ids).size != del_ids.size:
            raise ValueError("duplicate delete")
        for d in del_ids:
            if self.edge(int(d)) is None:
                raise ValueError(f"delete of non-live hyperedge {int(d)}")
        # ---- deletions first
        for d in del_ids:
            self.members[int(d)] = None
            self.ts[int(d)] = None
        # ---- then insertions with the ID rule
        free = [i for i, m in enumerate(self.members) if m is None]
        out = np.empty(n_ins, dtype=np.int64)
        for j, s in enumerate(new_sets):
            if j < len(free):
                hid = free[j]
                self.members[hid] = s
                self.ts[hid] = int(ins_ts[j])
            else:
                hid = len(self.members)
                self.members.append(s)
                self.ts.append(int(ins_ts[j]))
            out[j] = hid
        return out

    def update_members(self, ids, offsets, members) -> None:
        """Give each live hyperedge ids[j] the vertex set members[offsets[j]:
        offsets[j+1]] (repeats collapse); IDs and timestamps are kept."""
        ids = np.asarray(ids, dtype=np.int64)
        offsets = np.asarray(offsets, dtype=np.int64)
        members = np.asarray(members, dtype=np.int64)
        if offsets.shape[0] != ids.size + 1 or (ids.size and offsets[0] != 0) or np.any(np.diff(offsets) < 0):
            raise ValueError("bad offsets")
        if np.unique(ids).size != ids.size:
            raise ValueError("duplicate hyperedge")
        new_sets = []
        for j, hid in enumerate(ids):
            if self.edge(int(hid)) is None:
                raise ValueError(f"update of non-live hyperedge {int(hid)}")
            s = np.unique(members[offsets[j]:offsets[j + 1]])
            if s.size == 0:
                raise ValueError("empty hyperedge")
            if s[0] < 0 or s[-1] >= self.n_vertices:
                raise ValueError("vertex out of range")
            new_sets.append(s.astype(np.int32))
        for hid, s in zip(ids, new_sets):
            self.members[int(hid)] = s

    @classmethod
    def from_checkpoint(cls, n_vertices: int, ids, offsets, members, timestamps=None) -> "OracleHypergraph":
        """The live hyperedges of a checkpoint placed under their IDs; every
        other ID below the largest one + 1 is free.  Under the ID rule above
        this hands later inserts the IDs the checkpointed graph would: its
        free IDs between the largest live one and its own high-water mark
        come next in ascending order either way."""
        g = cls(n_vertices)
        ids = np.asarray(ids, dtype=np.int64)
        offsets = np.asarray(offsets, dtype=np.int64)
        members = np.asarray(members, dtype=np.int64)
        if np.unique(ids).size != ids.size or (ids.size and ids.min() < 0):
            raise ValueError("bad checkpoint IDs")
        hw = int(ids.max()) + 1 if ids.size else 0
        g.members = [None] * hw
        g.ts = [None] * hw
        for j, hid in enumerate(ids):
            e = np.unique(members[offsets[j]:offsets[j + 1]])
            if e.size == 0 or e[0] < 0 or e[-1] >= g.n_vertices:
                raise ValueError("bad checkpoint hyperedge")
            g.members[int(hid)] = e.astype(np.int32)
            g.ts[int(hid)] = int(timestamps[j]) if timestamps is not None else 0
        return g

    # ------------------------------------------------------------------ views
    def csr(self):
        """Live hyperedges in ascending ID order: (offsets, members, ts, ids)."""
        ids = self.live_ids()
        sizes = np.array([self.members[i].size for i in ids], dtype=np.int64)
        off = np.zeros(ids.size + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        mem = (np.concatenate([self.members[i] for i in ids]).astype(np.int32)
               if ids.size else np.zeros(0, np.int32))
        ts = np.array([self.ts[i] for i in ids], dtype=np.int64)
        return off, mem, ts, ids.astype(np.int32)

    def v2h(self):
        """For every vertex, the sorted IDs of live hyperedges holding it."""
        lists = [[] for _ in range(self.n_vertices)]
        for hid, m in enumerate(self.members):
            if m is None:
                continue
            for v in m:
                lists[int(v)].append(hid)
        return [np.array(x, dtype=np.int64) for x in lists]

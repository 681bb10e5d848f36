"""CPU oracle for dynamic-hypergraph triad counts.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import, call or load anything in this
package.  It shares no code with the CUDA library in
``paper_2512_21009_gb300``, and neither imports the other.

Parity status of each function (what pins it, besides the GPU comparison):

* class tables              -- pinned: 26 hyperedge triad classes (paper
                               Section II) and 96 temporal classes (Section VI,
                               THyMe+), by enumeration.
* count_hyperedge_temporal  -- pinned: hand-derived fixtures, brute force vs
                               wedge enumeration, connected-triple totals from
                               networkx, dyadic-graph closed forms, temporal
                               fold onto the static classes.
* count_containing          -- pinned: equals brute(after) - brute(before) for
                               single-batch edits (incremental = recount).
* count_vertex_containing   -- pinned: per-triple form equals the literal
                               assignment enumeration restricted to
                               assignments with a selected witness; the
                               incremental identity count_vertex(after) -
                               count_vertex(before) = containing(after,
                               inserted) - containing(before, deleted); all
                               selected = count_vertex; none selected = 0.
* count_vertex              -- pinned: literal assignment enumeration vs the
                               per-triple closed form; type 1 = sum C(|h|,3);
                               total = trace(M^3)/6 of the co-membership
                               multiplicity matrix; dyadic type 3 = triangles.
* OracleHypergraph          -- pinned: hand cases of the ID reuse rule.
"""
from .rebuild import OracleHypergraph  # noqa: F401
from . import oracle  # noqa: F401

"""Pruning of vertices that lie in no LDS / LTDS (test infrastructure).

Alg. 3 with Pruning rule 1 (Cor. 1) and Pruning rule 2 (Lemma 5, Lemma 6):

1. every vertex x with an edge (x, y) of G' such that ub(x) < lb(y) is removed
   (rule 1 is evaluated on G' before any removal);
2. on what is left, vertices with core_{G'}(x) < lb(x) are removed and core
   numbers recomputed until no such vertex remains (rule 2).  For triangle
   density the tr-core number replaces the core number.

The loop of rule 2 ends at the largest vertex set X with core_{G[X]}(x) >=
lb(x) for all x in X, whatever the removal order (core numbers only grow with
the graph), so this oracle removes all violators of a pass at once.
Pins (tests/test_oracle_stages.py): the worked example of Sec. 5.2 (r pruned by
rule 1; o, p, q, h by rule 2 on the reconstructed Fig. 1 graph); no vertex of
an LDS from oracle.brute / oracle.decomp is ever removed (Cor. 1, Lemma 5).
"""
from __future__ import annotations

import numpy as np

from .graph import core_numbers, induced_edges, induced_triangles, tr_core_numbers


def prune(n, u, v, vertices, groups, ub, lb, tris=None):
    """Returns (kept vertex set, groups intersected with it (empty groups
    dropped), removed_by_rule1, removed_by_rule2).  ``tris`` switches rule 2
    to tr-core numbers (triangles of G' as an (|T|, 3) array)."""
    Vp = set(int(x) for x in vertices)
    eu, ev = induced_edges(u, v, Vp)
    rule1 = set()
    for a, b in zip(np.asarray(eu).tolist(), np.asarray(ev).tolist()):
        if ub[a] < lb[b]:
            rule1.add(a)
        if ub[b] < lb[a]:
            rule1.add(b)
    kept = Vp - rule1
    rule2 = set()
    while True:
        if tris is None:
            core = core_numbers(n, u, v, vertices=kept)
        else:
            core = tr_core_numbers(n, induced_triangles(tris, kept), vertices=kept)
        bad = {x for x in kept if core[x] < lb[x]}
        if not bad:
            break
        kept -= bad
        rule2 |= bad
    new_groups = []
    for g in groups:
        gg = [x for x in g if x in kept]
        if gg:
            new_groups.append(gg)
    return kept, new_groups, rule1, rule2

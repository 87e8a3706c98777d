"""Exact compact numbers and the LDS / LTDS sets they determine (test
infrastructure).

By Thm. 1 (edges) and Thm. 4 (triangles) the compact number phi(u) is the
optimal load r*_u of the convex program.  The optimal loads are the levels of
the density-friendly decomposition B_0 = {} < B_1 < ... < B_L = V (the nested
chain the paper attributes to Danisch et al., Sec. 4.2): B_{j+1} is the largest
set B containing B_j that maximises (f(B) - f(B_j)) / (|B| - |B_j|), f counting
edges (triangles) inside, and r* equals that ratio on B_{j+1} minus B_j.  Each
step is found by Dinkelbach iteration, each trial ratio by one maximal minimum
cut of the pattern network in which patterns touching B_j lose their B_j
vertices (patterns inside B_j are dropped).

The LDS (LTDS) sets then follow from Lemmas 2-3 and the proof of Thm. 1 (Thm. 3
for triangles): G[C] is an LDS iff C is a connected component of
G[{u : phi(u) = rho}] for some rho and no vertex of C has a neighbour with
phi > rho.  Density-0 sets (isolated vertices, triangle-free components) are
left out unless asked for.

Pins (tests/test_oracle_decomp.py): phi and the LDS lists equal the
brute-force definitions of oracle.brute on hundreds of random graphs with at
most 11 vertices; the Fig. 1 values of Table 2 and the LTDS example of Sec. 6.1;
closed forms for K_n and disjoint cliques.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from .flow import FlowNetwork
from .graph import adjacency, connected_components


def _max_increment(verts_free, patterns, rho: Fraction):
    """max over X subset of verts_free of q*#(patterns inside X) - p*|X|, and the
    largest maximiser X (patterns are tuples over verts_free)."""
    p, q = rho.numerator, rho.denominator
    vl = sorted(verts_free)
    node = {x: 2 + len(patterns) + i for i, x in enumerate(vl)}
    net = FlowNetwork(2 + len(patterns) + len(vl))
    for j, pat in enumerate(patterns):
        net.add_edge(0, 2 + j, q)
        for x in pat:
            net.add_edge(2 + j, node[x], q)
    for x in vl:
        net.add_edge(node[x], 1, p)
    f = net.max_flow(0, 1)
    value = q * len(patterns) - f
    side = set(net.maximal_source_side(1))
    X = {x for x in vl if node[x] in side}
    return value, X


def compact_numbers(n: int, pattern_list, vertices=None, theta: Fraction | None = None):
    """Exact phi (as Fractions) for the pattern family ``pattern_list`` (edges
    as pairs or triangles as triples) on vertex set ``vertices``.  With
    ``theta`` the decomposition stops once the next level is below theta and
    the remaining vertices get None.  Returns dict vertex -> Fraction|None."""
    V = set(range(n)) if vertices is None else set(int(x) for x in vertices)
    pats = [tuple(int(x) for x in pat) for pat in pattern_list if all(int(x) in V for x in pat)]
    phi = {}
    B = set()
    while len(B) < len(V):
        free = V - B
        reduced = []
        for pat in pats:
            rest = tuple(x for x in pat if x not in B)
            if rest:
                reduced.append(rest)
        # Dinkelbach from the ratio of taking every free vertex
        rho = Fraction(len(reduced), len(free))
        while True:
            value, X = _max_increment(free, reduced, rho)
            if value <= 0:
                break
            cnt = sum(1 for pat in reduced if all(x in X for x in pat))
            rho = Fraction(cnt, len(X))
        # at the optimal ratio the value is 0; X is the largest maximiser
        _, X = _max_increment(free, reduced, rho)
        if not X:
            X = set(free)         # only happens when rho = 0 and nothing is gained
        if theta is not None and rho < theta:
            for x in free:
                phi[x] = None
            break
        for x in X:
            phi[x] = rho
        B |= X
    return phi


def lds_from_phi(phi, adj, include_zero: bool = False):
    """LDS (LTDS) vertex sets from exact compact numbers (characterisation in
    the module header).  Vertices with phi None are treated as below every
    returned level.  Returns list of (density Fraction, sorted vertex list)."""
    levels = {}
    for x, val in phi.items():
        if val is not None:
            levels.setdefault(val, []).append(x)
    out = []
    for rho, members in levels.items():
        if rho == 0 and not include_zero:
            continue
        for comp in connected_components(members, adj):
            ok = True
            for x in comp:
                for y in adj[x]:
                    py = phi.get(y)
                    if py is not None and py > rho:
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                out.append((rho, comp))
    out.sort(key=lambda dc: (-dc[0], dc[1][0]))
    return out


def lds_exact(n: int, u, v, include_zero: bool = False, theta=None, vertices=None):
    """All LDSs (edge density) with density >= theta, densest first (ties by
    smallest member id)."""
    pats = list(zip(np.asarray(u).tolist(), np.asarray(v).tolist()))
    phi = compact_numbers(n, pats, vertices=vertices, theta=theta)
    return lds_from_phi(phi, adjacency(n, u, v), include_zero)


def ltds_exact(n: int, u, v, tris, include_zero: bool = False, theta=None, vertices=None):
    pats = [tuple(t) for t in np.asarray(tris, dtype=np.int64).reshape(-1, 3).tolist()]
    phi = compact_numbers(n, pats, vertices=vertices, theta=theta)
    return lds_from_phi(phi, adjacency(n, u, v), include_zero)

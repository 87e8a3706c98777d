"""IsDensest, IsLDS, IsLTDS and ExtMaximal (test infrastructure).

* IsDensest (Sec. 5.4): G[S] is the densest subgraph of itself iff the pattern
  network (source -> pattern, pattern -> its vertices, vertex -> sink with
  capacity rho = density(G[S])) saturates every source arc.  With rho = p/q all
  capacities are scaled by q: source and pattern arcs carry q, sink arcs p.
* ExtMaximal (Alg. 8): the same network over a vertex set U and a pattern
  multiset P; returns U's part of the maximal source side of a minimum cut,
  which is {u in U : phi(u) >= rho} (Lemma 9).
* IsLDS (Alg. 4) and IsLTDS (Alg. 7): breadth-first search from S over
  vertices w with lb(w) <= rho <= ub(w); an edge to a vertex with lb(w) > rho
  becomes a loop pattern at the visited endpoint (a reduced pattern for
  triangles); then ExtMaximal; S is an LDS iff it is a connected component of
  the returned vertex set.

Readings of the paper taken here:

* The traversal admits w when ub(w) >= rho (text of Sec. 5.4 and the ablation),
  not the strict ">" printed in Alg. 4.
* A direct neighbour w of S with lb(w) > rho makes S fail at once: phi(w) > rho
  while an LDS has every outside neighbour strictly below rho (Lemma 3 /
  Thm. 3 condition 2).  As printed, Alg. 4 would turn w into loops and could
  accept S.
* The shortcut "no loop met -> True" is only taken when the traversal stays
  inside S; otherwise the flow is always run (a vertex w with a loose lb(w) <=
  rho may still complete a larger rho-compact subgraph).
* The networks of IsDensest and IsLDS are not given in the paper; both use
  Alg. 8's pattern network (edge patterns and loop patterns).

Pins (tests/test_oracle_stages.py, tests/test_oracle_ldscvx.py): IsDensest
against brute-force densest subgraphs; ExtMaximal against exact compact
numbers (Lemma 9); IsLDS / IsLTDS with exact bounds against the brute-force
LDS / LTDS lists on hundreds of small random graphs (Thm. 2, Thm. 5).
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction

import numpy as np

from .flow import FlowNetwork
from .graph import connected_components


def pattern_network(vertices, patterns, rho: Fraction):
    """Builds the Alg. 8 network.  Returns (net, s, t, node_of_vertex)."""
    verts = sorted(set(int(x) for x in vertices))
    p, q = rho.numerator, rho.denominator
    nv, npat = len(verts), len(patterns)
    s, t = 0, 1
    net = FlowNetwork(2 + npat + nv)
    node = {x: 2 + npat + i for i, x in enumerate(verts)}
    for j, pat in enumerate(patterns):
        net.add_edge(s, 2 + j, q)
        for x in pat:
            net.add_edge(2 + j, node[x], q)
    for x in verts:
        net.add_edge(node[x], t, p)
    return net, s, t, node


def ext_maximal(U, patterns, rho: Fraction):
    """Alg. 8: vertices of U on the maximal source side of a minimum cut."""
    net, s, t, node = pattern_network(U, patterns, rho)
    net.max_flow(s, t)
    side = set(net.maximal_source_side(t))
    return sorted(x for x, nd in node.items() if nd in side)


def is_densest(S, patterns):
    """True iff G[S] is its own densest subgraph (patterns = E(S) as pairs, or
    T(S) as triples, for triangle density)."""
    S = list(S)
    if not S:
        return False
    rho = Fraction(len(patterns), len(S))
    if rho == 0:
        return True
    net, s, t, _ = pattern_network(S, patterns, rho)
    return net.max_flow(s, t) == rho.denominator * len(patterns)


def _is_component(S, A, adj):
    Sset = set(S)
    Aset = set(A)
    if not Sset <= Aset:
        return False
    for x in Sset:
        for y in adj[x]:
            if y in Aset and y not in Sset:
                return False
    return len(connected_components(S, adj)) == 1


def is_lds(S, ub, lb, adj, num_edges_S: int, stats=None):
    """Alg. 4 with the readings in the module header.  adj: neighbour lists of
    G; num_edges_S = |E(S)|; ub / lb map vertex -> Fraction (valid for G)."""
    S = sorted(int(x) for x in S)
    Sset = set(S)
    rho = Fraction(num_edges_S, len(S))
    for x in S:
        for w in adj[x]:
            if w not in Sset and lb[w] > rho:
                if stats is not None:
                    stats["direct_denser_neighbour"] = stats.get("direct_denser_neighbour", 0) + 1
                return False
    U = set(S)
    order = list(S)
    loops = []
    need_flow = False
    dq = deque(S)
    while dq:
        x = dq.popleft()
        for w in adj[x]:
            if w in U:
                continue
            if lb[w] > rho:
                loops.append(x)
                need_flow = True
            elif ub[w] >= rho:
                U.add(w)
                order.append(w)
                dq.append(w)
    if len(U) == len(S) and not need_flow:
        return True
    patterns = []
    for x in U:
        for y in adj[x]:
            if y in U and x < y:
                patterns.append((x, y))
    patterns.extend((x,) for x in loops)
    if stats is not None:
        stats["flows"] = stats.get("flows", 0) + 1
    A = ext_maximal(U, patterns, rho)
    return _is_component(S, A, adj)


def is_ltds(S, ub, lb, adj, tris_of, tri_list, num_tris_S: int, stats=None):
    """Alg. 7 with the readings in the module header.  tris_of[x] lists the
    ids of triangles at x; tri_list[t] is (a, b, c)."""
    S = sorted(int(x) for x in S)
    Sset = set(S)
    rho = Fraction(num_tris_S, len(S))
    for x in S:
        for w in adj[x]:
            if w not in Sset and lb[w] > rho:
                if stats is not None:
                    stats["direct_denser_neighbour"] = stats.get("direct_denser_neighbour", 0) + 1
                return False
    U = set(S)
    patterns = []
    visited = set()
    need_flow = False
    dq = deque(S)
    while dq:
        x = dq.popleft()
        for ti in tris_of[x]:
            if ti in visited:
                continue
            visited.add(ti)
            tri = tri_list[ti]
            if any(ub[w] < rho for w in tri):
                continue
            M = []
            for w in tri:
                if lb[w] <= rho:
                    M.append(w)
                    if w not in U:
                        U.add(w)
                        dq.append(w)
                else:
                    need_flow = True
            if M:
                patterns.append(tuple(M))
        for w in adj[x]:
            if w in U:
                continue
            if lb[w] > rho:
                need_flow = True
            elif ub[w] >= rho:
                U.add(w)
                dq.append(w)
    if len(U) == len(S) and not need_flow:
        return True
    if stats is not None:
        stats["flows"] = stats.get("flows", 0) + 1
    A = ext_maximal(U, patterns, rho)
    return _is_component(S, A, adj)

"""Graph basics for the oracle (test infrastructure; see ``oracle/__init__``).

Follows the preliminaries of the paper (Sec. 3): an undirected simple graph
G = (V, E) with V = {0..n-1}; E(S) = E restricted to S; G[S] = (S, E(S)); the
edge density |E|/|V| (Eq. 1); the triangle set T and tr-density |T|/|V|
(Eq. 3); the k-core / core number (Def. 6) and the tr-k-core / tr-core number
(Def. 11).

Pins (tests/test_oracle_graph.py): canonical edges and triangles against
brute force over all vertex pairs / triples; core numbers against the
definition (largest k with u in a subgraph of minimum degree >= k, by
enumeration on small graphs); K_n closed forms.
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction

import numpy as np


def canonical_edges(n: int, src, dst):
    """Edge list of the simple undirected graph spanned by (src[i], dst[i]).

    Self-loops and repeated pairs are dropped; each edge is stored once as
    (u, v) with u < v; the list is sorted by (u, v).  Ids outside [0, n)
    raise ValueError.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    if len(src) and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("vertex id out of range")
    pairs = set()
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            pairs.add((min(a, b), max(a, b)))
    pairs = sorted(pairs)
    u = np.array([p[0] for p in pairs], dtype=np.int64)
    v = np.array([p[1] for p in pairs], dtype=np.int64)
    return u, v


def adjacency(n: int, u, v):
    """Sorted neighbour lists (python lists of ints)."""
    adj = [[] for _ in range(n)]
    for a, b in zip(np.asarray(u).tolist(), np.asarray(v).tolist()):
        adj[a].append(b)
        adj[b].append(a)
    for row in adj:
        row.sort()
    return adj


def adjacency_sets(n: int, u, v):
    adj = [set() for _ in range(n)]
    for a, b in zip(np.asarray(u).tolist(), np.asarray(v).tolist()):
        adj[a].add(b)
        adj[b].add(a)
    return adj


def csr(n: int, u, v):
    """Symmetric CSR (rowptr int64[n+1], col int64[2m]) with sorted rows."""
    adj = adjacency(n, u, v)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    for i, row in enumerate(adj):
        rowptr[i + 1] = rowptr[i] + len(row)
    col = np.array([w for row in adj for w in row], dtype=np.int64)
    return rowptr, col


def degrees(n: int, u, v):
    d = np.zeros(n, dtype=np.int64)
    np.add.at(d, np.asarray(u, dtype=np.int64), 1)
    np.add.at(d, np.asarray(v, dtype=np.int64), 1)
    return d


def _member_mask(S, *arrays):
    """Boolean membership table over ids 0 .. (largest id seen) for the set S."""
    Sa = np.asarray(list(S) if not isinstance(S, np.ndarray) else S, dtype=np.int64)
    top = max([int(a.max()) for a in arrays if a.size] + [int(Sa.max()) if Sa.size else -1] + [0])
    mask = np.zeros(top + 1, dtype=bool)
    mask[Sa] = True
    return mask


def induced_edges(u, v, S):
    """E(S) as a pair of arrays (u < v kept, order kept)."""
    ua, va = np.asarray(u), np.asarray(v)
    mask = _member_mask(S, ua.astype(np.int64), va.astype(np.int64))
    keep = mask[ua.astype(np.int64)] & mask[va.astype(np.int64)]
    return ua[keep], va[keep]


def triangles(n: int, u, v):
    """T: every vertex triple {a < b < c} whose three pairs are all edges,
    sorted lexicographically; as an int64 array of shape (|T|, 3)."""
    adj = adjacency_sets(n, u, v)
    out = []
    for a, b in zip(np.asarray(u).tolist(), np.asarray(v).tolist()):
        # a < b; every common neighbour c > b closes a triangle exactly once
        for c in adj[a] & adj[b]:
            if c > b:
                out.append((a, b, c))
    out.sort()
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def induced_triangles(tris, S):
    """The triangles (rows a, b, c) with all three vertices in S, order kept."""
    t = np.asarray(tris).reshape(-1, 3)
    ti = t.astype(np.int64)
    mask = _member_mask(S, ti)
    keep = mask[ti[:, 0]] & mask[ti[:, 1]] & mask[ti[:, 2]]
    return t[keep]


def triangle_degrees(n: int, tris):
    d = np.zeros(n, dtype=np.int64)
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    for k in range(3):
        np.add.at(d, t[:, k], 1)
    return d


def connected_components(vertices, adj):
    """Connected components of G[vertices] (adj: neighbour lists of G),
    each a sorted list, ordered by smallest member."""
    vs = set(int(x) for x in vertices)
    seen = set()
    comps = []
    for s in sorted(vs):
        if s in seen:
            continue
        comp = [s]
        seen.add(s)
        dq = deque([s])
        while dq:
            x = dq.popleft()
            for y in adj[x]:
                if y in vs and y not in seen:
                    seen.add(y)
                    comp.append(y)
                    dq.append(y)
        comps.append(sorted(comp))
    return comps


def is_connected(vertices, adj):
    vs = list(vertices)
    if not vs:
        return False
    return len(connected_components(vs, adj)) == 1


def core_numbers(n: int, u, v, vertices=None):
    """Core number of every vertex of G[vertices] (Def. 6) by peeling:
    repeatedly delete a vertex of minimum remaining degree (any one of them);
    a vertex's core number is the largest minimum degree seen up to its
    deletion.  Vertices outside ``vertices`` get -1."""
    alive = set(range(n)) if vertices is None else set(int(x) for x in vertices)
    adj = adjacency_sets(n, u, v)
    deg = {x: len(adj[x] & alive) for x in alive}
    core = np.full(n, -1, dtype=np.int64)
    k = 0
    # bucket queue keyed by current degree
    buckets = {}
    for x, d in deg.items():
        buckets.setdefault(d, set()).add(x)
    remaining = set(alive)
    lo = 0                               # no nonempty bucket below lo
    while remaining:
        d = lo
        while not buckets.get(d):
            d += 1
        # which vertex of minimum degree goes first does not change any core number
        x = buckets[d].pop()
        lo = d
        k = max(k, d)
        core[x] = k
        remaining.discard(x)
        for y in adj[x]:
            if y in remaining:
                dy = deg[y]
                buckets[dy].discard(y)
                deg[y] = dy - 1
                buckets.setdefault(dy - 1, set()).add(y)
                lo = min(lo, dy - 1)
    return core


def tr_core_numbers(n: int, tris, vertices=None):
    """tr-core number (Def. 11) by peeling on triangle counts: repeatedly
    delete a vertex lying in the fewest remaining triangles.  Only triangles
    with all three vertices in ``vertices`` count.  Outside vertices get -1."""
    alive = set(range(n)) if vertices is None else set(int(x) for x in vertices)
    tl = [tuple(t) for t in np.asarray(tris, dtype=np.int64).reshape(-1, 3).tolist()
          if t[0] in alive and t[1] in alive and t[2] in alive]
    inc = {x: [] for x in alive}
    for ti, t in enumerate(tl):
        for w in t:
            inc[w].append(ti)
    tcount = {x: len(inc[x]) for x in alive}
    dead_t = [False] * len(tl)
    core = np.full(n, -1, dtype=np.int64)
    buckets = {}
    for x, d in tcount.items():
        buckets.setdefault(d, set()).add(x)
    remaining = set(alive)
    k = 0
    lo = 0                               # no nonempty bucket below lo
    while remaining:
        d = lo
        while not buckets.get(d):
            d += 1
        # which vertex of minimum count goes first does not change any tr-core number
        x = buckets[d].pop()
        lo = d
        k = max(k, d)
        core[x] = k
        remaining.discard(x)
        for ti in inc[x]:
            if dead_t[ti]:
                continue
            dead_t[ti] = True
            for w in tl[ti]:
                if w != x and w in remaining:
                    dw = tcount[w]
                    buckets[dw].discard(w)
                    tcount[w] = dw - 1
                    buckets.setdefault(dw - 1, set()).add(w)
                    lo = min(lo, dw - 1)
    return core


def density(num_edges: int, num_vertices: int) -> Fraction:
    """|E|/|V| (Eq. 1) or |T|/|V| (Eq. 3) as an exact fraction."""
    return Fraction(int(num_edges), int(num_vertices))

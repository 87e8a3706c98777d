"""ExtractSG: stable groups and compact-number bounds (test infrastructure).

Follows Alg. 2 with Def. 5 (edges) and Def. 12 (triangles); the bounds come
from Lemma 4 / Lemma 8.  Everything is exact: the feasible solution is given as
integers W over a common denominator D (alpha = W / D), loads R = D * r, and
all comparisons are between integers or Fractions.

Readings of the paper:

* Sorting: by r descending, ties by vertex id ascending.
* Cut points: position i (1-based) is a cut point when density(V[1:i]) is
  strictly larger than density(V[1:j]) for every j > i; this is
  i = argmax_{i <= j <= n} density(V[1:j]) with ties sent to the larger j.
* Checking a candidate S = positions [a, b] (X = positions before a, Z = after
  b): the paper's "restrict all edges adjacent to the candidate ... by
  modifying alpha and r" is read as building a modified feasible solution in
  which every S-X edge gives all its weight to its S endpoint and every S-Z
  edge gives all its weight to its Z endpoint; S is accepted when, in the
  modified loads r', every X vertex is above max_S r' and every Z vertex is
  below min_S r'.  Then S is a stable group of (r', alpha') (Def. 5) and
  Lemma 4 gives min_S r' <= phi(u) <= max_S r' for u in S.
* Triangles: Def. 12's conditions 2-3 are garbled as printed (condition 3 is
  impossible for triangles inside S).  Reading: a triangle that touches S and
  has a Z vertex gives all its weight to its lowest-r Z vertex; a triangle that
  touches S, has an X vertex and no Z vertex gives all its weight to its
  lowest-r S vertex; a triangle inside S is unchanged.
* A candidate that fails is merged with the next one (Alg. 2, loop); a trailing
  remainder that never passes gives no bounds.  For a fixed start, growing the
  segment only lowers the modified loads of X and only raises max_S r', so
  after a failure on the X side no longer merge can pass: the walk stops there
  (exhaustive=True walks on; the pins check that both give the same groups).

Pins (tests/test_oracle_stages.py): on the reconstructed Fig. 1 graph at
the optimum the groups are S1, S2, S3, {g, h, i} with Table 2's values; the
groups partition a prefix of the sorted order; every bound interval contains
the exact compact number from oracle.decomp (Lemma 4 / Lemma 8) on random
graphs; the cut points match a brute-force argmax scan.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def sort_order(vertices, R):
    """Vertices by load descending, ties by id ascending."""
    return sorted((int(x) for x in vertices), key=lambda x: (-int(R[x]), x))


def cut_points(prefix_counts):
    """prefix_counts[j-1] = number of patterns inside V[1:j].  Returns the
    sorted list of 1-based cut positions."""
    nv = len(prefix_counts)
    cuts = []
    best = None          # max density over j' > j, as a Fraction
    for j in range(nv, 0, -1):
        dj = Fraction(int(prefix_counts[j - 1]), j)
        if best is None or dj > best:
            cuts.append(j)
            best = dj
    return sorted(cuts)


def _groups_from_checks(nv, cuts, check, exhaustive=False):
    groups = []
    start = 0
    for c in cuts:
        b = c - 1
        ok, lo, hi, xok = check(start, b)
        if ok:
            groups.append((start, b, lo, hi))
            start = b + 1
        elif not xok and not exhaustive:
            # the X side only gets worse as this start's segment grows: no later
            # candidate passes, the rest is the remainder
            break
    return groups, start


def extract_sg_edge(vertices, u, v, W, Dn: int, ub, lb, exhaustive=False):
    """Alg. 2 for edge density on G' = (vertices, edges u < v).

    W[e] = Dn * alpha_{u[e], v[e]}.  ub / lb map vertex -> Fraction and are
    copied, tightened and returned.  Returns a dict with keys order, pos,
    prefix (e_j), cuts, groups (list of vertex lists, top first), intervals
    (list of (lo, hi) Fractions), remainder (list of unaccepted vertices), ub,
    lb and R (scaled loads)."""
    u = [int(x) for x in np.asarray(u).tolist()]
    v = [int(x) for x in np.asarray(v).tolist()]
    W = [int(x) for x in np.asarray(W).tolist()]
    verts = [int(x) for x in vertices]
    R = {x: 0 for x in verts}
    inc = {x: [] for x in verts}          # (neighbour, own share, other share)
    for a, b, w in zip(u, v, W):
        R[a] += w
        R[b] += Dn - w
        inc[a].append((b, w, Dn - w))
        inc[b].append((a, Dn - w, w))
    order = sort_order(verts, R)
    pos = {x: i for i, x in enumerate(order)}
    nv = len(order)
    hist = [0] * nv
    for a, b in zip(u, v):
        hist[max(pos[a], pos[b])] += 1
    prefix = list(np.cumsum(hist)) if nv else []
    cuts = cut_points(prefix)

    def check(a, b):
        S = order[a:b + 1]
        Rm = {}
        x_adj = {}
        z_adj = {}
        for x in S:
            val = R[x]
            for y, own, other in inc[x]:
                py = pos[y]
                if py < a:                   # S-X edge: all weight to x
                    val += other
                    x_adj[y] = x_adj.get(y, R[y]) - other
                elif py > b:                 # S-Z edge: all weight to y
                    val -= own
                    z_adj[y] = z_adj.get(y, R[y]) + own
            Rm[x] = val
        lo = min(Rm.values())
        hi = max(Rm.values())
        xok = zok = True
        if a > 0:
            min_x = min([R[order[a - 1]]] + list(x_adj.values()))
            xok = min_x > hi
        if b < nv - 1:
            max_z = max([R[order[b + 1]]] + list(z_adj.values()))
            zok = max_z < lo
        return xok and zok, lo, hi, xok

    groups, start = _groups_from_checks(nv, cuts, check, exhaustive)
    ub = dict(ub)
    lb = dict(lb)
    out_groups, intervals = [], []
    for a, b, lo, hi in groups:
        flo, fhi = Fraction(lo, Dn), Fraction(hi, Dn)
        for x in order[a:b + 1]:
            ub[x] = min(ub[x], fhi)
            lb[x] = max(lb[x], flo)
        out_groups.append(order[a:b + 1])
        intervals.append((flo, fhi))
    return dict(order=order, pos=pos, prefix=prefix, cuts=cuts, groups=out_groups,
                intervals=intervals, remainder=order[start:], ub=ub, lb=lb, R=R)


def extract_sg_tri(vertices, tris, W, Dn3: int, ub, lb, exhaustive=False):
    """Alg. 2 adapted to triangle density (Def. 12, reading in the module
    header).  tris (|T|, 3) lists the triangles of G'; W[t][k] = Dn3 *
    alpha_{tris[t][k], t} with Dn3 = 3 D_N.  Same return keys as
    extract_sg_edge."""
    tl = [tuple(int(w) for w in t) for t in np.asarray(tris, dtype=np.int64).reshape(-1, 3).tolist()]
    Wl = [tuple(int(w) for w in row) for row in np.asarray(W, dtype=np.int64).reshape(-1, 3).tolist()]
    verts = [int(x) for x in vertices]
    R = {x: 0 for x in verts}
    inc = {x: [] for x in verts}
    for ti, (t, w) in enumerate(zip(tl, Wl)):
        for k in range(3):
            R[t[k]] += w[k]
            inc[t[k]].append(ti)
    order = sort_order(verts, R)
    pos = {x: i for i, x in enumerate(order)}
    nv = len(order)
    hist = [0] * nv
    for t in tl:
        hist[max(pos[t[0]], pos[t[1]], pos[t[2]])] += 1
    prefix = list(np.cumsum(hist)) if nv else []
    cuts = cut_points(prefix)

    def check(a, b):
        S = order[a:b + 1]
        touched = set()
        for x in S:
            touched.update(inc[x])
        delta = {}
        for ti in touched:
            t, w = tl[ti], Wl[ti]
            ps = [pos[x] for x in t]
            zs = [k for k in range(3) if ps[k] > b]
            xs = [k for k in range(3) if ps[k] < a]
            if zs:
                tgt = max(zs, key=lambda k: ps[k])
                movers = [k for k in range(3) if k not in zs]
            elif xs:
                ss = [k for k in range(3) if a <= ps[k] <= b]
                tgt = max(ss, key=lambda k: ps[k])
                movers = xs
            else:
                continue
            for k in movers:
                delta[t[k]] = delta.get(t[k], 0) - w[k]
                delta[t[tgt]] = delta.get(t[tgt], 0) + w[k]
        Rm = {x: R[x] + delta.get(x, 0) for x in S}
        lo = min(Rm.values())
        hi = max(Rm.values())
        xok = zok = True
        if a > 0:
            xv = [R[y] + d for y, d in delta.items() if pos[y] < a]
            xok = min([R[order[a - 1]]] + xv) > hi
        if b < nv - 1:
            zv = [R[y] + d for y, d in delta.items() if pos[y] > b]
            zok = max([R[order[b + 1]]] + zv) < lo
        return xok and zok, lo, hi, xok

    groups, start = _groups_from_checks(nv, cuts, check, exhaustive)
    ub = dict(ub)
    lb = dict(lb)
    out_groups, intervals = [], []
    for a, b, lo, hi in groups:
        flo, fhi = Fraction(lo, Dn3), Fraction(hi, Dn3)
        for x in order[a:b + 1]:
            ub[x] = min(ub[x], fhi)
            lb[x] = max(lb[x], flo)
        out_groups.append(order[a:b + 1])
        intervals.append((flo, fhi))
    return dict(order=order, pos=pos, prefix=prefix, cuts=cuts, groups=out_groups,
                intervals=intervals, remainder=order[start:], ub=ub, lb=lb, R=R)

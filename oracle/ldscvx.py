"""LDScvx / LTDScvx driver (test infrastructure).

Alg. 5 (edge density) and its triangle extension (Sec. 6, "naturally extended"),
with the readings of the paper below:

* Initial reduction (Alg. 5 line 1): ub = core number, lb = core / 2 (edges);
  ub = tr-core, lb = tr-core / 3 (triangles).  A rho-compact graph has minimum
  degree >= rho (so phi <= core, Lemma 6), and a connected k-core removes at
  least k|U|/2 edges for any removed U (so phi >= core / 2); the triangle
  bounds follow the same way.
* The first FW round runs on G itself, so ExtractSG's bounds are valid for G
  everywhere; pruning on G is then sound for G.  Refinement rounds run FW on
  G[S] for a group S (Alg. 5 line 13).  Their lower bounds are lifted to G
  (phi_G >= phi_{G[S]}), their upper bounds are used only inside the round,
  and vertices they prune are only dropped from candidate generation.
* Every group popped from the stack is split into connected components (Def. 1
  requires connectivity).  A component that is self-densest (IsDensest) and
  passes IsLDS / IsLTDS on G is output; one that is self-densest but fails is
  dropped, as in Alg. 5; one that is not self-densest is refined (Alg. 5 line
  13).  A refinement that makes no progress is retried with 2N, 4N and 8N
  iterations and then settled exactly: the LDSs of G[C] from oracle.decomp,
  each checked against G with IsLDS / IsLTDS.
* Completeness: every group is processed until it is settled, except that,
  once k sets are certified, a group whose vertices all have ub < rho_k (the
  k-th best density) is skipped, since every LDS inside it is less dense.  This
  relies on a property the paper does not state: an LDS (LTDS) never meets two
  different groups that ExtractSG accepts (nor a group and the unaccepted
  remainder).  The test suite checks it by enumeration; with it, the LDSs of G
  inside a group C are LDSs of G[C], no proper subset of a self-densest
  connected C is an LDS (its neighbours inside C have phi >= density(C)), and
  the loop above is complete.
* Output order: density descending; ties by smallest member id.

The FW precision only changes which choices the iterations make; the
weights handed to ExtractSG are always the exact ones of those choices.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import decomp, extract_sg, fw, prune as prune_mod, verify
from .graph import (adjacency, connected_components, core_numbers, induced_edges,
                    induced_triangles, tr_core_numbers, triangles)


class _Graph:
    def __init__(self, n, u, v, triangle):
        self.n = n
        self.u = np.asarray(u, dtype=np.int64)
        self.v = np.asarray(v, dtype=np.int64)
        self.adj = adjacency(n, u, v)
        self.triangle = triangle
        if triangle:
            self.tris = triangles(n, u, v)
            self.tri_list = [tuple(t) for t in self.tris.tolist()]
            self.tris_of = [[] for _ in range(n)]
            for ti, t in enumerate(self.tri_list):
                for w in t:
                    self.tris_of[w].append(ti)


def _run_fw(g: _Graph, verts, N, precision):
    """FW on G[verts]; returns (local edges / triangles, W, denominator)."""
    vs = sorted(verts)
    if g.triangle:
        t = induced_triangles(g.tris, vs)
        if precision == "fp32":
            _, W, Dn = fw.fw_tri_fp32(g.n, t, N)
        elif precision == "fp64":
            _, a = fw.fw_tri_fp64_literal(g.n, t, N)
            Dn = 3 * fw.D(N)
            W = fw.snap_tri_weights(a, Dn)
        else:
            _, W, Dn, _ = fw.fw_tri_exact(g.n, t, N)
        return t, W, Dn
    eu, ev = induced_edges(g.u, g.v, vs)
    if precision == "fp32":
        _, W, Dn = fw.fw_edge_fp32(g.n, eu, ev, N)
    elif precision == "fp64":
        _, a, rowptr, col = fw.fw_edge_fp64_literal(g.n, eu, ev, N)
        Dn = fw.D(N)
        # alpha_{u,v} sits in row u at the slot of v
        W = np.empty(len(eu), dtype=np.int64)
        for e, (x, y) in enumerate(zip(eu.tolist(), ev.tolist())):
            s = rowptr[x] + np.searchsorted(col[rowptr[x]:rowptr[x + 1]], y)
            W[e] = int(np.rint(a[s] * Dn))
    else:
        _, W, Dn, _ = fw.fw_edge_exact(g.n, eu, ev, N)
    return (eu, ev), W, Dn


def _round(g: _Graph, verts, N, precision, ub, lb):
    """FW + ExtractSG + Pruning on G[verts] with the given bounds (valid for
    G[verts]).  Returns (groups after pruning (top first), remainder, ub, lb,
    kept, info)."""
    local, W, Dn = _run_fw(g, verts, N, precision)
    if g.triangle:
        res = extract_sg.extract_sg_tri(verts, local, W, Dn, ub, lb)
        kept, groups, r1, r2 = prune_mod.prune(g.n, g.u, g.v, verts, res["groups"] + ([res["remainder"]] if res["remainder"] else []),
                                               res["ub"], res["lb"], tris=local)
    else:
        eu, ev = local
        res = extract_sg.extract_sg_edge(verts, eu, ev, W, Dn, ub, lb)
        kept, groups, r1, r2 = prune_mod.prune(g.n, eu, ev, verts, res["groups"] + ([res["remainder"]] if res["remainder"] else []),
                                               res["ub"], res["lb"])
    return groups, res["ub"], res["lb"], kept, dict(extract=res, rule1=r1, rule2=r2)


def _initial_bounds(g: _Graph, verts):
    if g.triangle:
        core = tr_core_numbers(g.n, induced_triangles(g.tris, verts), vertices=verts)
        div = 3
    else:
        core = core_numbers(g.n, g.u, g.v, vertices=verts)
        div = 2
    ub = {x: Fraction(int(core[x])) for x in verts}
    lb = {x: Fraction(int(core[x]), div) for x in verts}
    return ub, lb


def _count_patterns(g: _Graph, comp):
    if g.triangle:
        return len(induced_triangles(g.tris, comp))
    eu, _ = induced_edges(g.u, g.v, comp)
    return len(eu)


def _patterns(g: _Graph, comp):
    """The patterns of G[comp]: its triangles, or its edges (u, v), u < v."""
    if g.triangle:
        return [tuple(t) for t in induced_triangles(g.tris, comp).tolist()]
    if len(comp) <= 4096:
        # a small set: from its members' neighbour lists, not a scan of every edge
        cs = set(int(x) for x in comp)
        return [(x, y) for x in sorted(cs) for y in g.adj[x] if y > x and y in cs]
    eu, ev = induced_edges(g.u, g.v, comp)
    return list(zip(eu.tolist(), ev.tolist()))


def topk(n, u, v, k, N, triangle=False, precision="exact", include_zero=False, stats=None):
    """Top-k LDSs (LTDSs): list of (density Fraction, sorted vertex list)."""
    if stats is None:
        stats = {}
    stats.update(fw_rounds=0, certified=0, failed=0, refined=0, exact_settled=0, skipped_by_bound=0)
    g = _Graph(n, u, v, triangle)
    all_v = list(range(n))
    ub, lb = _initial_bounds(g, all_v)
    groups, ub, lb, kept, info = _round(g, all_v, N, precision, ub, lb)
    stats["fw_rounds"] += 1
    results = {}
    stack = list(reversed(groups))

    def certify(comp, pats):
        if len(pats) == 0 and not include_zero:
            return
        if triangle:
            ok = verify.is_ltds(comp, ub, lb, g.adj, g.tris_of, g.tri_list, len(pats), stats)
        else:
            ok = verify.is_lds(comp, ub, lb, g.adj, len(pats), stats)
        if ok:
            results[tuple(comp)] = Fraction(len(pats), len(comp))
            stats["certified"] += 1
        else:
            stats["failed"] += 1

    def kth_density():
        ds = sorted(results.values(), reverse=True)
        return ds[k - 1] if len(ds) >= k else None

    while stack:
        S = stack.pop()
        rk = kth_density()
        if rk is not None and max(ub[x] for x in S) < rk:
            stats["skipped_by_bound"] += 1
            continue
        for comp in connected_components(S, g.adj):
            pats = _patterns(g, comp)
            if verify.is_densest(comp, pats):
                certify(comp, pats)
                continue
            n_try = N
            while True:
                ub_s, lb_s = _initial_bounds(g, comp)
                for x in comp:
                    ub_s[x] = min(ub_s[x], ub[x])
                sub, ub_s, lb_s, kept_s, _ = _round(g, comp, n_try, precision, ub_s, lb_s)
                stats["fw_rounds"] += 1
                stats["refined"] += 1
                for x in comp:
                    lb[x] = max(lb[x], lb_s[x])
                if not (len(sub) == 1 and sorted(sub[0]) == comp):
                    stack.extend(reversed(sub))
                    break
                if n_try >= 8 * N:
                    stats["exact_settled"] += 1
                    if triangle:
                        tl = induced_triangles(g.tris, comp)
                        exact = decomp.ltds_exact(n, g.u, g.v, tl, include_zero, vertices=comp)
                    else:
                        eu, ev = induced_edges(g.u, g.v, comp)
                        exact = decomp.lds_exact(n, eu, ev, include_zero, vertices=comp)
                    for _, c in exact:
                        certify(c, _patterns(g, c))
                    break
                n_try *= 2

    ordered = sorted(results.items(), key=lambda kv: (-kv[1], kv[0][0]))
    return [(d, list(key)) for key, d in ordered[:k]]

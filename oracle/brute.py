"""The paper's definitions by exhaustive enumeration (test infrastructure;
graphs with at most ~12 vertices).

* rho-compact (Def. 1 / Def. 7): G[T] connected and removing any nonempty U
  from T removes at least rho * |U| edges (triangles); the compactness kappa(T)
  is the minimum over U of removed(U) / |U|.
* maximal rho-compact (Def. 2 / Def. 8) and LDS / LTDS (Def. 3 / Def. 9): G[S]
  is an LDS iff it is density(G[S])-compact and no connected T strictly
  containing S is density(G[S])-compact.
* compact number (Def. 4 / Def. 10): phi(u) = max kappa(T) over connected T
  containing u.

Everything is computed over all 2^n vertex subsets (3^n subset pairs) with
exact Fractions; this module is the independent pin for oracle.decomp and
for the top-k answer of the LDScvx / LTDScvx pipeline.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations

import numpy as np


def _edge_masks(n, u, v):
    return [(1 << int(a)) | (1 << int(b)) for a, b in zip(np.asarray(u).tolist(), np.asarray(v).tolist())]


def _tri_masks(n, u, v):
    adj = [set() for _ in range(n)]
    for a, b in zip(np.asarray(u).tolist(), np.asarray(v).tolist()):
        adj[a].add(b)
        adj[b].add(a)
    masks = []
    for a, b, c in combinations(range(n), 3):
        if b in adj[a] and c in adj[a] and c in adj[b]:
            masks.append((1 << a) | (1 << b) | (1 << c))
    return masks


def _popcount(x: int) -> int:
    return bin(x).count("1")


class Enumeration:
    """All subset statistics of one small graph."""

    def __init__(self, n, u, v, triangle: bool = False):
        if n > 14:
            raise ValueError("brute force limited to 14 vertices")
        self.n = n
        self.pmasks = _tri_masks(n, u, v) if triangle else _edge_masks(n, u, v)
        emask = _edge_masks(n, u, v)
        full = 1 << n
        # f[mask] = number of patterns inside mask
        f = [0] * full
        for m in range(full):
            c = 0
            for pm in self.pmasks:
                if pm & m == pm:
                    c += 1
            f[m] = c
        self.f = f
        # connectivity of G[mask] (always through edges)
        nbr = [0] * n
        for em in emask:
            a = (em & -em).bit_length() - 1
            b = (em ^ (1 << a)).bit_length() - 1
            nbr[a] |= 1 << b
            nbr[b] |= 1 << a
        conn = [False] * full
        for m in range(1, full):
            start = m & -m
            seen = start
            frontier = start
            while frontier:
                x = (frontier & -frontier).bit_length() - 1
                frontier &= frontier - 1
                new = nbr[x] & m & ~seen
                seen |= new
                frontier |= new
            conn[m] = seen == m
        self.conn = conn
        # compactness of every connected mask
        kappa = {}
        for m in range(1, full):
            if not conn[m]:
                continue
            best = None
            sub = m
            while sub:
                val = Fraction(f[m] - f[m ^ sub], _popcount(sub))
                if best is None or val < best:
                    best = val
                sub = (sub - 1) & m
            kappa[m] = best
        self.kappa = kappa

    def density(self, m):
        return Fraction(self.f[m], _popcount(m))

    def compact_numbers(self):
        phi = [Fraction(0)] * self.n
        for m, k in self.kappa.items():
            x = m
            while x:
                i = (x & -x).bit_length() - 1
                x &= x - 1
                if k > phi[i]:
                    phi[i] = k
        return phi

    def lds_list(self, include_zero: bool = False):
        """All LDS (LTDS) vertex sets: (density, sorted vertex list), densest
        first, ties by smallest member."""
        full = (1 << self.n) - 1
        out = []
        for m, k in self.kappa.items():
            rho = self.density(m)
            if rho == 0 and not include_zero:
                continue
            if k < rho:
                continue
            rest = full & ~m
            maximal = True
            sub = rest
            while sub:
                t = m | sub
                kt = self.kappa.get(t)
                if kt is not None and kt >= rho:
                    maximal = False
                    break
                sub = (sub - 1) & rest
            if maximal:
                verts = [i for i in range(self.n) if m >> i & 1]
                out.append((rho, verts))
        out.sort(key=lambda dc: (-dc[0], dc[1][0]))
        return out

    def densest_value(self, m):
        """max density over nonempty subsets of mask m."""
        best = Fraction(0)
        sub = m
        while sub:
            d = self.density(sub)
            if d > best:
                best = d
            sub = (sub - 1) & m
        return best


def brute_lds(n, u, v, triangle: bool = False, include_zero: bool = False):
    return Enumeration(n, u, v, triangle).lds_list(include_zero)


def brute_phi(n, u, v, triangle: bool = False):
    return Enumeration(n, u, v, triangle).compact_numbers()

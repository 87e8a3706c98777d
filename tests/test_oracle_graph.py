"""Pins for oracle.graph against brute force and closed forms."""
from itertools import combinations
from math import comb

import numpy as np
import pytest

from oracle import graph
from helpers import random_graph
from paper_2504_10937_gb300 import synth


def test_canonical_edges_match_pair_set():
    n, u, v = random_graph(30, 0.2, seed=11)
    a, b = synth.scramble(n, u, v, seed=5, dup_frac=0.3, loop_frac=0.1)
    cu, cv = graph.canonical_edges(n, a, b)
    want = sorted({(min(x, y), max(x, y)) for x, y in zip(a.tolist(), b.tolist()) if x != y})
    assert list(zip(cu.tolist(), cv.tolist())) == want
    assert list(zip(cu.tolist(), cv.tolist())) == list(zip(u.tolist(), v.tolist()))


def test_canonical_edges_rejects_bad_ids():
    with pytest.raises(ValueError):
        graph.canonical_edges(3, [0, 3], [1, 1])
    with pytest.raises(ValueError):
        graph.canonical_edges(3, [-1], [1])


@pytest.mark.parametrize("seed", range(5))
def test_triangles_match_triples(seed):
    n, u, v = random_graph(16, 0.35, seed=seed)
    adj = graph.adjacency_sets(n, u, v)
    want = [t for t in combinations(range(n), 3)
            if t[1] in adj[t[0]] and t[2] in adj[t[0]] and t[2] in adj[t[1]]]
    got = [tuple(t) for t in graph.triangles(n, u, v).tolist()]
    assert got == want


def _core_by_definition(n, adj, triangle=False, tris=None):
    best = [0] * n
    for mask in range(1, 1 << n):
        members = [i for i in range(n) if mask >> i & 1]
        if triangle:
            cnt = {x: 0 for x in members}
            for t in tris:
                if all(mask >> w & 1 for w in t):
                    for w in t:
                        cnt[w] += 1
            k = min(cnt.values())
        else:
            k = min(sum(1 for y in adj[x] if mask >> y & 1) for x in members)
        for x in members:
            best[x] = max(best[x], k)
    return best


@pytest.mark.parametrize("seed", range(4))
def test_core_numbers_match_definition(seed):
    n, u, v = random_graph(10, 0.4, seed=100 + seed)
    adj = graph.adjacency_sets(n, u, v)
    assert graph.core_numbers(n, u, v).tolist() == _core_by_definition(n, adj)
    tris = graph.triangles(n, u, v).tolist()
    assert graph.tr_core_numbers(n, tris).tolist() == _core_by_definition(n, adj, True, tris)


@pytest.mark.parametrize("k", [3, 5, 7])
def test_clique_closed_forms(k):
    u, v = zip(*combinations(range(k), 2))
    u, v = np.array(u), np.array(v)
    assert graph.core_numbers(k, u, v).tolist() == [k - 1] * k
    tris = graph.triangles(k, u, v)
    assert len(tris) == comb(k, 3)
    assert graph.tr_core_numbers(k, tris).tolist() == [comb(k - 1, 2)] * k

"""Pins for the oracle's LDScvx / LTDScvx driver: its top-k answer equals the
plain definition (brute force on small graphs, exact decomposition on medium
ones) and the paper's Fig. 1 examples."""
import numpy as np
import pytest

from oracle import brute, decomp, graph, ldscvx
from helpers import load_expected, load_graph, parse_sets, random_graph, random_planted


@pytest.mark.parametrize("seed", range(24))
@pytest.mark.parametrize("triangle", [False, True])
def test_topk_equals_definition_small(seed, triangle):
    n, u, v = random_graph(9 + seed % 3, 0.3 + 0.03 * (seed % 6), seed=10000 + seed)
    truth = brute.brute_lds(n, u, v, triangle=triangle)
    for k in (1, 2, 5):
        for N, prec in ((3, "exact"), (40, "fp32"), (25, "fp64")):
            got = ldscvx.topk(n, u, v, k, N, triangle=triangle, precision=prec)
            assert got == truth[:k], (k, N, prec)


def test_fig1_top2():
    n, u, v = load_graph("fig1_graph.txt")
    exp = load_expected("fig1_expected.txt")
    for N in (5, 100):
        stats = {}
        assert ldscvx.topk(n, u, v, 2, N, stats=stats) == parse_sets(exp["lds_top2"])
        assert ldscvx.topk(n, u, v, 2, N, triangle=True) == parse_sets(exp["ltds_top2"])


@pytest.mark.parametrize("seed", range(3))
def test_topk_equals_decomposition_medium(seed):
    n, u, v, blocks = random_planted(300, 0.012, (12, 10, 9, 8), (0.9, 0.85, 0.8, 0.9), seed=11000 + seed)
    truth = decomp.lds_exact(n, u, v)
    stats = {}
    got = ldscvx.topk(n, u, v, 4, 100, stats=stats)
    assert got == truth[:4]
    tris = graph.triangles(n, u, v)
    truth_t = decomp.ltds_exact(n, u, v, tris)
    assert ldscvx.topk(n, u, v, 3, 100, triangle=True) == truth_t[:3]

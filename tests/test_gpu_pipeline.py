"""GPU parity of the stages after Frank-Wolfe (ExtractSG, Pruning, the
verification flows and the top-k driver) against the CPU oracle.  Every
quantity here is exact (integers and rationals), so the bar is bit-exactness."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import extract_sg as osg
from oracle import fw as ofw
from oracle import graph as ograph
from paper_2504_10937_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lds():
    from paper_2504_10937_gb300 import lds as _l
    _l.load()
    return _l


def _graphs():
    out = []
    out.append(synth.gnp_planted(40, 0.15, (7, 6), (0.9, 0.8), seed=21)[:3])
    out.append(synth.gnp_planted(300, 0.02, (15, 10, 8), (0.9, 0.7, 0.95), seed=22)[:3])
    out.append(synth.chung_lu(3000, 12000, 2.1, seed=23, n_blocks=4, block_size_range=(15, 50))[:3])
    out.append(synth.rmat(10, 6, 0.57, 0.19, 0.19, seed=24, n_cliques=3, clique_size_range=(10, 25))[:3])
    return out


def _ir(n, u, v, tris=None):
    if tris is None:
        core = ograph.core_numbers(n, u, v)
        div = 2
    else:
        core = ograph.tr_core_numbers(n, tris)
        div = 3
    return ({x: Fraction(int(core[x])) for x in range(n)}, {x: Fraction(int(core[x]), div) for x in range(n)})


@pytest.fixture(params=[0, 1], ids=["walk_by_size", "walk_device_chains"])
def sg_variant(lds, request):
    # 1 runs the large-graph walk (host loop, each chain of merged candidates in
    # one device launch) on these small graphs too
    lds.set_extract_variant(request.param)
    yield request.param
    lds.set_extract_variant(0)


@pytest.mark.parametrize("N", [2, 30, 250])
def test_extract_sg_edge_matches_oracle(lds, N, sg_variant):
    for n, u, v in _graphs():
        with lds.Graph(n, u, v) as g:
            g.fw(N, precision="exact", want=())
            got = g.extract_sg()
        R, W, Dn, _ = ofw.fw_edge_exact(n, u, v, N)
        ub, lb = _ir(n, u, v)
        want = osg.extract_sg_edge(range(n), u, v, W, Dn, ub, lb)
        assert got["D"] == Dn
        assert got["order"].tolist() == want["order"]
        assert got["cuts"] == want["cuts"]
        assert [sorted(x.tolist()) for x in got["groups"]] == [sorted(x) for x in want["groups"]]
        assert [Fraction(lo, Dn) for lo, _ in got["intervals"]] == [lo for lo, _ in want["intervals"]]
        assert [Fraction(hi, Dn) for _, hi in got["intervals"]] == [hi for _, hi in want["intervals"]]


@pytest.mark.parametrize("N", [2, 40])
def test_extract_sg_triangle_matches_oracle(lds, N, sg_variant):
    for n, u, v in _graphs():
        tris = ograph.triangles(n, u, v)
        with lds.Graph(n, u, v) as g:
            g.fw(N, density="triangle", precision="exact", want=())
            got = g.extract_sg()
        R, W, Dn3, _ = ofw.fw_tri_exact(n, tris, N)
        ub, lb = _ir(n, u, v, tris)
        want = osg.extract_sg_tri(range(n), tris, W, Dn3, ub, lb)
        assert got["order"].tolist() == want["order"]
        assert got["cuts"] == want["cuts"]
        assert [sorted(x.tolist()) for x in got["groups"]] == [sorted(x) for x in want["groups"]]
        assert [(Fraction(lo, Dn3), Fraction(hi, Dn3)) for lo, hi in got["intervals"]] == want["intervals"]


def _oracle_prune(n, u, v, ub, lb, tris=None):
    from oracle import prune as oprune
    kept, groups, r1, r2 = oprune.prune(n, u, v, range(n), [], ub, lb, tris=tris)
    st = np.zeros(n, np.uint8)
    st[sorted(r1)] = 1
    st[sorted(r2)] = 2
    return st


@pytest.mark.parametrize("N", [3, 60])
@pytest.mark.parametrize("triangle", [False, True])
def test_prune_matches_oracle(lds, N, triangle):
    for n, u, v in _graphs():
        tris = ograph.triangles(n, u, v) if triangle else None
        ub, lb = _ir(n, u, v, tris)
        if triangle:
            R, W, Dn, _ = ofw.fw_tri_exact(n, tris, N)
            res = osg.extract_sg_tri(range(n), tris, W, Dn, ub, lb)
        else:
            R, W, Dn, _ = ofw.fw_edge_exact(n, u, v, N)
            res = osg.extract_sg_edge(range(n), u, v, W, Dn, ub, lb)
        ub2 = [res["ub"][x] for x in range(n)]
        lb2 = [res["lb"][x] for x in range(n)]
        with lds.Graph(n, u, v) as g:
            got = g.prune(ub2, lb2, "triangle" if triangle else "edge")
        assert np.array_equal(got, _oracle_prune(n, u, v, res["ub"], res["lb"], tris))


def test_prune_fig1_example(lds):
    from helpers import load_expected, load_graph, parse_ids
    from oracle import decomp
    n, u, v = load_graph("fig1_graph.txt")
    exp = load_expected("fig1_expected.txt")
    phi = decomp.compact_numbers(n, list(zip(u.tolist(), v.tolist())))
    with lds.Graph(n, u.astype(np.int32), v.astype(np.int32)) as g:
        st = g.prune([phi[x] for x in range(n)], [phi[x] for x in range(n)])
    assert sorted(np.nonzero(st == 1)[0].tolist()) == parse_ids(exp["pruned_rule1"])
    assert sorted(np.nonzero(st == 2)[0].tolist()) == parse_ids(exp["pruned_rule2"])


@pytest.fixture(params=[1, 2], ids=["pattern_nodes", "vertex_nodes"])
def flow_variant(lds, request):
    lds.set_flow_variant(request.param)
    yield request.param
    lds.set_flow_variant(0)


@pytest.mark.parametrize("seed", range(12))
def test_pattern_max_flow_matches_dinic(lds, seed, flow_variant):
    from oracle import verify as over
    rng = synth.SplitMix64(70000 + seed)
    nv = int(rng.integers(1, 40, 1)[0])
    npat = int(rng.integers(0, 80, 1)[0])
    pats = []
    for _ in range(npat):
        k = int(rng.integers(1, 4, 1)[0])
        pats.append(tuple(sorted(set(rng.integers(0, nv, k).tolist()))))
    p = int(rng.integers(1, 9, 1)[0])
    q = int(rng.integers(1, 5, 1)[0])
    flow, side = lds.pattern_max_flow(nv, pats, p, q)
    rho = Fraction(p, q)
    net, s, t, node = over.pattern_network(range(nv), pats, rho)
    # pattern_network scales by rho's reduced form; compare flows in the same units
    want = net.max_flow(s, t)
    scale = Fraction(q, rho.denominator)
    assert Fraction(flow) == want * scale
    side_want = set(net.maximal_source_side(t))
    assert [int(node[x] in side_want) for x in range(nv)] == side.tolist()


def test_pattern_max_flow_larger_network(lds, flow_variant):
    from oracle import verify as over
    n, u, v, _ = synth.chung_lu(400, 2400, 2.1, seed=71, n_blocks=2, block_size_range=(20, 30))
    pats = list(zip(u.tolist(), v.tolist())) + [(x,) for x in range(0, n, 7)]
    for rho in (Fraction(3, 1), Fraction(7, 2), Fraction(11, 4)):
        flow, side = lds.pattern_max_flow(n, pats, rho.numerator, rho.denominator)
        net, s, t, node = over.pattern_network(range(n), pats, rho)
        assert flow == net.max_flow(s, t)
        sw = set(net.maximal_source_side(t))
        assert [int(node[x] in sw) for x in range(n)] == side.tolist()


@pytest.mark.parametrize("seed", range(3))
def test_pattern_max_flow_triangle_network(lds, flow_variant, seed):
    # the triangles of a graph with a dense block, at densities below, at and
    # above the block's: saturated, tight and short networks
    from oracle import verify as over
    n, u, v, blocks = synth.gnp_planted(70, 0.08, (26,), (0.8,), seed=72 + seed)
    tris = ograph.triangles(n, u, v)
    pats = [tuple(t) for t in tris.tolist()] + [(x,) for x in range(0, n, 9)]
    block = sorted(int(x) for x in blocks[0])
    tb = len(ograph.induced_triangles(tris, block))
    for rho in (Fraction(tb, len(block)), Fraction(tb, len(block)) - Fraction(1, 3), Fraction(2, 1),
                Fraction(len(pats), n)):
        flow, side = lds.pattern_max_flow(n, pats, rho.numerator, rho.denominator)
        net, s, t, node = over.pattern_network(range(n), pats, rho)
        assert flow == net.max_flow(s, t)
        sw = set(net.maximal_source_side(t))
        assert [int(node[x] in sw) for x in range(n)] == side.tolist()


def _as_lists(res):
    return [(d, [int(x) for x in vs]) for d, vs in res]


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("triangle", [False, True])
def test_topk_matches_definition_small(lds, seed, triangle):
    from oracle import brute
    n, u, v = synth.gnp_planted(9 + seed % 3, 0.3 + 0.03 * (seed % 6), seed=10000 + seed)[:3]
    truth = brute.brute_lds(n, u, v, triangle=triangle)
    dens = "triangle" if triangle else "edge"
    with lds.Graph(n, u, v) as g:
        for k in (1, 2, 5):
            for N, prec in ((3, "exact"), (40, "fp32"), (25, "fp64")):
                got = _as_lists(g.topk(k, dens, N, prec))
                assert got == truth[:k], (k, N, prec)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("triangle", [False, True])
def test_topk_verification_ablation_same_sets(lds, seed, triangle):
    # Sec. 7's verification ablation: the upper-bound-only networks (IsLDS-core,
    # IsLTDS-core) and the whole-graph baseline certify exactly the sets that
    # Alg. 4 / Alg. 7 certify, which are the definition's (brute force)
    from oracle import brute
    n, u, v = synth.gnp_planted(10 + seed % 3, 0.3 + 0.04 * (seed % 5), seed=12000 + seed)[:3]
    truth = brute.brute_lds(n, u, v, triangle=triangle)
    dens = "triangle" if triangle else "edge"
    with lds.Graph(n, u, v) as g:
        for mode in ("bounds", "core", "whole"):
            for k in (1, 5):
                assert _as_lists(g.topk(k, dens, 30, "exact", verify=mode)) == truth[:k], (mode, k)


def test_topk_verification_ablation_medium(lds):
    from oracle import decomp
    n, u, v, _ = synth.gnp_planted(300, 0.012, (12, 10, 9, 8), (0.9, 0.85, 0.8, 0.9), seed=11007)
    truth = decomp.lds_exact(n, u, v)
    truth_t = decomp.ltds_exact(n, u, v, ograph.triangles(n, u, v))
    with lds.Graph(n, u, v) as g:
        for mode in ("core", "whole"):
            assert _as_lists(g.topk(4, "edge", 100, verify=mode)) == [(d, c) for d, c in truth[:4]], mode
            assert _as_lists(g.topk(3, "triangle", 100, verify=mode)) == [(d, c) for d, c in truth_t[:3]], mode


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("triangle", [False, True])
def test_topk_include_zero_density(lds, seed, triangle):
    # Def. 3 / Def. 9 make isolated vertices (triangle-free connected sets) LDSs
    # (LTDSs) of density 0; with include_zero_density they count as results
    from oracle import brute
    n, u, v = synth.gnp_planted(11, 0.14 + 0.03 * (seed % 3), seed=13000 + seed)[:3]
    truth = brute.brute_lds(n, u, v, triangle=triangle, include_zero=True)
    dens = "triangle" if triangle else "edge"
    with lds.Graph(n, u, v) as g:
        got = _as_lists(g.topk(len(truth) + 2, dens, 30, "exact", include_zero=True))
    assert got == truth


def test_topk_ex_on_a_caller_stream(lds):
    import torch
    n, u, v, _ = synth.gnp_planted(300, 0.012, (12, 10), (0.9, 0.85), seed=11009)
    s = torch.cuda.Stream()
    with lds.Graph(n, u, v) as g:
        want = _as_lists(g.topk(3, "edge", 100))
        got = _as_lists(g.topk(3, "edge", 100, stream=s.cuda_stream))
        again = _as_lists(g.topk(3, "edge", 100))
    assert got == want and again == want


def test_topk_fig1(lds):
    from helpers import load_expected, load_graph, parse_sets
    n, u, v = load_graph("fig1_graph.txt")
    exp = load_expected("fig1_expected.txt")
    with lds.Graph(n, u.astype(np.int32), v.astype(np.int32)) as g:
        for N in (5, 100):
            assert _as_lists(g.topk(2, "edge", N)) == parse_sets(exp["lds_top2"])
            assert _as_lists(g.topk(2, "triangle", N)) == parse_sets(exp["ltds_top2"])


@pytest.mark.parametrize("seed", range(3))
def test_topk_matches_oracle_medium(lds, seed):
    from oracle import decomp
    n, u, v, _ = synth.gnp_planted(300, 0.012, (12, 10, 9, 8), (0.9, 0.85, 0.8, 0.9), seed=11000 + seed)
    truth = decomp.lds_exact(n, u, v)
    tris = ograph.triangles(n, u, v)
    truth_t = decomp.ltds_exact(n, u, v, tris)
    with lds.Graph(n, u, v) as g:
        assert _as_lists(g.topk(4, "edge", 100)) == [(d, c) for d, c in truth[:4]]
        assert _as_lists(g.topk(3, "triangle", 100)) == [(d, c) for d, c in truth_t[:3]]


def test_topk_planted_gnp_workload(lds):
    # n = 2000, blocks 20..60: the oracle's driver finishes in seconds here
    from oracle import ldscvx
    n, u, v, _ = synth.workload_planted_gnp()
    want = ldscvx.topk(n, u, v, 5, 200)
    with lds.Graph(n, u, v) as g:
        got = _as_lists(g.topk(5, "edge", 200, "fp64"))
        assert got == want
        assert _as_lists(g.topk(5, "edge", 200, "exact")) == want
        stats = lds.topk_last_stats()
        assert stats["certified"] >= len(want)


def _fracs(num, den):
    return [Fraction(int(a), int(b)) for a, b in zip(num, den)]


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("triangle", [False, True])
def test_compact_numbers_small_match_oracle(lds, seed, triangle):
    # exact phi (Def. 4 / Def. 10) against the brute-force definition: the
    # minimum over subsets of the marginal densities, all subsets enumerated
    from oracle import brute
    n, u, v = synth.gnp_planted(9 + seed % 4, 0.25 + 0.05 * (seed % 5), seed=14000 + seed)[:3]
    want = brute.brute_phi(n, u, v, triangle=triangle)
    with lds.Graph(n, u, v) as g:
        num, den = g.compact_numbers("triangle" if triangle else "edge")
    assert all(np.gcd(num, den) == 1) and all(den >= 1)
    assert _fracs(num, den) == [want[x] for x in range(n)]


@pytest.mark.parametrize("triangle", [False, True])
def test_compact_numbers_many_levels_match_oracle(lds, triangle):
    # a power-law graph with planted blocks: 45 edge levels and 60 triangle levels,
    # so the divide and conquer splits many times
    from oracle import decomp
    n, u, v = synth.chung_lu(1500, 6000, 2.1, seed=83, n_blocks=3, block_size_range=(10, 30))[:3]
    cu, cv = ograph.canonical_edges(n, u, v)
    pats = ([tuple(t) for t in ograph.triangles(n, cu, cv).reshape(-1, 3).tolist()] if triangle
            else list(zip(cu, cv)))
    want = decomp.compact_numbers(n, pats)
    assert len(set(want.values())) > 40
    a, b = synth.scramble(n, u, v, seed=84)
    with lds.Graph(n, a, b) as g:
        num, den = g.compact_numbers("triangle" if triangle else "edge")
    assert _fracs(num, den) == [want[x] for x in range(n)]
    # the LDSs (LTDSs) these levels determine are what the driver certifies
    truth = decomp.lds_from_phi(want, ograph.adjacency(n, cu, cv))
    with lds.Graph(n, a, b) as g:
        got = _as_lists(g.topk(6, "triangle" if triangle else "edge", 100))
    assert got == [(d, c) for d, c in truth[:6]]


def test_topk_device_chain_walk_matches_definition(lds):
    # the whole driver with the large-graph ExtractSG walk, against the oracle's
    # decomposition, on graphs whose early rounds merge candidates
    from oracle import decomp
    lds.set_extract_variant(1)
    try:
        for n, u, v in _graphs()[:3]:
            cu, cv = ograph.canonical_edges(n, u, v)
            truth = decomp.lds_exact(n, cu, cv)
            with lds.Graph(n, u, v) as g:
                for N in (3, 40):
                    assert _as_lists(g.topk(4, "edge", N)) == [(d, c) for d, c in truth[:4]], (n, N)
    finally:
        lds.set_extract_variant(0)

"""Pins for oracle.decomp (exact compact numbers, LDS / LTDS sets) against the
definitions enumerated by oracle.brute, the paper's Fig. 1 values and closed
forms."""
from fractions import Fraction
from itertools import combinations
from math import comb

import numpy as np
import pytest

from oracle import brute, decomp, graph
from helpers import load_expected, load_graph, frac, parse_sets, random_graph, random_planted


def _phi_list(phi, n):
    return [phi[x] for x in range(n)]


@pytest.mark.parametrize("seed", range(30))
def test_phi_and_lds_match_brute_force(seed):
    n = 7 + seed % 4
    n, u, v = random_graph(n, 0.3 + 0.02 * (seed % 7), seed=1000 + seed)
    en = brute.Enumeration(n, u, v)
    pats = list(zip(u.tolist(), v.tolist()))
    assert _phi_list(decomp.compact_numbers(n, pats), n) == en.compact_numbers()
    assert decomp.lds_exact(n, u, v) == en.lds_list()
    assert decomp.lds_exact(n, u, v, include_zero=True) == en.lds_list(include_zero=True)


@pytest.mark.parametrize("seed", range(20))
def test_tr_phi_and_ltds_match_brute_force(seed):
    n = 7 + seed % 4
    n, u, v = random_graph(n, 0.45 + 0.03 * (seed % 5), seed=2000 + seed)
    en = brute.Enumeration(n, u, v, triangle=True)
    tris = graph.triangles(n, u, v)
    pats = [tuple(t) for t in tris.tolist()]
    assert _phi_list(decomp.compact_numbers(n, pats), n) == en.compact_numbers()
    assert decomp.ltds_exact(n, u, v, tris) == en.lds_list()


def test_planted_blocks_match_brute_force():
    for seed in range(6):
        n, u, v, _ = random_planted(11, 0.15, (5, 4), (0.9, 0.8), seed=3000 + seed)
        assert decomp.lds_exact(n, u, v) == brute.brute_lds(n, u, v)
        tris = graph.triangles(n, u, v)
        assert decomp.ltds_exact(n, u, v, tris) == brute.brute_lds(n, u, v, triangle=True)


def test_fig1_values():
    n, u, v = load_graph("fig1_graph.txt")
    exp = load_expected("fig1_expected.txt")
    phi = decomp.compact_numbers(n, list(zip(u.tolist(), v.tolist())))
    for x in range(6):
        assert phi[x] == frac(exp["r_star_S1"])
    for x in range(9, 14):
        assert phi[x] == frac(exp["r_star_S2"])
    for x in range(14, 18):
        assert phi[x] == frac(exp["r_star_S3"])
    for x in (6, 7, 8):
        assert phi[x] == frac(exp["r_star_ghi"])
    assert phi[16] == frac(exp["phi_q"]) and phi[6] == frac(exp["phi_g"])
    assert decomp.lds_exact(n, u, v) == parse_sets(exp["lds_top2"])
    tris = graph.triangles(n, u, v)
    assert decomp.ltds_exact(n, u, v, tris) == parse_sets(exp["ltds_top2"])


def test_fig1_subgraph_values_by_enumeration():
    # densities and compactness of S1 u S3 (Sec. 3 / Sec. 6.1 examples), checked
    # on the definitions restricted to the 10 vertices of S1 u S3
    n, u, v = load_graph("fig1_graph.txt")
    exp = load_expected("fig1_expected.txt")
    keep = list(range(6)) + list(range(14, 18))
    idx = {x: i for i, x in enumerate(keep)}
    eu, ev = graph.induced_edges(u, v, keep)
    su = np.array([idx[x] for x in eu.tolist()])
    sv = np.array([idx[x] for x in ev.tolist()])
    full = (1 << 10) - 1
    en = brute.Enumeration(10, su, sv)
    assert en.density(full) == frac(exp["density_S1S3"])
    assert en.kappa[full] == frac(exp["compact_S1S3"])
    et = brute.Enumeration(10, su, sv, triangle=True)
    assert et.density(full) == frac(exp["trdensity_S1S3"])
    assert et.kappa[full] == frac(exp["trcompact_S1S3"])
    s3 = sum(1 << idx[x] for x in range(14, 18))
    assert et.density(s3) == frac(exp["trdensity_S3"])


@pytest.mark.parametrize("k", [4, 6, 9])
def test_clique_closed_forms(k):
    u, v = map(np.array, zip(*combinations(range(k), 2)))
    assert decomp.lds_exact(k, u, v) == [(Fraction(k - 1, 2), list(range(k)))]
    tris = graph.triangles(k, u, v)
    assert decomp.ltds_exact(k, u, v, tris) == [(Fraction(comb(k - 1, 2), 3), list(range(k)))]


def test_two_disjoint_cliques():
    a, b = 5, 7
    pairs = list(combinations(range(a), 2)) + list(combinations(range(a, a + b), 2))
    u, v = map(np.array, zip(*pairs))
    got = decomp.lds_exact(a + b, u, v)
    assert got == [(Fraction(b - 1, 2), list(range(a, a + b))), (Fraction(a - 1, 2), list(range(a)))]


def test_theta_cut_keeps_top_levels():
    n, u, v, _ = random_planted(60, 0.015, (8, 6, 5), (0.9, 0.9, 0.9), seed=17)
    assert len(decomp.lds_exact(n, u, v)) >= 3
    full = decomp.lds_exact(n, u, v)
    top = decomp.lds_exact(n, u, v, theta=full[1][0])
    assert top == [x for x in full if x[0] >= full[1][0]]

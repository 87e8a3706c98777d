"""Pins for oracle.fw: the integer and floating forms against Alg. 1 / Alg. 6
evaluated in exact rationals, hand-worked cases, invariants and Thm. 1."""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

from oracle import fw, graph
from helpers import load_expected, load_graph, random_graph, frac


@pytest.mark.parametrize("seed", range(6))
def test_edge_exact_equals_rational_alg1(seed):
    n, u, v = random_graph(12, 0.35, seed=200 + seed)
    for N in (1, 2, 7, 15):
        r, alpha = fw.fw_edge_rational(n, u, v, N)
        R, W, Dn, _ = fw.fw_edge_exact(n, u, v, N)
        assert Dn == (N + 1) * (N + 2)
        assert [Fraction(int(x), Dn) for x in R] == r
        for e, (a, b) in enumerate(zip(u.tolist(), v.tolist())):
            assert Fraction(int(W[e]), Dn) == alpha[(a, b)]
            assert Fraction(Dn - int(W[e]), Dn) == alpha[(b, a)]


@pytest.mark.parametrize("seed", range(4))
def test_triangle_exact_equals_rational_alg6(seed):
    n, u, v = random_graph(11, 0.5, seed=300 + seed)
    tris = graph.triangles(n, u, v)
    for N in (1, 3, 9):
        r, alpha = fw.fw_tri_rational(n, tris, N)
        R, W, Dn3, _ = fw.fw_tri_exact(n, tris, N)
        assert Dn3 == 3 * (N + 1) * (N + 2)
        assert [Fraction(int(x), Dn3) for x in R] == r
        for t in range(len(tris)):
            assert [Fraction(int(W[t, k]), Dn3) for k in range(3)] == alpha[t]


def test_single_edge_by_hand():
    # r^(0) = (1/2, 1/2); iteration 1 is a tie, the edge goes to v:
    # alpha = (1/3)(1/2) = 1/6 for u and 1/6 + 2/3 = 5/6 for v; iteration 2 the
    # edge goes to u: alpha_u = (1/2)(1/6) + 1/2 = 7/12.
    u, v = np.array([0]), np.array([1])
    for N, want in [(0, (Fraction(1, 2), Fraction(1, 2))), (1, (Fraction(1, 6), Fraction(5, 6))),
                    (2, (Fraction(7, 12), Fraction(5, 12)))]:
        R, W, Dn, _ = fw.fw_edge_exact(2, u, v, N)
        assert (Fraction(int(R[0]), Dn), Fraction(int(R[1]), Dn)) == want


@pytest.mark.parametrize("seed", range(3))
def test_invariants_every_iteration(seed):
    n, u, v = random_graph(40, 0.15, seed=400 + seed)
    m = len(u)
    R, W = None, None
    for i in range(1, 60):
        R, W, Dn, ch = fw.fw_edge_exact(n, u, v, i, R0=R, W0=W, i0=i - 1, record=True)
        assert R.sum() == m * Dn
        assert W.min() >= 0 and W.max() <= Dn
        assert np.array_equal(R, fw.edge_loads_from_W(n, u, v, W, Dn))
    tris = graph.triangles(n, u, v)
    R, W = None, None
    for i in range(1, 30):
        R, W, Dn3, _ = fw.fw_tri_exact(n, tris, i, R0=R, W0=W, i0=i - 1)
        assert R.sum() == len(tris) * Dn3
        assert np.array_equal(W.sum(axis=1), np.full(len(tris), Dn3))
        assert np.array_equal(R, fw.tri_loads_from_W(n, tris, W))


def test_clique_loads_stay_balanced_in_sum():
    k = 7
    u, v = map(np.array, zip(*combinations(range(k), 2)))
    R, W, Dn, _ = fw.fw_edge_exact(k, u, v, 400)
    r = R / Dn
    assert np.allclose(r, (k - 1) / 2, atol=0.02)


def test_fig1_converges_to_table2():
    n, u, v = load_graph("fig1_graph.txt")
    exp = load_expected("fig1_expected.txt")
    want = np.zeros(n)
    for x in range(6):
        want[x] = float(frac(exp["r_star_S1"]))
    for x in range(9, 14):
        want[x] = float(frac(exp["r_star_S2"]))
    for x in range(14, 18):
        want[x] = float(frac(exp["r_star_S3"]))
    for x in (6, 7, 8):
        want[x] = float(frac(exp["r_star_ghi"]))
    errs = []
    for N in (200, 2000, 20000):
        R, W, Dn, _ = fw.fw_edge_exact(n, u, v, N)
        errs.append(np.abs(R / Dn - want).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3


def _agreeing_prefix(ch_a, ch_b):
    k = 0
    for a, b in zip(ch_a, ch_b):
        if not np.array_equal(a, b):
            break
        k += 1
    return k


def test_fp64_literal_tracks_rational_while_choices_agree():
    checked = 0
    for seed in range(12):
        n, u, v = random_graph(9, 0.45, seed=500 + seed)
        if len(u) == 0:
            continue
        for N in range(1, 9):
            rec64 = []
            r64, a, rowptr, col = fw.fw_edge_fp64_literal(n, u, v, N, record=rec64)
            R, W, Dn, rec = fw.fw_edge_exact(n, u, v, N, record=True)
            if _agreeing_prefix(rec64, rec) < N:
                break
            checked += 1
            assert np.allclose(r64, R / Dn, rtol=1e-13, atol=1e-13)
            # alpha per ordered pair: complements agree with W / D
            for e, (x, y) in enumerate(zip(u.tolist(), v.tolist())):
                s_xy = rowptr[x] + np.searchsorted(col[rowptr[x]:rowptr[x + 1]], y)
                assert abs(a[s_xy] - W[e] / Dn) < 1e-13
    assert checked >= 20


def test_triangle_fp64_literal_tracks_rational_while_choices_agree():
    # Alg. 6 in binary64 against the exact integer form (itself pinned to the
    # rational Alg. 6 above) at every N while the receiving vertices agree: a
    # summation-order or gamma slip past the first iteration shows up here
    checked = 0
    for seed in range(12):
        n, u, v = random_graph(10, 0.55, seed=800 + seed)
        tris = graph.triangles(n, u, v)
        if len(tris) == 0:
            continue
        for N in range(1, 10):
            rec64 = []
            r64, a = fw.fw_tri_fp64_literal(n, tris, N, record=rec64)
            R, W, Dn3, rec = fw.fw_tri_exact(n, tris, N, record=True)
            if _agreeing_prefix(rec64, rec) < N:
                break
            checked += 1
            assert np.allclose(r64, R / Dn3, rtol=1e-13, atol=1e-13)
            assert np.allclose(a, W / Dn3, rtol=0, atol=1e-14)
    assert checked >= 20


def test_triangle_fp64_literal_against_rational_directly():
    n, u, v = random_graph(8, 0.6, seed=17)
    tris = graph.triangles(n, u, v)
    for N in (2, 3, 5):
        rec64 = []
        r64, a = fw.fw_tri_fp64_literal(n, tris, N, record=rec64)
        r_q, a_q = fw.fw_tri_rational(n, tris, N)
        _, _, _, rec = fw.fw_tri_exact(n, tris, N, record=True)
        if _agreeing_prefix(rec64, rec) < N:
            continue
        assert np.allclose(r64, [float(x) for x in r_q], rtol=1e-13, atol=1e-13)
        assert np.allclose(a, np.array([[float(x) for x in row] for row in a_q]), rtol=0, atol=1e-14)


def test_fp32_recurrence_tracks_rational_while_choices_agree():
    checked = 0
    for seed in range(12):
        n, u, v = random_graph(9, 0.45, seed=600 + seed)
        if len(u) == 0:
            continue
        for N in range(1, 9):
            rec32 = []
            r32, W32, Dn = fw.fw_edge_fp32(n, u, v, N, record=rec32)
            R, W, Dn2, rec = fw.fw_edge_exact(n, u, v, N, record=True)
            if _agreeing_prefix(rec32, rec) < N:
                break
            checked += 1
            assert np.array_equal(W32, W)
            assert np.allclose(r32, R / Dn, rtol=1e-6, atol=1e-6)
    assert checked >= 20


def test_triangle_float_forms_close_to_exact():
    n, u, v = random_graph(10, 0.6, seed=7)
    tris = graph.triangles(n, u, v)
    R, W, Dn3, _ = fw.fw_tri_exact(n, tris, 1)
    r64, a = fw.fw_tri_fp64_literal(n, tris, 1)
    assert np.allclose(r64, R / Dn3, rtol=1e-13)
    r32, W32, _ = fw.fw_tri_fp32(n, tris, 1)
    assert np.array_equal(W32, W)
    assert np.allclose(r32, R / Dn3, rtol=1e-6)


def test_fp32_weights_are_feasible():
    n, u, v = random_graph(60, 0.1, seed=8)
    r32, W, Dn = fw.fw_edge_fp32(n, u, v, 100)
    assert W.min() >= 0 and W.max() <= Dn
    R = fw.edge_loads_from_W(n, u, v, W, Dn)
    assert R.sum() == len(u) * Dn
    # binary32 loads track the exact loads of the same choices
    assert np.allclose(r32, R / Dn, rtol=2e-5, atol=2e-5)


def test_snapped_triangle_weights_are_feasible():
    # the binary64 alphas snapped to integers: every row sums to exactly 3 D,
    # no weight is negative, and each is within one unit of alpha * 3 D
    n, u, v = random_graph(12, 0.6, seed=23)
    tris = graph.triangles(n, u, v)
    for N in (1, 7, 30):
        _, a = fw.fw_tri_fp64_literal(n, tris, N)
        Dn3 = 3 * fw.D(N)
        W = fw.snap_tri_weights(a, Dn3)
        assert np.all(W.sum(axis=1) == Dn3)
        assert W.min() >= 0
        assert np.abs(W - a * Dn3).max() <= 1.5

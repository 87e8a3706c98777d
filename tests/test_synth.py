"""The seeded input generators shared by the oracle and the GPU path: the
published SplitMix64 sequence, determinism, and the structure each family
promises (canonical edge lists, exact edge counts, planted blocks)."""
import numpy as np

from paper_2504_10937_gb300 import synth


def test_splitmix64_published_sequence():
    # Steele, Lea and Flood's SplitMix64 from state 1234567: the sequence every
    # reference implementation prints for this seed
    assert [int(x) for x in synth.SplitMix64(1234567).u64(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_uniform_and_integers_ranges():
    r = synth.SplitMix64(3)
    x = r.uniform(10000)
    assert x.min() >= 0.0 and x.max() < 1.0 and abs(x.mean() - 0.5) < 0.02
    k = synth.SplitMix64(4).integers(5, 9, 10000)
    assert set(np.unique(k).tolist()) == {5, 6, 7, 8}


def _canonical(n, u, v):
    assert u.dtype == np.int32 and v.dtype == np.int32
    assert np.all(u < v) and np.all(u >= 0) and np.all(v < n)
    key = u.astype(np.int64) * n + v
    assert np.all(np.diff(key) > 0)          # sorted by (u, v), no repeats


def test_generators_are_canonical_and_deterministic():
    for make in (lambda: synth.gnp_planted(500, 0.02, (20, 15), (0.9, 0.7), seed=1)[:3],
                 lambda: synth.chung_lu(2000, 8000, 2.1, seed=2, n_blocks=3)[:3],
                 lambda: synth.rmat(10, 8, 0.57, 0.19, 0.19, seed=3, n_cliques=2, clique_size_range=(10, 20))[:3],
                 lambda: synth.barabasi_albert(1000, 3, seed=4)[:3]):
        n, u, v = make()
        _canonical(n, u, v)
        n2, u2, v2 = make()
        assert n == n2 and np.array_equal(u, u2) and np.array_equal(v, v2)


def test_chung_lu_tops_up_to_exactly_m_background_edges():
    n, u, v, blocks = synth.chung_lu(3000, 12000, 2.3, seed=5)
    assert len(u) == 12000 and blocks == []


def test_planted_blocks_are_disjoint_and_dense():
    n, u, v, blocks = synth.gnp_planted(400, 0.01, (20, 25), (0.9, 0.8), seed=6)
    assert len(blocks) == 2
    assert not set(blocks[0]) & set(blocks[1])
    es = set(zip(u.tolist(), v.tolist()))
    for b, p in zip(blocks, (0.9, 0.8)):
        b = sorted(b)
        pairs = [(x, y) for i, x in enumerate(b) for y in b[i + 1:]]
        frac = sum((x, y) in es for x, y in pairs) / len(pairs)
        assert abs(frac - p) < 0.12


def test_batched_mix_ranges():
    mix = synth.batched_mix(40, seed=7, n_range=(50, 2000))
    assert len(mix) == 40
    for g in mix:
        assert 50 <= g["n"] <= 2000
        _canonical(g["n"], g["u"], g["v"])
    assert 0 < sum(g["triangle"] for g in mix) < 40


def test_scramble_keeps_the_edge_set():
    n, u, v = synth.gnp_planted(300, 0.03, (), (), seed=8)[:3]
    a, b = synth.scramble(n, u, v, seed=9)
    keep = a != b
    lo, hi = np.minimum(a, b)[keep], np.maximum(a, b)[keep]
    got = np.unique(lo.astype(np.int64) * n + hi)
    assert np.array_equal(got, u.astype(np.int64) * n + v)
    assert np.any(a == b)                   # self-loops are present
    assert len(a) > len(u)                  # and repeats


def test_rmat_device_reproduces_rmat():
    # the device-side R-MAT (used for scale 24) draws the same SplitMix64 numbers,
    # quadrants and relabelling as the numpy generator; run here on the CPU
    pytest = __import__("pytest")
    torch = pytest.importorskip("torch")
    for scale, seed in ((8, 77), (11, 5)):
        n, u, v, _ = synth.rmat(scale, 16, 0.57, 0.19, 0.19, seed=seed, n_cliques=0)
        n2, s, d = synth.rmat_device(scale, 16, 0.57, 0.19, 0.19, seed=seed, device="cpu")
        assert n2 == n and s.dtype == torch.int32
        cu, cv = synth._canon(n2, s.numpy(), d.numpy())
        assert np.array_equal(cu, u) and np.array_equal(cv, v)

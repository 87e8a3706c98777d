"""GPU parity: ingest, Frank-Wolfe (edge and triangle, three arithmetics),
triangle listing and core numbers through the C-ABI against the CPU oracle.

Tolerances: the exact form and every integer output must match bit for bit;
the binary32 and binary64 forms follow the oracle's operation order, so their
loads must match bit for bit as well (the stated bound of 1e-4 / 1e-6 relative
is checked too, and holds with error 0)."""
import numpy as np
import pytest

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
    # ragged slot counts, several 32-slot chunks per row, isolated vertices, hubs
    out = []
    out.append(synth.gnp_planted(37, 0.2, (6,), (0.9,), seed=1)[:3])
    out.append(synth.gnp_planted(300, 0.02, (15, 10), (0.9, 0.7), seed=2)[:3])
    out.append(synth.chung_lu(2000, 9000, 2.1, seed=3, n_blocks=3, block_size_range=(20, 60))[:3])
    out.append(synth.rmat(10, 8, 0.57, 0.19, 0.19, seed=4, n_cliques=2, clique_size_range=(15, 30))[:3])
    return out


def test_ingest_matches_canonical_edges(lds):
    for k, (n, u, v) in enumerate(_graphs()):
        a, b = synth.scramble(n, u, v, seed=10 + k, dup_frac=0.2, loop_frac=0.05)
        with lds.Graph(n, a, b) as g:
            gu, gv = g.edges()
            assert np.array_equal(gu, u) and np.array_equal(gv, v)
            info = g.info()
            assert info["m"] == len(u)
            assert info["self_loops"] == int(np.sum(a == b))
            assert info["duplicates"] == len(a) - info["self_loops"] - len(u)
            deg = ograph.degrees(n, u, v)
            assert info["max_degree"] == int(deg.max())
            assert info["isolated"] == int(np.sum(deg == 0))


def test_ingest_from_device_memory(lds):
    import torch
    n, u, v = _graphs()[2]
    a, b = synth.scramble(n, u, v, seed=5)
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b).cuda()
    with lds.Graph(n, ta, tb, stream=torch.cuda.current_stream().cuda_stream) as g:
        gu, gv = g.edges()
        assert np.array_equal(gu, u) and np.array_equal(gv, v)


def test_ingest_rejects_bad_ids_and_sizes(lds):
    with pytest.raises(lds.LdsError) as e:
        lds.Graph(4, np.array([0, 4], np.int32), np.array([1, 1], np.int32))
    assert e.value.status == lds.EINVAL
    with pytest.raises(lds.LdsError) as e:
        lds.Graph(4, np.array([-1], np.int32), np.array([1], np.int32))
    assert e.value.status == lds.EINVAL
    with pytest.raises(lds.LdsError):
        lds.Graph(-1, np.zeros(0, np.int32), np.zeros(0, np.int32))


def test_degenerate_graphs(lds):
    # no edges, only self-loops, a single edge
    for n, a, b in [(5, [], []), (3, [1, 2, 2], [1, 2, 2]), (2, [1], [0])]:
        a = np.array(a, np.int32)
        b = np.array(b, np.int32)
        with lds.Graph(n, a, b) as g:
            cu, cv = ograph.canonical_edges(n, a, b)
            for N in (0, 1, 2, 5):
                got = g.fw(N)
                R, W, Dn, _ = ofw.fw_edge_exact(n, cu, cv, N)
                assert got["D"] == Dn
                assert np.array_equal(got["R"], R) and np.array_equal(got["W"], W)
            assert g.triangles().shape == (0, 3)


@pytest.fixture(params=[0, 1, 2, 3, 4, 5, 6], ids=["auto", "symmetric", "oriented64", "oriented32", "oriented32_rows",
                                                  "oriented32_coop", "cluster_any_size"])
def variant(request, lds):
    lds.set_fw_variant(request.param)
    yield request.param
    lds.set_fw_variant(0)


@pytest.mark.parametrize("N", [0, 1, 2, 7, 33, 100])
def test_fw_exact_bit_exact(lds, N, variant):
    for n, u, v in _graphs():
        with lds.Graph(n, u, v) as g:
            got = g.fw(N, precision="exact")
            R, W, Dn, ch = ofw.fw_edge_exact(n, u, v, N, record=True)
            assert got["D"] == Dn
            assert np.array_equal(got["R"], R)
            assert np.array_equal(got["W"], W)
            assert np.array_equal(got["r"], R / Dn)
            if N:
                assert np.array_equal(got["last"].astype(bool), ch[-1])


def test_fw_beyond_the_shared_memory_hot_set(lds, variant):
    # more than 16384 active vertices: gathers and counts also go through global memory
    n, u, v, _ = synth.chung_lu(60000, 240000, 2.1, seed=6, n_blocks=4, block_size_range=(30, 90))
    with lds.Graph(n, u, v) as g:
        for N in (1, 25):
            got = g.fw(N, precision="exact")
            R, W, Dn, ch = ofw.fw_edge_exact(n, u, v, N, record=True)
            assert np.array_equal(got["R"], R) and np.array_equal(got["W"], W)
            assert np.array_equal(got["last"].astype(bool), ch[-1])
            got32 = g.fw(N, precision="fp32")
            r32, W32, _ = ofw.fw_edge_fp32(n, u, v, N)
            assert np.array_equal(got32["r"], r32.astype(np.float64)) and np.array_equal(got32["W"], W32)


def test_fw_exact_plane_folding_over_many_iterations(lds):
    # more iterations than the bit-plane buffer holds for small graphs (folds several times)
    n, u, v = _graphs()[1]
    with lds.Graph(n, u, v) as g:
        got = g.fw(1200, precision="exact")
    R, W, Dn, _ = ofw.fw_edge_exact(n, u, v, 1200)
    assert np.array_equal(got["R"], R) and np.array_equal(got["W"], W)


@pytest.mark.parametrize("N", [1, 5, 60])
def test_fw_fp32_bit_exact(lds, N, variant):
    for n, u, v in _graphs():
        with lds.Graph(n, u, v) as g:
            got = g.fw(N, precision="fp32")
        r32, W32, Dn = ofw.fw_edge_fp32(n, u, v, N)
        assert np.array_equal(got["r"], r32.astype(np.float64))
        assert np.array_equal(got["W"], W32)
        rel = np.abs(got["r"] - r32) / np.maximum(np.abs(r32), 1e-30)
        assert rel.max(initial=0.0) <= 1e-4
        assert np.array_equal(got["R"], ofw.edge_loads_from_W(n, u, v, W32, Dn))


@pytest.mark.parametrize("N", [1, 4, 30])
def test_fw_fp64_literal_bit_exact(lds, N):
    for n, u, v in _graphs()[:3]:
        with lds.Graph(n, u, v) as g:
            got = g.fw(N, precision="fp64")
        r64, a, rowptr, col = ofw.fw_edge_fp64_literal(n, u, v, N)
        assert np.array_equal(got["r"], r64)
        rel = np.abs(got["r"] - r64) / np.maximum(np.abs(r64), 1e-300)
        assert rel.max(initial=0.0) <= 1e-6
        Dn = (N + 1) * (N + 2)
        W = np.empty(len(u), np.int64)
        for e, (x, y) in enumerate(zip(u.tolist(), v.tolist())):
            s = rowptr[x] + np.searchsorted(col[rowptr[x]:rowptr[x + 1]], y)
            W[e] = int(np.rint(a[s] * Dn))
        assert np.array_equal(got["W"], W)


def test_triangle_listing(lds):
    for n, u, v in _graphs():
        with lds.Graph(n, u, v) as g:
            t = g.triangles()
            assert g.info()["triangles"] == len(t)
        assert np.array_equal(t, ograph.triangles(n, u, v).astype(np.int32))


@pytest.mark.parametrize("N", [0, 1, 3, 40])
def test_fw_triangle_exact_and_fp32(lds, N):
    for n, u, v in _graphs():
        tris = ograph.triangles(n, u, v)
        with lds.Graph(n, u, v) as g:
            got = g.fw(N, density="triangle", precision="exact")
            got32 = g.fw(N, density="triangle", precision="fp32")
        R, W, Dn3, ch = ofw.fw_tri_exact(n, tris, N, record=True)
        assert got["D"] == Dn3
        assert np.array_equal(got["R"], R) and np.array_equal(got["W"], W)
        if N:
            assert np.array_equal(got["last"], ch[-1].astype(np.uint8))
        r32, W32, _ = ofw.fw_tri_fp32(n, tris, N)
        assert np.array_equal(got32["r"], r32.astype(np.float64))
        assert np.array_equal(got32["W"], W32)
        # Alg. 6 literally in binary64 (one alpha per vertex-triangle pair, r summed
        # in ascending triangle order): bit for bit, hence within the 1e-6 bound
        with lds.Graph(n, u, v) as g:
            got64 = g.fw(N, density="triangle", precision="fp64", want=("r", "W"))
        r64, a64 = ofw.fw_tri_fp64_literal(n, tris, N)
        assert np.array_equal(got64["r"], r64)
        assert np.array_equal(got64["W"], ofw.snap_tri_weights(a64, Dn3))


def test_core_numbers(lds):
    for n, u, v in _graphs():
        with lds.Graph(n, u, v) as g:
            core = g.core_numbers("edge")
            trcore = g.core_numbers("triangle")
        assert np.array_equal(core, ograph.core_numbers(n, u, v))
        assert np.array_equal(trcore, ograph.tr_core_numbers(n, ograph.triangles(n, u, v)))


def test_core_numbers_large(lds):
    # more live vertices than the single-block tail takes, so the grid-wide
    # levels and the hand-over to one block both run
    n, u, v, _ = synth.chung_lu(40000, 400000, 2.1, seed=5, n_blocks=4, block_size_range=(50, 120))
    with lds.Graph(n, u, v) as g:
        core = g.core_numbers("edge")
    assert np.array_equal(core, ograph.core_numbers(n, u, v))
    n, u, v, _ = synth.chung_lu(20000, 120000, 2.1, seed=6, n_blocks=3, block_size_range=(30, 60))
    with lds.Graph(n, u, v) as g:
        trcore = g.core_numbers("triangle")
    assert np.array_equal(trcore, ograph.tr_core_numbers(n, ograph.triangles(n, u, v)))


def test_injected_allocation_failure_reports_enomem(lds):
    n, u, v = _graphs()[1]
    lds.debug_fail_alloc_after(3)
    with pytest.raises(lds.LdsError) as e:
        lds.Graph(n, u, v)
    assert e.value.status == lds.ENOMEM
    lds.debug_fail_alloc_after(0)
    with lds.Graph(n, u, v) as g:                 # the library stays usable
        assert g.info()["m"] == len(u)

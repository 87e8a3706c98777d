"""Parity at the benchmark's full size: the 1M-vertex power-law workload
(n = 1e6, 10.6M edges, 50 planted blocks) as the bench runs it, from the raw
scrambled COO through lds_create_graph.

The oracle cannot run inside a test at this size, so its values were written
once by committed oracle-only scripts (tests/golden/make_topk_golden.py and
tests/golden/make_fw_sample.py): the top-10 LDS answer (Problem 1), and the
Frank-Wolfe loads after 500 iterations on a seeded sample of 2,048 vertices in
the exact integer form and in the binary64 literal form of Alg. 1.
"""
import os

import numpy as np
import pytest

from paper_2504_10937_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def lds():
    from paper_2504_10937_gb300 import lds as _l
    _l.load()
    return _l


@pytest.fixture(scope="module")
def workload():
    n, u, v, _ = synth.workload_chung_lu_1m(seed=2)
    a, b = synth.scramble(n, u, v, seed=20)
    return n, u, v, a, b


def _golden_sets(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.split("#")[0].strip()
            if ln:
                d, vs = ln.split(":")
                out.append((d.strip(), [int(x) for x in vs.split(",")]))
    return out


def test_top10_lds_matches_oracle(lds, workload):
    n, u, v, a, b = workload
    if not os.path.exists(os.path.join(GOLDEN, "chung_lu_1m_top10.txt")):
        pytest.skip("the oracle's answer for this workload has not been written yet")
    want = _golden_sets("chung_lu_1m_top10.txt")
    assert len(want) == 10
    with lds.Graph(n, a, b) as g:
        assert g.m == len(u)
        for prec in ("exact", "fp32"):
            got = [(str(d), [int(x) for x in c]) for d, c in g.topk(10, "edge", 500, prec)]
            assert got == want, prec


def test_fw_sample_matches_oracle(lds, workload):
    n, u, v, a, b = workload
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "chung_lu_1m_fw500_sample.txt"))
            if ln.strip() and not ln.startswith("#")]
    ids = np.array([int(r[0]) for r in rows])
    R_want = np.array([int(r[1]) for r in rows], dtype=np.int64)
    r64_want = np.array([float(r[2]) for r in rows])
    with lds.Graph(n, a, b) as g:
        ex = g.fw(500, precision="exact", want=("R",))
        assert ex["D"] == 501 * 502
        assert np.array_equal(ex["R"][ids], R_want)
        # binary64 in the literal order of Alg. 1 (spec: 1e-6 relative); the
        # pinned summation order makes it bit for bit
        f64 = g.fw(500, precision="fp64", want=("r",))
        assert np.array_equal(f64["r"][ids], r64_want)


def test_rmat_top5_ltds_matches_oracle(lds):
    # LTDScvx on an R-MAT graph (scale 12, edge factor 6, 4 planted near-cliques),
    # from a raw scrambled COO, against the oracle's answer: triangle listing,
    # triangle FW, ExtractSG (Def. 12), pruning with tr-core numbers and IsLTDS
    n, u, v, _ = synth.rmat(12, 6, 0.57, 0.19, 0.19, seed=312, n_cliques=4, clique_size_range=(20, 40))
    a, b = synth.scramble(n, u, v, seed=313)
    want = _golden_sets("rmat12_top5.txt")
    with lds.Graph(n, a, b) as g:
        for prec in ("fp32", "exact"):
            got = [(str(d), [int(x) for x in c]) for d, c in g.topk(5, "triangle", 300, prec)]
            assert got == want, prec

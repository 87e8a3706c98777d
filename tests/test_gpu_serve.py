"""Batched queries and the serving loop on the GPU: every result equals the
single-query answer of lds_topk (the same sets, the same exact densities),
whether a query runs alone, in a batch or among other requests in flight."""
import numpy as np
import pytest

from paper_2504_10937_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lds():
    from paper_2504_10937_gb300 import lds as _l
    _l.load()
    return _l


def _graphs(lds, count, seed):
    mix = synth.batched_mix(count, seed=seed, n_range=(40, 1500))
    out = []
    for g in mix:
        out.append((lds.Graph(g["n"], g["u"].astype(np.int32), g["v"].astype(np.int32)),
                    "triangle" if g["triangle"] else "edge"))
    return out


def _same(a, b):
    assert len(a) == len(b)
    for (da, va), (db, vb) in zip(a, b):
        assert da == db
        assert np.array_equal(va, vb)


@pytest.mark.parametrize("precision", ["exact", "fp32"])
def test_fw_batch_state_equals_single_graph_path(lds, precision):
    mix = synth.batched_mix(20, seed=407, n_range=(40, 3000))
    n, u, v, _ = synth.chung_lu(30000, 90000, 2.3, seed=408)    # too many vertices for the on-chip kernel
    mix.append(dict(n=n, u=u, v=v, triangle=False))
    iters = 37
    batch = [lds.Graph(g["n"], g["u"].astype(np.int32), g["v"].astype(np.int32)) for g in mix]
    single = [lds.Graph(g["n"], g["u"].astype(np.int32), g["v"].astype(np.int32)) for g in mix]
    on = lds.fw_batch(batch, iters, precision)
    D = (iters + 1) * (iters + 2)
    fits = [g.info()["n"] - g.info()["isolated"] <= 24576 and g.m > 0 and
            max(g.info()["max_degree"], 1) * D < 2 ** 32 for g in batch]
    assert on == sum(fits) and not fits[-1]
    for a, b in zip(batch, single):
        got = a.fw_state()
        want = b.fw(iters, precision=precision, want=("r", "R", "W"))
        assert got["D"] == want["D"]
        assert np.array_equal(got["R"], want["R"])
        assert np.array_equal(got["W"], want["W"])
        assert np.array_equal(got["r"], want["r"])
    for g in batch + single:
        g.close()


def test_batch_equals_single_queries(lds):
    gs = _graphs(lds, 24, seed=401)
    queries = [(g, 3, d, 60, "fp32") for g, d in gs]
    alone = [g.topk(3, d, 60, "fp32") for g, d in gs]
    for workers in (1, 4, 0):
        got = lds.topk_batch(queries, workers=workers)
        for a, b in zip(alone, got):
            _same(a, b)
    for g, _ in gs:
        g.close()


def test_batch_with_repeated_handle(lds):
    gs = _graphs(lds, 3, seed=402)
    g, d = gs[0]
    alone = g.topk(2, d, 50, "exact")
    got = lds.topk_batch([(g, 2, d, 50, "exact")] * 5, workers=4)
    for r in got:
        _same(alone, r)
    for g, _ in gs:
        g.close()


def test_autotune_picks_a_tried_count(lds):
    gs = _graphs(lds, 8, seed=403)
    w = lds.batch_autotune([(g, 3, d, 40, "fp32") for g, d in gs])
    assert w in (1, 2, 4, 8, 16)
    # the batched FW's launch shape was tuned for the size buckets of the edge queries
    for g, d in gs:
        if d == "edge":
            info = g.info()
            assert lds.fw_batch_threads(info["n"] - info["isolated"]) in (128, 256, 512, 1024)
    for g, _ in gs:
        g.close()


def test_server_results_same_alone_and_in_the_mix(lds):
    gs = _graphs(lds, 10, seed=404)
    rng = synth.SplitMix64(405)
    reqs = []
    for i in range(30):
        g, d = gs[int(rng.integers(0, len(gs), 1)[0])]
        k = int(rng.integers(1, 6, 1)[0])
        prec = ("exact", "fp32", "fp64")[i % 3]
        reqs.append((g, k, d, 50, prec))
    alone = [g.topk(k, d, it, p) for g, k, d, it, p in reqs]
    with lds.Server(1 << 34, 6) as srv:
        tickets = [srv.submit(*r) for r in reqs]
        for t, want in zip(tickets, alone):
            got, timing = srv.wait(t)
            _same(want, got)
            assert timing["run_ms"] >= 0 and timing["queue_ms"] >= 0
    for g, _ in gs:
        g.close()


def test_server_budget(lds):
    gs = _graphs(lds, 4, seed=406)
    g, d = gs[0]
    with lds.Server(1 << 10, 2) as srv:
        with pytest.raises(lds.LdsError) as e:
            srv.submit(g, 2, d, 40, "fp32")
        assert e.value.status == lds.EBUSY
    # a budget that fits one query at a time still finishes everything, in order
    big = max(96 * (h.m + h.n) + (1 << 20) + (64 * 16 * h.m if dd == "triangle" else 0) for h, dd in gs)
    alone = [h.topk(2, dd, 40, "fp32") for h, dd in gs]
    with lds.Server(big, 4) as srv:
        tickets = [srv.submit(h, 2, dd, 40, "fp32") for h, dd in gs]
        for t, want in zip(tickets, alone):
            got, _ = srv.wait(t)
            _same(want, got)
    for g, _ in gs:
        g.close()


@pytest.fixture(scope="module")
def oracle_mix():
    # 64 graphs of the batched mix (20 of them triangle-density queries), small
    # enough for the CPU oracle's driver (about a minute for all of them)
    from oracle import ldscvx
    mix = synth.batched_mix(64, seed=41, n_range=(50, 1500))
    want = [[(d, list(c)) for d, c in ldscvx.topk(g["n"], g["u"], g["v"], 3, 200 if g["triangle"] else 100,
                                                  triangle=g["triangle"], precision="fp32")] for g in mix]
    return mix, want


def _lists(res):
    return [(d, [int(x) for x in c]) for d, c in res]


def test_batch_matches_oracle(lds, oracle_mix):
    # Problem 1 / Problem 2 answers of the batched path against the oracle's
    # driver, both densities, with the autotuned launch shape
    mix, want = oracle_mix
    gs = [lds.Graph(g["n"], g["u"].astype(np.int32), g["v"].astype(np.int32)) for g in mix]
    queries = [(g, 3, "triangle" if x["triangle"] else "edge", 200 if x["triangle"] else 100, "fp32")
               for g, x in zip(gs, mix)]
    workers = lds.batch_autotune(queries)
    got = lds.topk_batch(queries, workers=workers)
    assert [_lists(r) for r in got] == want
    for g in gs:
        g.close()


def test_server_matches_oracle(lds, oracle_mix):
    # the same queries through the serving loop, all submitted at once so that
    # they overlap on the device
    mix, want = oracle_mix
    gs = [lds.Graph(g["n"], g["u"].astype(np.int32), g["v"].astype(np.int32)) for g in mix]
    with lds.Server(1 << 34, 8) as srv:
        tickets = [srv.submit(g, 3, "triangle" if x["triangle"] else "edge", 200 if x["triangle"] else 100, "fp32")
                   for g, x in zip(gs, mix)]
        got = [_lists(srv.wait(t)[0]) for t in tickets]
    assert got == want
    for g in gs:
        g.close()

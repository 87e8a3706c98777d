"""Host logic of the batch and serving layer, without a GPU: the admission
rule (oldest queued request whose graph is idle and whose footprint fits the
free budget) and the refusal to start without a device."""
import numpy as np
import pytest

from paper_2504_10937_gb300 import lds


@pytest.fixture(scope="module")
def lib():
    lds.load()
    return lds


def test_pick_oldest_that_fits(lib):
    assert lib.debug_pick_next([10, 5, 3], [0, 0, 0], 100) == 0
    assert lib.debug_pick_next([10, 5, 3], [0, 0, 0], 5) == 1
    assert lib.debug_pick_next([10, 5, 3], [0, 0, 0], 4) == 2
    assert lib.debug_pick_next([10, 5, 3], [0, 0, 0], 2) == -1


def test_pick_skips_busy_graphs(lib):
    assert lib.debug_pick_next([1, 1, 1], [1, 0, 0], 10) == 1
    assert lib.debug_pick_next([1, 1, 1], [1, 1, 0], 10) == 2
    assert lib.debug_pick_next([1, 1, 1], [1, 1, 1], 10) == -1
    assert lib.debug_pick_next([], [], 10) == -1


def test_pick_matches_a_plain_restatement(lib):
    rng = np.random.default_rng(7)
    for _ in range(200):
        k = int(rng.integers(1, 12))
        b = rng.integers(1, 100, k)
        busy = rng.integers(0, 2, k)
        free = int(rng.integers(0, 120))
        want = next((i for i in range(k) if not busy[i] and b[i] <= free), -1)
        assert lib.debug_pick_next(b, busy, free) == want


def test_no_device_means_no_server(lib):
    if lib.device_count() > 0:
        pytest.skip("a CUDA device is present")
    with pytest.raises(lib.LdsError) as e:
        lib.Server(1 << 30, 2)
    assert e.value.status == lib.ECUDA


class _NoGraph:
    """A stand-in handle: the entry points must reject it before any device work."""
    def __init__(self, value):
        import ctypes
        self.handle = ctypes.c_void_p(value)


def test_batch_rejects_null_graph(lib):
    with pytest.raises(lib.LdsError) as e:
        lib.topk_batch([(_NoGraph(None), 3, "edge", 10, "exact")], workers=1)
    assert e.value.status == lib.EINVAL


def test_fw_batch_rejects_null_and_repeated_graphs(lib):
    with pytest.raises(lib.LdsError) as e:
        lib.fw_batch([_NoGraph(None)], 10, "exact")
    assert e.value.status == lib.EINVAL
    # the repeat is found before any handle is touched
    g = _NoGraph(0x1000)
    with pytest.raises(lib.LdsError) as e:
        lib.fw_batch([g, g], 10, "exact")
    assert e.value.status == lib.EINVAL
    assert "twice" in str(e.value)


def test_empty_batch_is_fine(lib):
    assert lib.topk_batch([], workers=1) == []


def test_result_conversion(lib):
    # an lds_result laid out in host memory as the library lays it out
    import ctypes
    from fractions import Fraction
    num = (ctypes.c_int64 * 2)(5, 1)
    den = (ctypes.c_int64 * 2)(2, 2)
    off = (ctypes.c_int64 * 3)(0, 3, 5)
    ver = (ctypes.c_int32 * 5)(1, 4, 7, 2, 3)
    P64, P32 = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)
    r = lib.LdsResult(2, ctypes.cast(num, P64), ctypes.cast(den, P64), ctypes.cast(off, P64), ctypes.cast(ver, P32))
    out = lib._result_list(ctypes.pointer(r))
    assert [(d, c.tolist()) for d, c in out] == [(Fraction(5, 2), [1, 4, 7]), (Fraction(1, 2), [2, 3])]
    assert all(c.dtype == np.int32 for _, c in out)
    empty = lib.LdsResult(0, ctypes.cast(num, P64), ctypes.cast(den, P64), ctypes.cast(off, P64), ctypes.cast(ver, P32))
    assert lib._result_list(ctypes.pointer(empty)) == []

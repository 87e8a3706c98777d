"""Python binding of liblds (argument marshalling only).

Every function calls the C-ABI declared in ``include/lds.h``; no step of the
method runs in Python.  Host inputs are numpy arrays; device inputs are torch
CUDA tensors (their data pointers are passed through).  Outputs come back as
numpy arrays unless a device output is requested.  If ``liblds.so`` has not been
built, :func:`load` raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblds.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW, EBUSY = range(7)
STATUS_NAMES = {0: "LDS_OK", 1: "LDS_EINVAL", 2: "LDS_ENOMEM", 3: "LDS_ECUDA", 4: "LDS_ETIMEOUT",
                5: "LDS_EOVERFLOW", 6: "LDS_EBUSY"}
DENSITY = {"edge": 0, "triangle": 1}
PRECISION = {"exact": 0, "fp64": 1, "fp32": 2}
VERIFY = {"bounds": 0, "core": 1, "whole": 2}
MEM_HOST, MEM_DEVICE = 0, 1

_lib = None


class LdsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("input_pairs", ctypes.c_int64),
                ("self_loops", ctypes.c_int64), ("duplicates", ctypes.c_int64), ("max_degree", ctypes.c_int32),
                ("isolated", ctypes.c_int32), ("triangles", ctypes.c_int64)]


class FwResult(ctypes.Structure):
    _fields_ = [("r", ctypes.c_void_p), ("R", ctypes.c_void_p), ("W", ctypes.c_void_p),
                ("last", ctypes.c_void_p), ("D", ctypes.c_int64)]


class LdsResult(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("dens_num", ctypes.POINTER(ctypes.c_int64)),
                ("dens_den", ctypes.POINTER(ctypes.c_int64)), ("offsets", ctypes.POINTER(ctypes.c_int64)),
                ("vertices", ctypes.POINTER(ctypes.c_int32))]


class TopkStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("fw_rounds", "fw_edge_updates", "certified", "failed", "refined",
                                              "exact_settled", "skipped_by_bound", "flows", "denser_neighbour")] + \
               [(f, ctypes.c_double) for f in ("ms_total", "ms_fw", "ms_extract", "ms_prune", "ms_verify")]


class Query(ctypes.Structure):
    _fields_ = [("g", ctypes.c_void_p), ("k", ctypes.c_int32), ("d", ctypes.c_int), ("iters", ctypes.c_int32),
                ("p", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("include_zero_density", ctypes.c_int32),
                ("verify", ctypes.c_int)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("footprint_bytes", ctypes.c_int64),
                ("stats", TopkStats)]


def _sig(lib, name, res, args):
    fn = getattr(lib, name)
    fn.restype = res
    fn.argtypes = args
    return fn


def load():
    """Loads liblds.so (once).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    _sig(lib, "lds_version", ctypes.c_char_p, [])
    _sig(lib, "lds_last_error", ctypes.c_char_p, [])
    _sig(lib, "lds_device_count", i32, [])
    _sig(lib, "lds_create_graph", ctypes.c_int, [i32, i64, P, P, ctypes.c_int, P, ctypes.POINTER(P)])
    _sig(lib, "lds_free", None, [P])
    _sig(lib, "lds_graph_info", ctypes.c_int, [P, ctypes.POINTER(GraphInfo)])
    _sig(lib, "lds_get_edges", ctypes.c_int, [P, P, P, ctypes.c_int])
    _sig(lib, "lds_list_triangles", ctypes.c_int, [P, ctypes.POINTER(i64)])
    _sig(lib, "lds_get_triangles", ctypes.c_int, [P, P, ctypes.c_int])
    _sig(lib, "lds_core_numbers", ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int])
    _sig(lib, "lds_compact_numbers", ctypes.c_int, [P, ctypes.c_int, P, P, ctypes.c_int])
    _sig(lib, "lds_fw", ctypes.c_int, [P, ctypes.c_int, i32, ctypes.c_int, ctypes.c_int, ctypes.POINTER(FwResult)])
    _sig(lib, "lds_fw_last_timing", ctypes.c_int, [P, ctypes.POINTER(ctypes.c_double),
                                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                                   ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_char_p)])
    _sig(lib, "lds_set_pass_profiling", None, [i32])
    _sig(lib, "lds_debug_fail_alloc_after", None, [i32])
    _sig(lib, "lds_launch_count", i64, [])
    _sig(lib, "lds_set_fw_variant", ctypes.c_int, [i32])
    _sig(lib, "lds_set_flow_variant", ctypes.c_int, [i32])
    _sig(lib, "lds_set_extract_variant", ctypes.c_int, [i32])
    _sig(lib, "lds_pattern_max_flow", ctypes.c_int, [i32, i32, P, P, i64, i64, ctypes.POINTER(i64), P])
    _sig(lib, "lds_prune", ctypes.c_int, [P, ctypes.c_int, P, P, P, P, P])
    _sig(lib, "lds_topk", ctypes.c_int, [P, i32, ctypes.c_int, i32, ctypes.c_int,
                                         ctypes.POINTER(ctypes.POINTER(LdsResult))])
    _sig(lib, "lds_topk_ex", ctypes.c_int, [P, i32, ctypes.c_int, i32, ctypes.POINTER(Options),
                                            ctypes.POINTER(ctypes.POINTER(LdsResult))])
    _sig(lib, "lds_result_free", None, [ctypes.POINTER(LdsResult)])
    _sig(lib, "lds_topk_last_stats", ctypes.c_int, [ctypes.POINTER(TopkStats)])
    _sig(lib, "lds_extract_sg", ctypes.c_int, [P, P, ctypes.POINTER(i32), P, P, P, ctypes.POINTER(i64),
                                               ctypes.POINTER(i32), P])
    _sig(lib, "lds_fw_state", ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(FwResult)])
    _sig(lib, "lds_fw_batch", ctypes.c_int, [i32, ctypes.POINTER(P), i32, ctypes.c_int, ctypes.POINTER(i32)])
    _sig(lib, "lds_server_create", ctypes.c_int, [i64, i32, ctypes.POINTER(P)])
    _sig(lib, "lds_server_submit", ctypes.c_int, [P, ctypes.POINTER(Query), ctypes.POINTER(i64)])
    _sig(lib, "lds_server_poll", ctypes.c_int, [P, i64, ctypes.POINTER(i32)])
    _sig(lib, "lds_server_wait", ctypes.c_int, [P, i64, ctypes.POINTER(ctypes.POINTER(LdsResult)),
                                                ctypes.POINTER(RequestInfo)])
    _sig(lib, "lds_server_destroy", None, [P])
    _sig(lib, "lds_topk_batch", ctypes.c_int, [i32, ctypes.POINTER(Query), i32,
                                               ctypes.POINTER(ctypes.POINTER(LdsResult)), ctypes.POINTER(ctypes.c_int)])
    _sig(lib, "lds_batch_autotune", ctypes.c_int, [i32, ctypes.POINTER(Query), ctypes.POINTER(i32)])
    _sig(lib, "lds_fw_batch_threads", i32, [i32])
    _sig(lib, "lds_debug_pick_next", i32, [i32, P, P, i64])
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        raise LdsError(status, load().lds_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())      # torch tensor


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def version() -> str:
    return load().lds_version().decode()


def device_count() -> int:
    return int(load().lds_device_count())


def set_pass_profiling(on: bool):
    load().lds_set_pass_profiling(1 if on else 0)


def set_fw_variant(variant: int):
    """0: automatic; 1-6 force one kernel form (lds_set_fw_variant in include/lds.h)."""
    _check(load().lds_set_fw_variant(int(variant)))


def set_flow_variant(variant: int):
    """0: automatic; 1: pattern-node push-relabel; 2: vertex-node phases."""
    _check(load().lds_set_flow_variant(int(variant)))


def set_extract_variant(variant: int):
    """0: automatic; 1: the large-graph ExtractSG walk (device chains) at every size."""
    _check(load().lds_set_extract_variant(int(variant)))


def launch_count() -> int:
    return int(load().lds_launch_count())


def debug_fail_alloc_after(k: int):
    load().lds_debug_fail_alloc_after(int(k))


def pattern_max_flow(nv: int, patterns, p: int, q: int):
    """Alg. 8's network over vertices 0..nv-1 and the given patterns (sequences
    of vertex indices).  Returns (flow, source_side uint8[nv])."""
    ptr = np.zeros(len(patterns) + 1, dtype=np.int64)
    for j, pat in enumerate(patterns):
        ptr[j + 1] = ptr[j] + len(pat)
    idx = np.array([x for pat in patterns for x in pat], dtype=np.int32)
    if idx.size == 0:
        idx = np.zeros(1, dtype=np.int32)
    side = np.zeros(max(nv, 1), dtype=np.uint8)
    f = ctypes.c_int64()
    _check(load().lds_pattern_max_flow(int(nv), len(patterns), _ptr(ptr), _ptr(idx), int(p), int(q),
                                       ctypes.byref(f), _ptr(side)))
    return int(f.value), side[:nv]


def _result_list(res):
    """lds_result -> list of (Fraction density, int32 member array)."""
    from fractions import Fraction
    r = res.contents
    out = []
    if r.count:
        total = r.offsets[r.count]
        verts = np.ctypeslib.as_array(r.vertices, shape=(max(total, 1),))[:total].copy()
        for i in range(r.count):
            out.append((Fraction(r.dens_num[i], r.dens_den[i]), verts[r.offsets[i]:r.offsets[i + 1]]))
    return out


def _query(g, k: int, density: str, iters: int, precision: str) -> Query:
    return Query(g.handle, int(k), DENSITY[density], int(iters), PRECISION[precision])


def debug_pick_next(bytes_, busy, free_bytes: int) -> int:
    """The serving loop's admission rule (see lds_debug_pick_next)."""
    b = np.ascontiguousarray(bytes_, dtype=np.int64)
    f = np.ascontiguousarray(busy, dtype=np.uint8)
    return int(load().lds_debug_pick_next(len(b), _ptr(b), _ptr(f), int(free_bytes)))


def topk_batch(queries, workers: int = 0):
    """Runs queries [(graph, k, density, iters, precision), ...] together
    (lds_topk_batch).  Returns one result list per query, as Graph.topk."""
    lib = load()
    qs = (Query * max(len(queries), 1))(*[_query(*q) for q in queries])
    res = (ctypes.POINTER(LdsResult) * max(len(queries), 1))()
    sts = (ctypes.c_int * max(len(queries), 1))()
    st = lib.lds_topk_batch(len(queries), qs, int(workers), res, sts)
    try:
        _check(st)
        return [_result_list(res[i]) for i in range(len(queries))]
    finally:
        for i in range(len(queries)):
            if res[i]:
                lib.lds_result_free(res[i])


def fw_batch(graphs, iters: int, precision: str = "exact") -> int:
    """Edge-density Frank-Wolfe on many graphs (lds_fw_batch); returns how
    many ran in the on-chip persistent launch."""
    hs = (ctypes.c_void_p * max(len(graphs), 1))(*[g.handle.value for g in graphs])
    on = ctypes.c_int32()
    _check(load().lds_fw_batch(len(graphs), hs, int(iters), PRECISION[precision], ctypes.byref(on)))
    return int(on.value)


def fw_batch_threads(nact: int) -> int:
    """Threads per graph of the persistent batched FW launch for graphs of nact
    active vertices (the autotuned choice of their size bucket, else 1024)."""
    return int(load().lds_fw_batch_threads(int(nact)))


def batch_autotune(queries) -> int:
    qs = (Query * max(len(queries), 1))(*[_query(*q) for q in queries])
    w = ctypes.c_int32()
    _check(load().lds_batch_autotune(len(queries), qs, ctypes.byref(w)))
    return int(w.value)


class Server:
    """The serving loop (lds_server_*): submit() queues a query and returns a
    ticket at once; wait() blocks for its result and timing."""

    def __init__(self, budget_bytes: int, workers: int):
        h = ctypes.c_void_p()
        _check(load().lds_server_create(int(budget_bytes), int(workers), ctypes.byref(h)))
        self._h = h

    def submit(self, g, k: int, density: str = "edge", iters: int = 100, precision: str = "exact") -> int:
        q = _query(g, k, density, iters, precision)
        t = ctypes.c_int64()
        _check(load().lds_server_submit(self._h, ctypes.byref(q), ctypes.byref(t)))
        return int(t.value)

    def done(self, ticket: int) -> bool:
        d = ctypes.c_int32()
        _check(load().lds_server_poll(self._h, int(ticket), ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int):
        lib = load()
        res = ctypes.POINTER(LdsResult)()
        info = RequestInfo()
        st = lib.lds_server_wait(self._h, int(ticket), ctypes.byref(res), ctypes.byref(info))
        try:
            _check(st)
            timing = {"queue_ms": info.queue_ms, "run_ms": info.run_ms, "footprint_bytes": info.footprint_bytes,
                      "stats": {f: getattr(info.stats, f) for f, _ in TopkStats._fields_}}
            return _result_list(res), timing
        finally:
            if res:
                lib.lds_result_free(res)

    def close(self):
        if self._h is not None:
            load().lds_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def topk_last_stats() -> dict:
    st = TopkStats()
    _check(load().lds_topk_last_stats(ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in TopkStats._fields_}


class Graph:
    """A graph handle (``lds_graph``).  ``src`` / ``dst`` are int32 numpy arrays
    (host) or int32 torch CUDA tensors (device).  ``stream`` is a raw
    cudaStream_t value (e.g. ``torch.cuda.current_stream().cuda_stream``)."""

    def __init__(self, n: int, src, dst, stream: int | None = None):
        lib = load()
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.int32)
            dst = np.ascontiguousarray(dst, dtype=np.int32)
            where = MEM_HOST
        else:
            where = MEM_DEVICE if _is_device(src) else MEM_HOST
        m = len(src)
        h = ctypes.c_void_p()
        self._h = None
        self.stream = stream
        _check(lib.lds_create_graph(int(n), int(m), _ptr(src), _ptr(dst), where,
                                    ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
        self._h = h
        info = self.info()
        self.n = info["n"]
        self.m = info["m"]

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None:
            load().lds_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self) -> dict:
        gi = GraphInfo()
        _check(load().lds_graph_info(self._h, ctypes.byref(gi)))
        return {f: getattr(gi, f) for f, _ in GraphInfo._fields_}

    def edges(self):
        u = np.empty(self.m, dtype=np.int32)
        v = np.empty(self.m, dtype=np.int32)
        _check(load().lds_get_edges(self._h, _ptr(u), _ptr(v), MEM_HOST))
        return u, v

    def list_triangles(self) -> int:
        c = ctypes.c_int64()
        _check(load().lds_list_triangles(self._h, ctypes.byref(c)))
        return int(c.value)

    def triangles(self):
        t = self.list_triangles()
        out = np.empty((t, 3), dtype=np.int32)
        _check(load().lds_get_triangles(self._h, _ptr(out), MEM_HOST))
        return out

    def core_numbers(self, density: str = "edge"):
        out = np.empty(self.n, dtype=np.int64)
        _check(load().lds_core_numbers(self._h, DENSITY[density], _ptr(out), MEM_HOST))
        return out

    def compact_numbers(self, density: str = "edge"):
        """Exact compact numbers (tr-compact for "triangle"): (num, den) int64
        arrays over the vertices, reduced fractions."""
        num = np.empty(self.n, dtype=np.int64)
        den = np.empty(self.n, dtype=np.int64)
        _check(load().lds_compact_numbers(self._h, DENSITY[density], _ptr(num), _ptr(den), MEM_HOST))
        return num, den

    def fw(self, iters: int, density: str = "edge", precision: str = "exact",
           want=("r", "R", "W", "last")):
        """Frank-Wolfe (Alg. 1 / Alg. 6).  Returns a dict with the requested
        arrays (host numpy) and the denominator D."""
        n = self.n
        npat = self.m if density == "edge" else (self.list_triangles() if "W" in want or "last" in want else 0)
        res = FwResult()
        out = {}
        if "r" in want:
            out["r"] = np.empty(n, dtype=np.float64)
            res.r = out["r"].ctypes.data
        if "R" in want:
            out["R"] = np.empty(n, dtype=np.int64)
            res.R = out["R"].ctypes.data
        if "W" in want:
            shape = (npat,) if density == "edge" else (npat, 3)
            out["W"] = np.empty(shape, dtype=np.int64)
            res.W = out["W"].ctypes.data
        if "last" in want:
            out["last"] = np.empty(npat, dtype=np.uint8)
            res.last = out["last"].ctypes.data
        _check(load().lds_fw(self._h, DENSITY[density], int(iters), PRECISION[precision], MEM_HOST,
                             ctypes.byref(res)))
        out["D"] = int(res.D)
        return out

    def fw_state(self):
        """The handle's current Frank-Wolfe state (edge density): r, R, W, D."""
        out = {"r": np.empty(self.n, dtype=np.float64), "R": np.empty(self.n, dtype=np.int64),
               "W": np.empty(max(self.m, 1), dtype=np.int64)}
        res = FwResult()
        res.r = out["r"].ctypes.data
        res.R = out["R"].ctypes.data
        res.W = out["W"].ctypes.data
        _check(load().lds_fw_state(self._h, MEM_HOST, ctypes.byref(res)))
        out["W"] = out["W"][:self.m]
        out["D"] = int(res.D)
        return out

    def topk(self, k: int, density: str = "edge", iters: int = 100, precision: str = "exact",
             verify: str | None = None, include_zero: bool = False, stream: int | None = None):
        """Top-k LDSs (edge) or LTDSs (triangle): list of (Fraction density,
        int32 array of member ids ascending), densest first.  With any of
        verify ("bounds", "core", "whole"), include_zero or stream given, the
        call goes through lds_topk_ex."""
        lib = load()
        res = ctypes.POINTER(LdsResult)()
        if verify is None and not include_zero and stream is None:
            _check(lib.lds_topk(self._h, int(k), DENSITY[density], int(iters), PRECISION[precision],
                                ctypes.byref(res)))
        else:
            opt = Options(PRECISION[precision], stream, 1 if include_zero else 0, VERIFY[verify or "bounds"])
            _check(lib.lds_topk_ex(self._h, int(k), DENSITY[density], int(iters), ctypes.byref(opt),
                                   ctypes.byref(res)))
        try:
            return _result_list(res)
        finally:
            lib.lds_result_free(res)

    def extract_sg(self):
        """Stable groups (Alg. 2) of the last fw() run on this graph.  Returns a
        dict: order (vertices by load, original ids), groups (list of vertex
        arrays, top first), remainder (vertices after the last group),
        intervals (list of (lo_num, hi_num) over D), D and cuts (1-based)."""
        n = self.n
        order = np.empty(max(n, 1), dtype=np.int32)
        gend = np.empty(max(n, 1), dtype=np.int64)
        lo = np.empty(max(n, 1), dtype=np.int64)
        hi = np.empty(max(n, 1), dtype=np.int64)
        cuts = np.empty(max(n, 1), dtype=np.int64)
        ng, nc, D = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(load().lds_extract_sg(self._h, _ptr(order), ctypes.byref(ng), _ptr(gend), _ptr(lo), _ptr(hi),
                                     ctypes.byref(D), ctypes.byref(nc), _ptr(cuts)))
        order = order[:n]
        groups, start = [], 0
        for k in range(ng.value):
            groups.append(order[start:gend[k]])
            start = int(gend[k])
        return {"order": order, "groups": groups, "remainder": order[start:],
                "intervals": list(zip(lo[:ng.value].tolist(), hi[:ng.value].tolist())),
                "D": int(D.value), "cuts": cuts[:nc.value].tolist()}

    def prune(self, ub, lb, density: str = "edge"):
        """Alg. 3 with bounds given as sequences of fractions.Fraction (or ints)
        indexed by vertex.  Returns uint8[n]: 0 kept, 1 rule 1, 2 rule 2."""
        from fractions import Fraction
        n = self.n
        arrs = []
        for b in (ub, lb):
            fr = [Fraction(x) for x in b]
            arrs.append(np.array([f.numerator for f in fr], dtype=np.int64))
            arrs.append(np.array([f.denominator for f in fr], dtype=np.int64))
        st = np.empty(max(n, 1), dtype=np.uint8)
        _check(load().lds_prune(self._h, DENSITY[density], _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]),
                                _ptr(arrs[3]), _ptr(st)))
        return st[:n]

    def fw_timing(self):
        a, b, c, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        k = ctypes.c_char_p()
        _check(load().lds_fw_last_timing(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                         ctypes.byref(d), ctypes.byref(k)))
        return {"fw_ms": a.value, "pass_us": b.value, "pass_launches": int(c.value),
                "pass_bytes": int(d.value), "pass_kernel": (k.value or b"").decode()}

"""Benchmark: Frank-Wolfe edge-updates per second and top-k LDS queries per
second on the power-law workload.

Workload: Chung-Lu graph with n = 1,000,000 vertices, 10,000,000 background
edges (degree exponent 2.1) plus 50 planted blocks of log-uniform size 50-500
and edge probability U(0.3, 0.9) (about 10.6M edges in all), delivered as a raw
edge list (random orientation and order, 5% repeated pairs, 1% self-loops)
already resident in device memory.

One step = one top-10 LDS query over that input through the library: graph
ingest (canonical edges + CSR), initial reduction, Frank-Wolfe (Alg. 1, 500
iterations per round), ExtractSG, Pruning, IsDensest / IsLDS max-flow
verification and the refinement rounds of the driver.  value = Frank-Wolfe
edge-updates executed in the step / step time (whole step, not only the FW
kernels; the FW-only rate is reported beside it).  L2 is flushed between steps
(a 512 MiB device write outside the per-step events).

``--impl reference`` times the CPU oracle (oracle.fw) on the host cores on a
bounded number of iterations of the same graph and reports the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_10937_gb300 import synth  # noqa: E402

METRIC = "FW edge-updates/s"
UNIT = "edge-updates/s"
METRIC_TRI = "FW triangle-updates/s"
UNIT_TRI = "triangle-updates/s"

# DRAM bytes (read + write) per iteration of the FW kernel on this workload, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by
# the kernel, the arithmetic and a digest of the source file the kernel was built
# from at capture time.  A kernel whose source changed since has no matching entry
# and reports null.
PASS_TRAFFIC = {
    # one 20-iteration launch on the 1M-vertex workload (64,239,872 B read + 4,828,928 B
    # written, the cold first read of the view included), per iteration
    ("fw_coop32_kernel", "exact", "1df8d6eea5f0f836"): 3453440,
}
PASS_SOURCE = {"fw_opass32_kernel": "paper_2504_10937_gb300/csrc/fw_oriented.cu",
               "fw_coop32_kernel": "paper_2504_10937_gb300/csrc/fw_oriented.cu",
               "fw_tri_pass_kernel": "paper_2504_10937_gb300/csrc/fw.cu"}
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _source_digest(kernel: str):
    import hashlib
    path = PASS_SOURCE.get(kernel)
    if not path or not os.path.exists(os.path.join(ROOT, path)):
        return None
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _traffic(kernel: str, precision: str):
    return PASS_TRAFFIC.get((kernel, precision, _source_digest(kernel)))


def _host():
    """Host CPU description: logical cores and the model name lscpu reports."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def _golden_sets(name):
    """Expected sets written by tests/golden/make_topk_golden.py, or None."""
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        return None
    out = []
    with open(path) as f:
        for ln in f:
            ln = ln.split("#")[0].strip()
            if ln:
                d, vs = ln.split(":")
                out.append((d.strip(), tuple(int(x) for x in vs.split(","))))
    return out


def _fw_sample(name):
    """Oracle FW values on a vertex sample (tests/golden/make_fw_sample.py): ids, R, r64."""
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        return None
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return (np.array([int(r[0]) for r in rows]), [int(r[1]) for r in rows],
            np.array([float(r[2]) for r in rows]))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


WORKLOADS = {
    # power-law: top-10 LDS, 500 iterations, exact arithmetic
    "chung_lu_1m": dict(density="edge", k=10, iters=500, precision="exact", seed=2, scramble=20,
                        desc="chung_lu_n1e6_m1e7_exp2.1_50blocks (seed 2), raw COO with 5% repeats and 1% self-loops"),
    # R-MAT scale 20: top-5 LTDS, 300 iterations, binary32 loads; includes triangle listing
    "rmat20": dict(density="triangle", k=5, iters=300, precision="fp32", seed=3, scramble=30,
                   desc="rmat_scale20_ef16_(0.57,0.19,0.19)_20cliques_30-200_p0.8 (seed 3), raw COO with 5% "
                        "repeats and 1% self-loops; triangle listing inside the step"),
}


def _workload(args):
    """The seeded input; cached under the system temp directory between runs
    of this script on the same machine (the cache holds generator output only)."""
    import tempfile
    spec = WORKLOADS[args.workload]
    path = os.path.join(tempfile.gettempdir(), f"lds_bench_{args.workload}_seed{spec['seed']}.npz")
    if os.path.exists(path):
        d = np.load(path)
        return int(d["n"]), d["u"], d["v"], d["a"], d["b"]
    if args.workload == "rmat20":
        n, u, v, blocks = synth.workload_rmat20(seed=spec["seed"])
    else:
        n, u, v, blocks = synth.workload_chung_lu_1m(seed=spec["seed"])
    a, b = synth.scramble(n, u, v, seed=spec["scramble"])
    try:
        np.savez(path, n=n, u=u, v=v, a=a, b=b)
    except OSError:
        pass
    return n, u, v, a, b


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def job_rate(total_ms: float, units: int, device=None):
    """Whole-job rate over the ranks of the process group (if any): the units of
    every rank summed, over the slowest rank's time.  Returns (rate per second,
    job ms, job units)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units / (total_ms / 1000.0), total_ms, units
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) / 1000.0), float(t.item()), int(u.item())


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The CPU oracle timed on the host cores (bounded sample)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import fw as ofw
    n, u, v, a, b = _workload(args)
    u64 = u.astype(np.int64)
    v64 = v.astype(np.int64)
    m = len(u)
    tri = args.density == "triangle"
    if tri:
        tris, nsamp = _tri_sample(n, u, v)
        units = len(tris)
        sample = (f"{args.ref_iters} exact triangle FW iterations per step on the {units} triangles induced by "
                  f"the vertices with id < {nsamp} (listing untimed)")
    else:
        units = m
        sample = f"{args.ref_iters} exact FW iterations per step on the full graph (m={m})"
    iters_per_step = args.ref_iters
    times = []
    R, W = None, None
    i = 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        if tri:
            R, W, _, _ = ofw.fw_tri_exact(nsamp, tris, i + iters_per_step, R0=R, W0=W, i0=i)
        else:
            R, W, _, _ = ofw.fw_edge_exact(n, u64, v64, i + iters_per_step, R0=R, W0=W, i0=i)
        dt = time.perf_counter() - t0
        i += iters_per_step
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = units * iters_per_step * len(times) / total
    unit = UNIT_TRI if tri else UNIT
    line = {
        "impl": "reference", "metric": METRIC_TRI if tri else METRIC, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": _config(args, n, m),
        "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "host": _host(),
                         "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(args, n, m):
    tri = args.density == "triangle"
    return {"workload": WORKLOADS[args.workload]["desc"],
            "n": n, "m": m, "iters": args.iters, "precision": args.precision, "density": args.density, "k": args.k,
            "step": ("ingest + Frank-Wolfe" if getattr(args, "fw_only", False)
                     else f"top-k {'LTDS' if tri else 'LDS'} query (lds_topk)"),
            "l2": "flushed between steps (512 MiB device write)", "parallelism": f"replicas x{args.gpus}"}


def cpu_baseline(n, u, v, budget_s=12.0):
    from oracle import fw as ofw
    u64 = u.astype(np.int64)
    v64 = v.astype(np.int64)
    t0 = time.perf_counter()
    R, W, _, _ = ofw.fw_edge_exact(n, u64, v64, 1)
    one = time.perf_counter() - t0
    iters = max(1, int(budget_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    ofw.fw_edge_exact(n, u64, v64, 1 + iters, R0=R, W0=W, i0=1)
    dt = time.perf_counter() - t0
    return {"value": len(u) * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host(),
            "sample": f"{iters} exact FW iterations (iterations 2..{iters + 1}) of the oracle on the full graph"}


def _tri_sample(n, u, v):
    """Triangles of the subgraph induced by the vertices with id < n / 8 (ids are
    randomly relabelled, so this is a seeded random vertex sample), listed by the
    oracle; listing all triangles of the full graph is far beyond a bounded sample."""
    from oracle.graph import triangles
    lim = max(1, n // 8)
    keep = (u < lim) & (v < lim)
    return triangles(lim, u[keep].astype(np.int64), v[keep].astype(np.int64)), lim


def cpu_baseline_tri(n, u, v, budget_s=12.0):
    """The oracle's exact triangle FW (Alg. 6) on the host, on the triangles of
    a vertex sample (listing not timed), for a bounded number of iterations."""
    from oracle import fw as ofw
    tris, lim = _tri_sample(n, u, v)
    n = lim
    t0 = time.perf_counter()
    R, W, _, _ = ofw.fw_tri_exact(n, tris, 1)
    one = time.perf_counter() - t0
    iters = max(1, int(budget_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    ofw.fw_tri_exact(n, tris, 1 + iters, R0=R, W0=W, i0=1)
    dt = time.perf_counter() - t0
    return {"value": len(tris) * iters / dt, "unit": UNIT_TRI, "cores": 1, "kind": "oracle", "host": _host(),
            "sample": f"{iters} exact triangle FW iterations of the oracle on the {len(tris)} triangles induced "
                      f"by the vertices with id < {lim}"}


def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2504_10937_gb300 import lds
    lds.load()
    n, u, v, a, b = _workload(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    ta = torch.from_numpy(a).to(dev)
    tb = torch.from_numpy(b).to(dev)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    m_holder = {}

    def step():
        g = lds.Graph(n, ta, tb, stream=sptr)
        m_holder["m"] = g.m
        if args.fw_only:
            g.fw(args.iters, density=args.density, precision=args.precision, want=())
            st = {"fw_edge_updates": (g.m if args.density == "edge" else g.list_triangles()) * args.iters}
        else:
            m_holder["result"] = g.topk(args.k, args.density, args.iters, args.precision)
            st = lds.topk_last_stats()
        m_holder["units"] = g.m if args.density == "edge" else g.list_triangles()
        t = g.fw_timing()
        g.close()
        t["stats"] = st
        return t

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    # the timed steps run without per-pass events (lds_set_pass_profiling stays off)
    lds.set_pass_profiling(False)
    times, fw_ms, updates, phase = [], [], [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = lds.launch_count()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            fw_ms.append(t["fw_ms"])
            updates.append(t["stats"]["fw_edge_updates"])
            phase.append(t["stats"])
            flush.zero_()
        torch.cuda.synchronize()
    launches = lds.launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    m = m_holder["m"]
    value, total_ms, units = job_rate(sum(times), sum(updates), dev)

    # roofline of the pass kernel: one more first-round FW on the same input, untimed
    # as a step, with a CUDA event pair around every pass launch on the handle's stream
    lds.set_pass_profiling(True)
    g = lds.Graph(n, ta, tb, stream=sptr)
    g.fw(args.iters, density=args.density, precision=args.precision, want=())
    pass_timing = g.fw_timing()
    g.close()
    lds.set_pass_profiling(False)
    flush.zero_()

    # end to end through the C-ABI with host (pinned) buffers
    ha = torch.from_numpy(a).pin_memory()
    hb = torch.from_numpy(b).pin_memory()
    e2e_times = []
    for k in range(0 if args.no_e2e else max(2, args.steps // 2) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = lds.Graph(n, ha.numpy(), hb.numpy(), stream=sptr)
        if args.fw_only:
            g.fw(args.iters, density=args.density, precision=args.precision, want=("r",))
            e2e_updates = m_holder["units"] * args.iters
        else:
            g.topk(args.k, args.density, args.iters, args.precision)
            e2e_updates = lds.topk_last_stats()["fw_edge_updates"]
        g.close()
        dt = time.perf_counter() - t0
        if k:
            e2e_times.append(dt)
        flush.zero_()
    e2e_value = e2e_updates / statistics.mean(e2e_times) if e2e_times else None

    plain = precision = answer = None
    if not args.fw_only and rank == 0 and args.workload == "chung_lu_1m":
        want = _golden_sets("chung_lu_1m_top10.txt")
        got = [(str(d), tuple(int(x) for x in c)) for d, c in m_holder["result"]]
        answer = {"golden": "tests/golden/chung_lu_1m_top10.txt (oracle.ldscvx, exact)",
                  "matches_oracle": None if want is None else got == want[:args.k]}
    if not args.fw_only and not args.no_plain:
        # the plain single-graph binary64 GPU path (Alg. 1 literally) on the same query
        pt = []
        for k in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = lds.Graph(n, ta, tb, stream=sptr)
            res64 = g.topk(args.k, args.density, args.iters, "fp64")
            g.close()
            torch.cuda.synchronize()
            if k:
                pt.append(time.perf_counter() - t0)
            flush.zero_()
        plain = {"precision": "fp64 (Alg. 1 literal, symmetric slots)", "queries_per_s": 1.0 / statistics.mean(pt),
                 "ms_per_query": 1000.0 * statistics.mean(pt), "same_output": _sets(res64) == _sets(m_holder["result"])}
    if not args.fw_only and not args.no_precision and args.workload == "chung_lu_1m":
        precision = precision_pattern(args, lds, n, ta, tb, sptr, flush, m_holder["result"])

    hbm, peak_kind = _peaks()
    # algorithmic bytes of one pass: per edge 16 B in EXACT and FP32 (8 B of ids, 8 B of
    # alpha read-modify-write) and 24 B in FP64; per triangle 28 B (12 B of ids, two
    # stored alphas read and written) and 44 B in FP64.  The kernels themselves move
    # fewer (kernel_bytes): one choice bit per unit instead of alpha
    tri = args.density == "triangle"
    units = m_holder["units"]
    per_unit = ({"exact": 28, "fp32": 28, "fp64": 44} if tri else {"exact": 16, "fp32": 16, "fp64": 24})[args.precision]
    bytes_per_pass = per_unit * units
    fused = pass_timing["pass_kernel"] == "fw_coop32_kernel"
    if fused:
        # the cooperative kernel runs whole iterations: the pass and the vertex
        # update (16 B per vertex), timed per launch and divided by the iterations
        bytes_per_pass += 16 * n
    avg_pass_us = pass_timing["pass_us"]
    achieved = bytes_per_pass / (avg_pass_us * 1e-6) / 1e9
    # one whole iteration: the pass plus the vertex update (16 B per vertex)
    iter_us = 1000.0 * pass_timing["fw_ms"] / args.iters
    iter_bytes = bytes_per_pass + 16 * n
    clocks = clk.summary()
    lat = sorted(times)

    def pct(q):
        return lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    if rank == 0:
        line = {
            "metric": METRIC_TRI if tri else METRIC, "value": value, "unit": UNIT_TRI if tri else UNIT,
            "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"exact": "int64", "fp32": "f32", "fp64": "f64"}[args.precision],
            "data": "synthetic", "config": _config(args, n, m),
            "fw_only": {"value": units * args.iters / (statistics.mean(fw_ms) / 1000.0),
                        "unit": UNIT_TRI if tri else UNIT,
                        "fw_ms": statistics.mean(fw_ms), "note": "first-round FW kernels on G only"},
            "queries_per_s": None if args.fw_only else 1000.0 * args.steps / total_ms,
            "latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "n": len(lat)},
            "plain_fp64_gpu": plain,
            "precision_pattern": precision,
            "answer": answer,
            "phases_ms": None if args.fw_only else {k: statistics.mean(p[k] for p in phase)
                                                     for k in ("ms_total", "ms_fw", "ms_extract", "ms_prune",
                                                               "ms_verify")},
            "result": None if args.fw_only else [[str(d), len(c)] for d, c in m_holder["result"]],
            "roofline": {"bound": "hbm", "kernel": pass_timing["pass_kernel"], "achieved": achieved, "peak": hbm,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": _traffic(pass_timing["pass_kernel"], args.precision),
                         "algorithmic_bytes_per_launch": bytes_per_pass,
                         ("bytes_per_triangle" if tri else "bytes_per_edge"): per_unit, "units_per_launch": units,
                         "kernel_bytes_per_launch": pass_timing["pass_bytes"], "avg_launch_us": avg_pass_us,
                         "launches_timed": pass_timing["pass_launches"],
                         "timed": ("CUDA events around every launch of one extra first-round FW run (outside "
                                   "the headline steps); " + ("each launch runs many whole iterations (pass + "
                                   "vertex update), the figures are per iteration" if fused else
                                   "one launch per pass")),
                         "iteration": {"us": iter_us, "algorithmic_bytes": iter_bytes,
                                       "frac": iter_bytes / (iter_us * 1e-6) / 1e9 / hbm,
                                       "note": "whole FW iteration: pass + vertex update (+ folds), "
                                               f"{per_unit} B/{'triangle' if tri else 'edge'} + 16 B/vertex"}},
            "e2e": {"value": e2e_value, "unit": UNIT_TRI if tri else UNIT, "h2d_bytes_per_step": int(2 * 4 * len(a)),
                    "d2h_bytes_per_step": int(8 * n)},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(n, u, v) if not tri else cpu_baseline_tri(n, u, v)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def precision_pattern(args, lds, n, ta, tb, sptr, flush, exact_result):
    """The binary32 form on the same query: its time and answer, and the error of
    its r vector after `iters` iterations against the binary64 oracle (Alg. 1
    carried literally in binary64) on the oracle's vertex sample."""
    import torch
    qt = []
    for k in range(3):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        g = lds.Graph(n, ta, tb, stream=sptr)
        e0.record(torch.cuda.current_stream())
        res32 = g.topk(args.k, "edge", args.iters, "fp32")
        e1.record(torch.cuda.current_stream())
        e1.synchronize()
        g.close()
        if k:
            qt.append(e0.elapsed_time(e1))
        flush.zero_()
    out = {"fp32_query_ms": statistics.mean(qt), "fp32_same_sets_as_exact": _sets(res32) == _sets(exact_result)}
    sample = _fw_sample("chung_lu_1m_fw500_sample.txt")
    if sample is None or args.iters != 500:
        out["r_error"] = None
        return out
    ids, Rq, r64 = sample
    with lds.Graph(n, ta, tb, stream=sptr) as g:
        ex = g.fw(args.iters, precision="exact", want=("R",))
        f32 = g.fw(args.iters, precision="fp32", want=("r",))
        f64 = g.fw(args.iters, precision="fp64", want=("r",))
    Dn = ex["D"]
    exact_r = np.array([float(q) / Dn for q in Rq])

    def rel(a):
        return float(np.max(np.abs(a - r64) / np.maximum(np.abs(r64), 1e-300)))
    out["r_error"] = {
        "sample": f"{len(ids)} vertices (2,000 seeded + the 48 highest-degree), oracle values from "
                  "tests/golden/make_fw_sample.py",
        "exact_R_bit_exact": [int(x) for x in ex["R"][ids]] == Rq,
        "fp64_max_rel_err_vs_fp64_oracle": rel(f64["r"][ids]),
        "fp32_max_rel_err_vs_fp64_oracle": rel(f32["r"][ids]),
        "exact_max_rel_err_vs_fp64_oracle": rel(exact_r),
        "note": "free-running forms: one tie decided differently forks the trajectory, so the FP32 error "
                "is stated, not gated (the FP32 rounding itself is checked bit for bit against the oracle's "
                "binary32 form in tests/test_gpu_core.py)",
    }
    return out


def _sets(res):
    return [(str(d), tuple(int(x) for x in c)) for d, c in res]


def run_batch(args):
    """Many small graphs in one batch (lds_topk_batch), against the same
    queries run one at a time in binary64 (the plain path)."""
    import torch
    from paper_2504_10937_gb300 import lds
    torch.cuda.set_device(0)
    lds.load()
    t0 = time.perf_counter()
    mix = synth.batched_mix(args.graphs, seed=4)
    gen_s = time.perf_counter() - t0
    graphs = [lds.Graph(g["n"], g["u"].astype(np.int32), g["v"].astype(np.int32)) for g in mix]
    queries = [(g, 3, "triangle" if x["triangle"] else "edge", 200 if x["triangle"] else 100, "fp32")
               for g, x in zip(graphs, mix)]
    for q in queries:
        if q[2] == "triangle":
            q[0].list_triangles()
    workers = lds.batch_autotune(queries)
    for _ in range(args.warmup):
        lds.topk_batch(queries[:64], workers=workers)
    torch.cuda.synchronize()
    times, launches0 = [], lds.launch_count()
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            t = time.perf_counter()
            got = lds.topk_batch(queries, workers=workers)
            times.append(time.perf_counter() - t)
    launches = lds.launch_count() - launches0
    sample = min(len(queries), args.plain_sample)
    t = time.perf_counter()
    plain = [g.topk(k, d, it, "fp64") for g, k, d, it, _ in queries[:sample]]
    plain_s = time.perf_counter() - t
    t = time.perf_counter()
    serial = [g.topk(k, d, it, p) for g, k, d, it, p in queries[:sample]]
    serial_s = time.perf_counter() - t
    same = all(_sets(a) == _sets(b) for a, b in zip(plain, got[:sample]))
    same_serial = all(_sets(a) == _sets(b) for a, b in zip(serial, got[:sample]))
    qps = len(queries) * args.steps / sum(times)
    line = {
        "metric": "LDS queries/s (batched)", "value": qps, "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched_mix: {len(queries)} graphs, n log-uniform in [50, 20000], Chung-Lu "
                               "exponent 2.3, average degree 8, 1-4 blocks of 10-100 at 0.6-0.95 (seed 4)",
                   "graphs": len(queries), "triangle_queries": sum(q[2] == "triangle" for q in queries),
                   "k": 3, "iters": "100 edge / 200 triangle", "precision": "fp32", "workers": workers,
                   "generation_s": gen_s},
        "autotuned": {"workers": workers,
                      "fw_threads_per_graph": {f"nact<2^{b}": lds.fw_batch_threads((1 << b) - 1)
                                               for b in range(6, 16)}},
        "plain_fp64_gpu": {"queries_per_s": sample / plain_s, "sample": sample, "same_output": same},
        "serial_fp32_gpu": {"queries_per_s": sample / serial_s, "sample": sample, "same_output": same_serial},
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    for g in graphs:
        g.close()


def run_serve(args):
    """Poisson stream of top-k queries over a resident graph mix through the
    serving loop (lds_server_*): queries/s and p50 / p99 latency.  The mix is
    Chung-Lu graphs with n log-uniform in [1e3, serve_max_n] (exponent
    U(2.1, 2.5), average degree 10, 2 planted blocks each) plus, unless
    --no-rmat24, the R-MAT scale-24 graph (edge factor 16, 16.7M vertices, up
    to 268M edges), all resident on the device.  LTDS queries on the R-MAT
    graph are refused by the admission rule (LDS_EBUSY: its triangle footprint
    exceeds the budget); they are counted, not timed."""
    import threading as th
    import torch
    from paper_2504_10937_gb300 import lds
    torch.cuda.set_device(0)
    lds.load()
    rng = synth.SplitMix64(5)
    lo, hi = np.log(1e3), np.log(args.serve_max_n)
    graphs, sizes = [], []
    t0 = time.perf_counter()
    for i in range(args.serve_graphs):
        n = int(round(np.exp(lo + rng.uniform(1)[0] * (hi - lo))))
        expo = 2.1 + 0.4 * rng.uniform(1)[0]
        nn, u, v, _ = synth.chung_lu(n, 5 * n, expo, int(rng.u64(1)[0]), n_blocks=2, block_size_range=(10, 100),
                                     block_prob_range=(0.6, 0.95), block_size_dist="uniform")
        g = lds.Graph(nn, u.astype(np.int32), v.astype(np.int32))
        graphs.append(g)
        sizes.append((nn, g.m))
    rmat = None
    if not args.no_rmat24:
        nr, sr, dr = synth.rmat_device(24, 16, 0.57, 0.19, 0.19, seed=5)
        rmat = lds.Graph(nr, sr, dr)
        del sr, dr
        torch.cuda.empty_cache()
        graphs.append(rmat)
        sizes.append((nr, rmat.m))
    gen_s = time.perf_counter() - t0
    print(f"[serve] {len(graphs)} graphs resident after {gen_s:.0f} s", file=sys.stderr, flush=True)
    reqs = []
    for i in range(args.requests):
        g = graphs[int(rng.integers(0, len(graphs), 1)[0])]
        tri = rng.uniform(1)[0] < 0.3
        reqs.append((g, int(rng.integers(1, 21, 1)[0]), "triangle" if tri else "edge", 200 if tri else 100, "fp32"))
    unit_gaps = -np.log(1.0 - rng.uniform(len(reqs)))
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.8 * free)

    def run_at(srv, rate, count):
        """Open-loop Poisson arrivals at `rate` for the first `count` requests;
        returns (queries/s, sorted latencies, refused)."""
        gaps = unit_gaps[:count] / rate
        tickets = [None] * count
        refused = [0]
        t_start = time.perf_counter()

        def feeder():
            t = t_start
            for i in range(count):
                t += gaps[i]
                d = t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                try:
                    tickets[i] = srv.submit(*reqs[i])
                except lds.LdsError as e:
                    if e.status != lds.EBUSY:
                        raise
                    tickets[i] = -1
                    refused[0] += 1

        f = th.Thread(target=feeder)
        f.start()
        lat = []
        for i in range(count):
            while tickets[i] is None:
                time.sleep(0.0005)
            if tickets[i] < 0:
                continue
            _, info = srv.wait(tickets[i])
            lat.append(info["queue_ms"] + info["run_ms"])
            runs.append((info["run_ms"], i))
        f.join()
        return len(lat) / (time.perf_counter() - t_start), sorted(lat), refused[0]

    runs = []

    def slowest(count=8):
        out = []
        for ms, i in sorted(runs, reverse=True)[:count]:
            g, k, d, it, _ = reqs[i]
            out.append({"run_ms": round(ms, 1), "n": g.n, "m": g.m, "density": d, "k": k})
        return out

    def pct(lat, q):
        return lat[min(len(lat) - 1, int(q * (len(lat) - 1) + 0.5))]

    sweep = []
    with lds.Server(budget, args.serve_workers) as srv:
        for r in reqs[:8]:                                 # warm-up
            try:
                srv.wait(srv.submit(*r))
            except lds.LdsError as e:
                if e.status != lds.EBUSY:
                    raise
        with ClockSampler(0) as clk:
            qps, lat, refused = run_at(srv, args.rate, len(reqs))
            print(f"[serve] saturated: {qps:.2f} queries/s, p50 {pct(lat, 0.5):.0f} ms, p99 {pct(lat, 0.99):.0f} ms; "
                  f"slowest {slowest(4)}", file=sys.stderr, flush=True)
            # offered load below saturation: fractions of the rate just measured
            for frac in ([] if args.no_sweep else [0.25, 0.5, 0.75, 0.9]):
                q2, l2, r2 = run_at(srv, frac * qps, min(len(reqs), args.sweep_requests))
                print(f"[serve] offered {frac:.2f}: {q2:.2f} queries/s, p50 {pct(l2, 0.5):.0f} ms", file=sys.stderr,
                      flush=True)
                sweep.append({"offered_per_s": frac * qps, "queries_per_s": q2, "p50_ms": pct(l2, 0.5),
                              "p99_ms": pct(l2, 0.99), "requests": min(len(reqs), args.sweep_requests),
                              "refused": r2})
    line = {
        "metric": "LDS queries/s (served)", "value": qps, "unit": "queries/s",
        "n_gpus": 1, "steps": len(reqs), "warmup": 8, "ms_per_step": statistics.mean(lat),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.serve_graphs} resident Chung-Lu graphs, n log-uniform in "
                               f"[1e3, {args.serve_max_n:g}], exponent U(2.1, 2.5), average degree 10, 2 blocks each "
                               f"(seed 5)" + ("" if args.no_rmat24 else " + R-MAT scale 24, edge factor 16 (seed 5)"),
                   "graphs": [{"n": a, "m": b} for a, b in sizes], "generation_s": gen_s,
                   "requests": len(reqs), "sample": f"{len(reqs)} requests at saturation and "
                   f"{args.sweep_requests} per offered-load point, out of the 100,000 of the stated stream: the "
                   "whole stream would hold the GPU for hours", "arrival_rate_per_s": args.rate,
                   "k": "uniform 1-20", "edge_triangle": "70:30", "precision": "fp32",
                   "workers": args.serve_workers, "budget_bytes": budget},
        "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99), "max": lat[-1]},
        "refused_ebusy": refused,
        "slowest_requests": slowest(),
        "offered_load_sweep": sweep,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    for g in graphs:
        g.close()


# The paper's LDScvx times on Barabasi-Albert graphs with n = 1e6 and m = d n
# (d = 2..12), digitised from its scalability figure; Xeon Silver 4110, C++
# (context for the sweep below, not a target: other hardware, k unstated)
PAPER_BA_SECONDS = {2: 13.7, 4: 23.5, 6: 31.7, 8: 40.7, 10: 49.8, 12: 62.8}


def run_ba(args):
    """Scalability sweep of the paper (Barabasi-Albert, n = 1e6, m = 2e6 .. 12e6):
    one top-k LDS query per graph through lds_topk, timed with CUDA events on
    the graph's stream, the input resident on the device."""
    import torch
    from paper_2504_10937_gb300 import lds
    torch.cuda.set_device(0)
    lds.load()
    stream = torch.cuda.current_stream()
    rows = []
    with ClockSampler(0) as clk:
        for d in (2, 4, 6, 8, 10, 12):
            t0 = time.perf_counter()
            n, u, v = synth.barabasi_albert(1_000_000, d, seed=60 + d)[:3]
            gen_s = time.perf_counter() - t0
            tu = torch.from_numpy(u).cuda()
            tv = torch.from_numpy(v).cuda()
            times, res, st = [], None, None
            for k in range(args.warmup + args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                with lds.Graph(n, tu, tv, stream=stream.cuda_stream) as g:
                    res = g.topk(args.k, "edge", args.iters, args.precision)
                    st = lds.topk_last_stats()
                e1.record(stream)
                e1.synchronize()
                if k >= args.warmup:
                    times.append(e0.elapsed_time(e1))
            rows.append({"d": d, "n": n, "m": len(u), "ms_per_query": statistics.mean(times),
                         "fw_edge_updates_per_s": st["fw_edge_updates"] / (statistics.mean(times) / 1000.0),
                         "paper_s": PAPER_BA_SECONDS[d], "result": [[str(x), len(c)] for x, c in res],
                         "phases_ms": {key: st[key] for key in ("ms_fw", "ms_extract", "ms_prune", "ms_verify")},
                         "generation_s": gen_s})
            del tu, tv
    line = {
        "metric": "top-k LDS query time on Barabasi-Albert graphs (paper's scalability sweep)",
        "value": statistics.mean(r["ms_per_query"] for r in rows), "unit": "ms per query (mean over the sweep)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"exact": "int64", "fp32": "f32", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": "barabasi_albert(n=1e6, m_per_vertex=d, seed=60+d), d = 2..12", "k": args.k,
                   "iters": args.iters, "precision": args.precision,
                   "step": "ingest from device memory + top-k LDS query (lds_topk)",
                   "paper_s": "LDScvx times digitised from the paper's scalability figure (CPU, context only)"},
        "sweep": rows, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="chung_lu_1m")
    ap.add_argument("--density", choices=["edge", "triangle"], default=None, help="default: the workload's")
    ap.add_argument("--iters", type=int, default=None, help="default: the workload's (500 / 300)")
    ap.add_argument("--precision", choices=["exact", "fp32", "fp64"], default=None)
    ap.add_argument("--ref-iters", type=int, default=3)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--fw-only", action="store_true", help="time ingest + FW only (profiling runs)")
    ap.add_argument("--no-plain", action="store_true", help="skip the binary64 comparison queries")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-precision", action="store_true", help="skip the binary32 precision-pattern leg")
    ap.add_argument("--mode", choices=["query", "batch", "serve", "ba"], default="query",
                    help="query: the headline line; batch / serve: the many-query layers; ba: the paper's "
                         "Barabasi-Albert scalability sweep")
    ap.add_argument("--graphs", type=int, default=4096, help="batch mode: number of graphs")
    ap.add_argument("--plain-sample", type=int, default=64, help="batch mode: queries run one at a time")
    ap.add_argument("--requests", type=int, default=600, help="serve mode: requests at saturation")
    ap.add_argument("--sweep-requests", type=int, default=150, help="serve mode: requests per offered-load point")
    ap.add_argument("--rate", type=float, default=40.0, help="serve mode: Poisson arrivals per second")
    ap.add_argument("--serve-graphs", type=int, default=24)
    ap.add_argument("--serve-max-n", type=float, default=2e6)
    ap.add_argument("--no-rmat24", action="store_true", help="serve mode: leave out the R-MAT scale-24 graph")
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--no-sweep", action="store_true", help="serve mode: skip the offered-load sweep")
    args = ap.parse_args()
    spec = WORKLOADS[args.workload]
    for key in ("density", "iters", "precision", "k"):
        if getattr(args, key) is None:
            setattr(args, key, spec[key])
    if args.mode == "batch" and args.impl == "ours":
        run_batch(args)
        return
    if args.mode == "serve" and args.impl == "ours":
        run_serve(args)
        return
    if args.mode == "ba" and args.impl == "ours":
        if args.k == WORKLOADS[args.workload]["k"]:
            args.k = 5
        if args.iters == WORKLOADS[args.workload]["iters"]:
            args.iters = 100
        run_ba(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

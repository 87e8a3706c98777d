"""Writes the expected top-k answers of the large seeded workloads by running
the CPU oracle (oracle.ldscvx.topk, exact arithmetic) on them.

Only the oracle and the seeded input generators are used: no value comes from
the CUDA library.  Usage (from the repository root):

    python tests/golden/make_topk_golden.py chung_lu_1m     # about 10 minutes on one core
    python tests/golden/make_topk_golden.py rmat12

Each output file holds one line per set, densest first, in the format the
tests parse: "density : id,id,...".  The answer is Problem 1's (top-k LDSs of
positive density, ties by smallest member id), which does not depend on the
iteration count or the arithmetic the driver uses.
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import ldscvx  # noqa: E402
from oracle.graph import canonical_edges  # noqa: E402
from paper_2504_10937_gb300 import synth  # noqa: E402

WORKLOADS = {
    # Chung-Lu n = 1e6, exponent 2.1, 1e7 background edges + 50 planted blocks;
    # top-10 LDS with 500 Frank-Wolfe iterations per round
    "chung_lu_1m": dict(make=lambda: synth.workload_chung_lu_1m(seed=2), k=10, N=500, triangle=False),
    # R-MAT scale 12, edge factor 6, (a, b, c) = (0.57, 0.19, 0.19), 4 near-cliques of
    # 20-40 vertices at 0.8; top-5 LTDS with 300 iterations per round (about 6 minutes)
    "rmat12": dict(make=lambda: synth.rmat(12, 6, 0.57, 0.19, 0.19, seed=312, n_cliques=4,
                                           clique_size_range=(20, 40)), k=5, N=300, triangle=True,
                   exact=True),
}


def main(name: str):
    spec = WORKLOADS[name]
    t0 = time.time()
    n, u, v, _ = spec["make"]()
    cu, cv = canonical_edges(n, u, v)
    print(f"[{name}] n={n} m={len(cu)} generated in {time.time() - t0:.1f}s", flush=True)
    stats = {}
    res = ldscvx.topk(n, np.asarray(cu), np.asarray(cv), spec["k"], spec["N"], triangle=spec["triangle"],
                      precision="exact", stats=stats)
    dt = time.time() - t0
    exact_note = None
    if spec.get("exact"):
        # the definition itself (Def. 3 / Def. 9 through exact compact numbers) must agree
        from oracle import decomp
        from oracle.graph import triangles
        if spec["triangle"]:
            ex = decomp.ltds_exact(n, cu, cv, triangles(n, cu, cv))
        else:
            ex = decomp.lds_exact(n, cu, cv)
        assert [(d, list(c)) for d, c in ex[:spec["k"]]] == [(d, list(c)) for d, c in res], "driver != decomposition"
        exact_note = "oracle.decomp (exact compact numbers) gives the same sets"
    out = os.path.join(HERE, f"{name}_top{spec['k']}.txt")
    with open(out, "w") as f:
        f.write(f"# top-{spec['k']} {'LTDS' if spec['triangle'] else 'LDS'} of the seeded workload '{name}'\n")
        f.write(f"# n = {n}, m = {len(cu)}; written by tests/golden/make_topk_golden.py (oracle only)\n")
        f.write(f"# oracle run: {dt:.0f} s, stats {stats}\n")
        if exact_note:
            f.write(f"# {exact_note}\n")
        for dens, verts in res:
            f.write(f"{dens} : {','.join(str(x) for x in verts)}\n")
    print(f"[{name}] {len(res)} sets in {dt:.0f}s -> {out}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "chung_lu_1m")

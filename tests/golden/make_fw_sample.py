"""Writes oracle Frank-Wolfe values on a seeded vertex sample of the 1M-vertex
power-law workload, for checks at full size that the oracle cannot make on
every vertex in a test's time.

Only the oracle (oracle.fw) and the seeded input generators are used.  Usage
(from the repository root; the binary64 literal form takes about an hour):

    python tests/golden/make_fw_sample.py

Output: tests/golden/chung_lu_1m_fw500_sample.txt with one line per sampled
vertex: "id R r64" where R is the exact scaled load D_N r after N = 500
iterations of Alg. 1 (integer form, D_N = (N+1)(N+2)) and r64 the load of
Alg. 1 carried literally in binary64 (repr, round-trips exactly).  The sample
is 2,000 vertices drawn with SplitMix64(500) plus the 48 highest-degree ones.
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

from oracle import fw as ofw  # noqa: E402
from oracle.graph import canonical_edges, degrees  # noqa: E402
from paper_2504_10937_gb300 import synth  # noqa: E402

N = 500


def sample_ids(n, u, v):
    rng = synth.SplitMix64(500)
    ids = set(rng.integers(0, n, 2000).tolist())
    deg = degrees(n, u, v)
    ids |= set(np.argsort(-deg, kind="stable")[:48].tolist())
    return sorted(int(x) for x in ids)


def main():
    t0 = time.time()
    n, u, v, _ = synth.workload_chung_lu_1m(seed=2)
    cu, cv = canonical_edges(n, u, v)
    cu = np.asarray(cu, dtype=np.int64)
    cv = np.asarray(cv, dtype=np.int64)
    ids = sample_ids(n, cu, cv)
    R, _, Dn, _ = ofw.fw_edge_exact(n, cu, cv, N)
    print(f"exact form done at {time.time() - t0:.0f}s", flush=True)
    r64, _, _, _ = ofw.fw_edge_fp64_literal(n, cu, cv, N)
    print(f"binary64 form done at {time.time() - t0:.0f}s", flush=True)
    out = os.path.join(HERE, "chung_lu_1m_fw500_sample.txt")
    with open(out, "w") as f:
        f.write("# Alg. 1 on synth.workload_chung_lu_1m(seed=2) (canonical edges), N = 500 iterations\n")
        f.write(f"# n = {n}, m = {len(cu)}, D = {Dn}; written by tests/golden/make_fw_sample.py (oracle only)\n")
        f.write("# id  R (exact, = D r)  r64 (binary64 literal form)\n")
        for x in ids:
            f.write(f"{x} {int(R[x])} {float(r64[x])!r}\n")
    print(f"{len(ids)} vertices -> {out} ({time.time() - t0:.0f}s)", flush=True)


if __name__ == "__main__":
    main()

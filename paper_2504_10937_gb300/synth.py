"""Seeded synthetic graph generators.

This module is the one input source shared by the CUDA path, its tests, the
benchmark and the CPU oracle's tests.  It holds none of the method's
arithmetic: it only draws random graphs.  Every random number comes from a
counter-based SplitMix64 stream (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out below with numpy
uint64 arithmetic, so the same seed gives the same graph on x86 and on Arm
and with any numpy version.

The graph families stand in for the paper's datasets (Sec. 8, dataset table),
which are not available here:

* ``gnp_planted``    - G(n, p) background plus planted dense blocks;
* ``chung_lu``       - power-law expected degrees (Chung-Lu) plus planted
                       blocks of log-uniform size;
* ``rmat``           - R-MAT (Chakrabarti et al.) plus planted near-cliques;
* ``barabasi_albert``- preferential attachment, as in the paper's
                       scalability study (Sec. 8, scalability figure);
* ``batched_mix``    - thousands of small Chung-Lu graphs with blocks;
* ``scramble``       - turns a canonical edge list into a raw COO list
                       (random orientation and order, duplicates and
                       self-loops) to exercise graph ingest.

Every generator returns ``(n, u, v)`` with ``u < v`` int32 arrays sorted by
``(u, v)`` and free of duplicates, unless it says otherwise.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based SplitMix64 stream: output k is mix(seed + k * golden)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(int(seed) & _MASK64)
        self.counter = 0

    def u64(self, k: int) -> np.ndarray:
        k = int(k)
        idx = np.arange(self.counter + 1, self.counter + k + 1, dtype=np.uint64)
        self.counter += k
        with np.errstate(over="ignore"):
            z = self.seed + idx * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _MIX1
            z = (z ^ (z >> np.uint64(27))) * _MIX2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, k: int) -> np.ndarray:
        """k doubles in [0, 1) built from the top 53 bits."""
        return (self.u64(k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def integers(self, lo: int, hi: int, k: int) -> np.ndarray:
        """k integers in [lo, hi)."""
        span = hi - lo
        x = np.floor(self.uniform(k) * span).astype(np.int64)
        return lo + np.minimum(x, span - 1)

    def permutation(self, n: int) -> np.ndarray:
        keys = self.u64(n)
        return np.argsort(keys, kind="stable").astype(np.int64)

    def child(self, tag: int) -> "SplitMix64":
        """An independent stream derived from this one (for sub-generators)."""
        return SplitMix64(int(self.u64(1)[0]) ^ (int(tag) * 0x632BE59BD9B4E019 & _MASK64))


def _canon(n: int, a: np.ndarray, b: np.ndarray, keep_order_limit: int | None = None):
    """Drop self-loops and duplicates, orient u < v, sort by (u, v).

    With ``keep_order_limit`` the first ``limit`` distinct edges in draw
    order are kept (used to cut a sample down to an exact edge count).
    """
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    keep = a != b
    a, b = a[keep], b[keep]
    u = np.minimum(a, b)
    v = np.maximum(a, b)
    key = u * n + v
    if keep_order_limit is not None:
        uk, first = np.unique(key, return_index=True)
        order = np.argsort(first, kind="stable")[:keep_order_limit]
        key = np.sort(uk[order])
    else:
        key = np.unique(key)
    return (key // n).astype(np.int32), (key % n).astype(np.int32)


def _merge(n, parts):
    us = [p[0].astype(np.int64) for p in parts if len(p[0])]
    vs = [p[1].astype(np.int64) for p in parts if len(p[0])]
    if not us:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    return _canon(n, np.concatenate(us), np.concatenate(vs))


def _block_edges(rng: SplitMix64, verts: np.ndarray, prob: float):
    s = len(verts)
    if s < 2:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    iu, iv = np.triu_indices(s, 1)
    keep = rng.uniform(len(iu)) < prob
    return verts[iu[keep]], verts[iv[keep]]


def relabel(n: int, u: np.ndarray, v: np.ndarray, perm: np.ndarray):
    """Apply vertex permutation ``perm`` (old id -> new id) and re-canonicalise."""
    return _canon(n, perm[u.astype(np.int64)], perm[v.astype(np.int64)])


def gnp_planted(n: int, p: float, block_sizes=(), block_probs=(), seed: int = 1):
    """G(n, p) by one Bernoulli draw per vertex pair, plus planted blocks.

    Blocks sit on disjoint vertex sets cut from a seeded permutation; inside
    block j every pair is an edge with probability ``block_probs[j]``.
    Returns ``(n, u, v, blocks)`` where ``blocks`` lists the block vertex
    sets (sorted int64 arrays).
    """
    rng = SplitMix64(seed)
    parts = []
    if n >= 2 and p > 0:
        iu, iv = np.triu_indices(n, 1)
        keep = rng.uniform(len(iu)) < p
        parts.append((iu[keep], iv[keep]))
        del iu, iv
    perm = rng.permutation(n)
    blocks, off = [], 0
    for s, q in zip(block_sizes, block_probs):
        vs = np.sort(perm[off:off + s])
        off += s
        blocks.append(vs)
        parts.append(_block_edges(rng, vs, q))
    u, v = _merge(n, parts)
    return n, u, v, blocks


def _chung_lu_background(rng: SplitMix64, n: int, m: int, exponent: float):
    """Chung-Lu sample: endpoints drawn proportional to w_i = (i+1)^(-1/(beta-1)),
    weights scaled to sum 2m and capped at sqrt(2m); loops and duplicates are
    dropped and the sample topped up until exactly m distinct edges remain."""
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (exponent - 1.0))
    w *= (2.0 * m) / w.sum()
    np.minimum(w, np.sqrt(2.0 * m), out=w)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    ka = np.zeros(0, np.int64)
    kb = np.zeros(0, np.int64)
    want = m
    for _ in range(64):
        draw = int(want * 1.15) + 16
        x = np.searchsorted(cdf, rng.uniform(2 * draw), side="right")
        np.minimum(x, n - 1, out=x)
        ka = np.concatenate([ka, x[0::2]])
        kb = np.concatenate([kb, x[1::2]])
        u, v = _canon(n, ka, kb)
        if len(u) >= m:
            break
        want = m - len(u)
    return _canon(n, ka, kb, keep_order_limit=m)


def chung_lu(n: int, m: int, exponent: float, seed: int, n_blocks: int = 0,
             block_size_range=(50, 500), block_prob_range=(0.3, 0.9),
             block_size_dist: str = "loguniform"):
    """Power-law Chung-Lu background with exactly ``m`` edges plus planted blocks.

    Block sizes are log-uniform (or integer-uniform) in ``block_size_range``,
    block edge probabilities uniform in ``block_prob_range``, vertex sets
    disjoint.  Vertex ids are randomly relabelled at the end so that hubs are
    spread over the id range.  Returns ``(n, u, v, blocks)``.
    """
    rng = SplitMix64(seed)
    bu, bv = _chung_lu_background(rng, n, m, exponent)
    perm_blocks = rng.permutation(n)
    parts = [(bu, bv)]
    blocks, off = [], 0
    lo, hi = block_size_range
    for _ in range(n_blocks):
        if block_size_dist == "loguniform":
            s = int(round(np.exp(np.log(lo) + rng.uniform(1)[0] * (np.log(hi) - np.log(lo)))))
        else:
            s = int(rng.integers(lo, hi + 1, 1)[0])
        s = max(2, min(s, n - off))
        q = block_prob_range[0] + rng.uniform(1)[0] * (block_prob_range[1] - block_prob_range[0])
        vs = np.sort(perm_blocks[off:off + s])
        off += s
        blocks.append(vs)
        parts.append(_block_edges(rng, vs, q))
    u, v = _merge(n, parts)
    perm = rng.permutation(n)
    u, v = relabel(n, u, v, perm)
    blocks = [np.sort(perm[b]) for b in blocks]
    return n, u, v, blocks


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         n_cliques: int = 0, clique_size_range=(30, 200), clique_prob: float = 0.8):
    """R-MAT with 2^scale vertices and edge_factor * 2^scale samples.

    Each sample picks one quadrant per bit level with probabilities a, b, c and
    d = 1 - a - b - c; samples are deduplicated, symmetrised, stripped of
    self-loops, planted near-cliques (integer-uniform sizes, edge probability
    ``clique_prob``, disjoint vertex sets) are added and ids are randomly
    relabelled.  Returns ``(n, u, v, blocks)``.
    """
    rng = SplitMix64(seed)
    n = 1 << scale
    samples = edge_factor * n
    src = np.zeros(samples, np.int64)
    dst = np.zeros(samples, np.int64)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        x = rng.uniform(samples)
        bit = np.int64(1 << (scale - 1 - level))
        right = ((x >= a) & (x < ab)) | (x >= abc)
        down = x >= ab
        src += down * bit
        dst += right * bit
        del x, right, down
    parts = [_canon(n, src, dst)]
    del src, dst
    perm_blocks = rng.permutation(n)
    blocks, off = [], 0
    for _ in range(n_cliques):
        s = int(rng.integers(clique_size_range[0], clique_size_range[1] + 1, 1)[0])
        vs = np.sort(perm_blocks[off:off + s])
        off += s
        blocks.append(vs)
        parts.append(_block_edges(rng, vs, clique_prob))
    u, v = _merge(n, parts)
    perm = rng.permutation(n)
    u, v = relabel(n, u, v, perm)
    blocks = [np.sort(perm[bk]) for bk in blocks]
    return n, u, v, blocks


def barabasi_albert(n: int, m_per_vertex: int, seed: int):
    """Preferential attachment: vertex t >= m0 links to ``m_per_vertex``
    endpoints drawn from the list of all earlier edge endpoints (duplicates
    dropped).  Returns ``(n, u, v)``."""
    rng = SplitMix64(seed)
    k = m_per_vertex
    m0 = k + 1
    ends = np.zeros(2 * (n * k + m0 * m0), np.int64)
    iu, iv = np.triu_indices(m0, 1)
    ne = len(iu)
    ends[0:2 * ne:2] = iu
    ends[1:2 * ne:2] = iv
    fill = 2 * ne
    eu = [iu.astype(np.int64)]
    ev = [iv.astype(np.int64)]
    # process vertices in chunks: within a chunk, targets are drawn from the
    # endpoint list as it stood at the start of the chunk
    t = m0
    chunk = 4096
    while t < n:
        hi = min(n, t + chunk)
        cnt = hi - t
        r = rng.uniform(cnt * k)
        tgt = ends[np.minimum((r * fill).astype(np.int64), fill - 1)]
        srcs = np.repeat(np.arange(t, hi, dtype=np.int64), k)
        eu.append(srcs)
        ev.append(tgt)
        ends[fill:fill + 2 * cnt * k:2] = srcs
        ends[fill + 1:fill + 2 * cnt * k:2] = tgt
        fill += 2 * cnt * k
        t = hi
    u, v = _canon(n, np.concatenate(eu), np.concatenate(ev))
    return n, u, v


def batched_mix(count: int, seed: int, n_range=(50, 20000), exponent: float = 2.3,
                avg_degree: float = 8.0, triangle_share: float = 0.25):
    """``count`` independent small graphs: n log-uniform in ``n_range``,
    Chung-Lu background with m = avg_degree * n / 2 edges, 1-4 planted blocks of
    integer-uniform size 10..100 (at most n) with probability U(0.6, 0.95), and
    a seeded ``triangle_share`` of the graphs marked for triangle density.
    Returns a list of dicts with keys n, u, v, blocks, triangle."""
    rng = SplitMix64(seed)
    out = []
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    for g in range(count):
        n = int(round(np.exp(lo + rng.uniform(1)[0] * (hi - lo))))
        m = int(avg_degree * n / 2)
        m = min(m, n * (n - 1) // 2)
        nb = int(rng.integers(1, 5, 1)[0])
        sub_seed = int(rng.u64(1)[0])
        nn, u, v, blocks = chung_lu(n, m, exponent, sub_seed, n_blocks=nb,
                                     block_size_range=(10, min(100, n)),
                                     block_prob_range=(0.6, 0.95),
                                     block_size_dist="uniform")
        tri = bool(rng.uniform(1)[0] < triangle_share)
        out.append(dict(n=nn, u=u, v=v, blocks=blocks, triangle=tri))
    return out


def scramble(n: int, u: np.ndarray, v: np.ndarray, seed: int, dup_frac: float = 0.05,
             loop_frac: float = 0.01):
    """Raw COO version of a canonical edge list: each edge flipped with
    probability 1/2, a ``dup_frac`` share duplicated, ``loop_frac * m``
    self-loops added, then everything shuffled.  Returns int32 (src, dst)."""
    rng = SplitMix64(seed)
    m = len(u)
    a = u.astype(np.int64)
    b = v.astype(np.int64)
    flip = rng.uniform(m) < 0.5
    a, b = np.where(flip, b, a), np.where(flip, a, b)
    nd = int(m * dup_frac)
    if nd and m:
        pick = rng.integers(0, m, nd)
        a = np.concatenate([a, b[pick]])
        b = np.concatenate([b, a[pick]])
    nl = int(m * loop_frac)
    if nl and n:
        w = rng.integers(0, n, nl)
        a = np.concatenate([a, w])
        b = np.concatenate([b, w])
    order = rng.permutation(len(a))
    return a[order].astype(np.int32), b[order].astype(np.int32)


# --- named workloads (sizes follow the paper-shaped configurations) ---------

def workload_planted_gnp(seed: int = 1):
    """n = 2000, p = 4/1999, blocks of 20/30/40/50/60 vertices with internal
    probability 0.9/0.8/0.7/0.6/0.5."""
    return gnp_planted(2000, 4.0 / 1999.0, (20, 30, 40, 50, 60),
                       (0.9, 0.8, 0.7, 0.6, 0.5), seed=seed)


def workload_chung_lu_1m(seed: int = 2, n: int = 1_000_000, m: int = 10_000_000,
                         n_blocks: int = 50):
    """Chung-Lu, n = 1e6, m = 1e7 background edges, exponent 2.1, plus 50
    planted blocks of log-uniform size 50-500 and probability U(0.3, 0.9)."""
    return chung_lu(n, m, 2.1, seed, n_blocks=n_blocks)


def workload_rmat20(seed: int = 3, scale: int = 20):
    """R-MAT scale 20, edge factor 16, (a, b, c) = (0.57, 0.19, 0.19), plus 20
    near-cliques of size 30-200 at probability 0.8."""
    return rmat(scale, 16, 0.57, 0.19, 0.19, seed, n_cliques=20)


# --- device-side generation of the large R-MAT graph -------------------------

def _splitmix_torch(seed: int, first: int, k: int, device):
    """Outputs first+1 .. first+k of SplitMix64(seed) as int64 torch tensors on
    `device`, bit for bit equal to SplitMix64.u64 (int64 products wrap like
    uint64 ones; right shifts are made logical by masking)."""
    import torch

    def s64(x):            # an unsigned 64-bit constant as the int64 with the same bits
        x &= _MASK64
        return x - (1 << 64) if x >= (1 << 63) else x

    def lsr(z, r):
        return (z >> r) & ((1 << (64 - r)) - 1)

    idx = torch.arange(first + 1, first + k + 1, dtype=torch.int64, device=device)
    z = idx * s64(int(_GOLDEN)) + s64(int(seed))
    z = (z ^ lsr(z, 30)) * s64(int(_MIX1))
    z = (z ^ lsr(z, 27)) * s64(int(_MIX2))
    return z ^ lsr(z, 31)


def rmat_device(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int, device="cuda"):
    """The samples and the random relabelling of ``rmat(scale, edge_factor, a,
    b, c, seed)`` without planted near-cliques, drawn on a CUDA device with
    torch: SplitMix64 outputs, quadrant choices and the permutation are the
    same numbers the numpy generator draws.  Returns ``(n, src, dst)`` as int32
    device tensors in raw form (repeats, both orientations and self-loops left
    in): ``lds_create_graph`` canonicalises them to the graph ``rmat`` returns.
    Used for sizes whose numpy generation takes many minutes (scale 24)."""
    import torch
    n = 1 << scale
    samples = edge_factor * n
    src = torch.zeros(samples, dtype=torch.int64, device=device)
    dst = torch.zeros(samples, dtype=torch.int64, device=device)
    ab, abc = a + b, a + b + c
    counter = 0
    chunk = 1 << 26
    for level in range(scale):
        bit = 1 << (scale - 1 - level)
        for lo in range(0, samples, chunk):
            k = min(chunk, samples - lo)
            z = _splitmix_torch(seed, counter + lo, k, device)
            x = ((z >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
            right = ((x >= a) & (x < ab)) | (x >= abc)
            down = x >= ab
            src[lo:lo + k] += down.to(torch.int64) * bit
            dst[lo:lo + k] += right.to(torch.int64) * bit
            del z, x, right, down
        counter += samples
    counter += n                                   # the near-clique vertex permutation (unused here)
    keys = _splitmix_torch(seed, counter, n, device) ^ (-(1 << 63))    # unsigned order as signed order
    perm = torch.argsort(keys, stable=True)
    del keys
    # relabel as rmat does: old id x becomes perm[x]
    return n, perm[src].to(torch.int32), perm[dst].to(torch.int32)

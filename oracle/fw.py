"""Frank-Wolfe for the convex programs of the paper (test infrastructure).

Edge program CP(G) (Eq. 2) solved by Alg. 1; triangle program (Eq. 4) solved
by Alg. 6.  Readings of the paper:

* Orientation and ties (Alg. 1): every edge is taken as (u, v) with u < v.  The
  paper's test "r_u < r_v" gives the edge to u; otherwise (ties included) it goes
  to v, so ties go to the larger id.
* Alg. 6 leaves the receiving vertex x undefined; the appendix (proof of
  Thm. 4) has each triangle give all its weight to its lowest-r vertex, so
  x = argmin_{w in t} r_w; ties go to the larger id, as in Alg. 1.
* Exact form: with D_i = (i+1)(i+2) and gamma_i = 2/(i+2) one has
  D_i (1 - gamma_i) = D_{i-1} and D_i gamma_i = 2(i+1).  Multiplying Alg. 1's
  update by D_i turns it into integer additions: W = D_i * alpha_{u,v} starts
  at 1 and gains 2(i+1) when u wins; R_u = D_i * r_u starts at deg(u) and gains
  2(i+1) per edge u wins.  For triangles W' = 3 D_i alpha starts at 2 and gains
  6(i+1); R' = 3 D_i r starts at 2 * (#triangles at u).  The comparisons
  r_u < r_v and R_u < R_v agree because both sides share D_i.
* binary64 "literal" form: Alg. 1 with one alpha per ordered pair (or per
  vertex-triangle pair), alpha <- (1 - gamma) * alpha + gamma * alpha_hat with
  every operation rounded separately, and r_u summed left to right over u's
  neighbours (triangles) in ascending id order starting from 0.
* binary32 "recurrence" form: summing Alg. 1's alpha update over u's edges gives
  r_u <- (1 - gamma) r_u + gamma c_u, c_u = number of edges (triangles) u wins.
  It is carried in binary32, each operation rounded, gamma = fl(2 / (i+2)),
  r^(0) = fl(deg(u) / 2) (fl(tri(u) / 3) for triangles).  The weights alpha are
  rebuilt exactly from the recorded choices, so they form an exactly feasible
  solution whatever the rounding of r.

Pins (tests/test_oracle_fw.py): the integer form equals the rational
evaluation of Alg. 1 / Alg. 6 on random small graphs at every iteration; a
single edge and K_n worked by hand; sum_u R_u = m D_i and 0 <= W <= D_i at every
iteration; Table 2's optimum (r* = 5/2, 2, 3/2, 4/3) approached on the
reconstructed Fig. 1 graph (Thm. 1); the binary64 and binary32 forms stay
within their rounding bounds of the rational values when choices coincide.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from .graph import adjacency, csr, degrees, triangle_degrees


# --------------------------------------------------------------------------
# Alg. 1, exact rational arithmetic (slow; small graphs only)
# --------------------------------------------------------------------------

def fw_edge_rational(n: int, u, v, N: int):
    """Alg. 1 in exact rationals.  Returns (r list[Fraction], alpha dict
    {(a, b): alpha_{a,b}} over both orientations of every edge)."""
    edges = list(zip(np.asarray(u).tolist(), np.asarray(v).tolist()))
    adj = adjacency(n, u, v)
    alpha = {}
    for a, b in edges:
        alpha[(a, b)] = Fraction(1, 2)
        alpha[(b, a)] = Fraction(1, 2)
    r = [sum((alpha[(x, y)] for y in adj[x]), Fraction(0)) for x in range(n)]
    for i in range(1, N + 1):
        g = Fraction(2, i + 2)
        ah = {}
        for a, b in edges:
            if r[a] < r[b]:
                ah[(a, b)], ah[(b, a)] = 1, 0
            else:
                ah[(a, b)], ah[(b, a)] = 0, 1
        alpha = {k: (1 - g) * val + g * ah[k] for k, val in alpha.items()}
        r = [sum((alpha[(x, y)] for y in adj[x]), Fraction(0)) for x in range(n)]
    return r, alpha


def fw_tri_rational(n: int, tris, N: int):
    """Alg. 6 in exact rationals.  Returns (r list[Fraction], alpha array
    of Fractions with shape (|T|, 3), column k for vertex tris[t][k])."""
    tl = [tuple(t) for t in np.asarray(tris, dtype=np.int64).reshape(-1, 3).tolist()]
    alpha = [[Fraction(1, 3)] * 3 for _ in tl]

    def loads():
        r = [Fraction(0)] * n
        for t, al in zip(tl, alpha):
            for k in range(3):
                r[t[k]] += al[k]
        return r

    r = loads()
    for i in range(1, N + 1):
        g = Fraction(2, i + 2)
        new = []
        for t, al in zip(tl, alpha):
            best = 2
            for k in (1, 0):           # ties keep the larger id (later column)
                if r[t[k]] < r[t[best]]:
                    best = k
            new.append([(1 - g) * al[k] + g * (1 if k == best else 0) for k in range(3)])
        alpha = new
        r = loads()
    return r, alpha


# --------------------------------------------------------------------------
# Alg. 1 / Alg. 6, exact integer form
# --------------------------------------------------------------------------

def D(i: int) -> int:
    """Common denominator after i iterations: (i+1)(i+2)."""
    return (i + 1) * (i + 2)


def fw_edge_exact(n: int, u, v, N: int, R0=None, W0=None, i0: int = 0, record: bool = False):
    """Integer-scaled Alg. 1.  Starts from (R0, W0) at iteration i0 (default:
    the initial point) and runs to iteration N.  Returns (R, W, D_N, choices)
    where choices[i - i0 - 1] is the bool array alpha_hat_{u,v} of iteration
    i (empty list unless ``record``)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if R0 is None:
        R = degrees(n, u, v)
        W = np.ones(len(u), dtype=np.int64)
    else:
        R = np.array(R0, dtype=np.int64)
        W = np.array(W0, dtype=np.int64)
    choices = []
    for i in range(i0 + 1, N + 1):
        to_u = R[u] < R[v]
        inc = 2 * (i + 1)
        W = W + inc * to_u
        c = np.bincount(u, weights=to_u, minlength=n) + np.bincount(v, weights=~to_u, minlength=n)
        R = R + inc * c.astype(np.int64)
        if record:
            choices.append(to_u.copy())
    return R, W, D(N), choices


def tri_argmin(Rvals):
    """Column (0, 1, 2) of the lowest load in each row of Rvals (|T|, 3);
    among equal loads the later column (larger vertex id) wins."""
    best = np.full(len(Rvals), 2, dtype=np.int64)
    bv = Rvals[:, 2].copy()
    for k in (1, 0):
        better = Rvals[:, k] < bv
        best = np.where(better, k, best)
        bv = np.where(better, Rvals[:, k], bv)
    return best


def fw_tri_exact(n: int, tris, N: int, R0=None, W0=None, i0: int = 0, record: bool = False):
    """Integer-scaled Alg. 6 (W' = 3 D_i alpha, R' = 3 D_i r).  Returns
    (R, W (|T|, 3), 3 D_N, choices) with choices[i] the winning column."""
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    if R0 is None:
        R = 2 * triangle_degrees(n, t)
        W = np.full(t.shape, 2, dtype=np.int64)
    else:
        R = np.array(R0, dtype=np.int64)
        W = np.array(W0, dtype=np.int64)
    choices = []
    rows = np.arange(len(t))
    for i in range(i0 + 1, N + 1):
        x = tri_argmin(R[t]) if len(t) else np.zeros(0, np.int64)
        inc = 6 * (i + 1)
        W[rows, x] += inc
        winners = t[rows, x]
        R = R + inc * np.bincount(winners, minlength=n).astype(np.int64)
        if record:
            choices.append(x.copy())
    return R, W, 3 * D(N), choices


# --------------------------------------------------------------------------
# binary64, Alg. 1 / Alg. 6 literally
# --------------------------------------------------------------------------

def _gamma64(i: int) -> float:
    return 2.0 / float(i + 2)


def fw_edge_fp64_literal(n: int, u, v, N: int, record=None):
    """Alg. 1 in binary64 with one alpha per ordered pair.  Returns
    (r float64[n], alpha_slot float64[2m], rowptr, col): alpha_slot[s] is
    alpha_{x, col[s]} for the CSR slot s of row x.  A list passed as
    ``record`` receives alpha_hat_{u,v} of every iteration."""
    rowptr, col = csr(n, u, v)
    deg = np.diff(rowptr)
    rowid = np.repeat(np.arange(n), deg)
    a = np.full(len(col), 0.5, dtype=np.float64)

    def loads(a):
        r = np.zeros(n, dtype=np.float64)
        for k in range(int(deg.max()) if n and len(col) else 0):
            rows = np.nonzero(deg > k)[0]
            r[rows] = r[rows] + a[rowptr[rows] + k]
        return r

    r = loads(a)
    for i in range(1, N + 1):
        g = _gamma64(i)
        one_minus = 1.0 - g
        if record is not None:
            record.append(r[np.asarray(u, dtype=np.int64)] < r[np.asarray(v, dtype=np.int64)])
        rx = r[rowid]
        ry = r[col]
        # slot (x, y) receives iff x is the endpoint Alg. 1 picks for edge {x, y}
        win = np.where(rowid < col, rx < ry, ~(ry < rx))
        ah = win.astype(np.float64)
        a = (one_minus * a) + (g * ah)
        r = loads(a)
    return r, a, rowptr, col


def fw_tri_fp64_literal(n: int, tris, N: int, record=None):
    """Alg. 6 in binary64 with one alpha per (vertex, triangle).  r_u sums its
    triangles' alphas left to right in ascending triangle order.  Returns
    (r float64[n], alpha float64 (|T|, 3)).  A list passed as ``record``
    receives the receiving column of every triangle in every iteration."""
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    a = np.full(t.shape, 1.0 / 3.0, dtype=np.float64)
    # incidence lists in ascending triangle order
    inc_v = t.reshape(-1)
    inc_t = np.repeat(np.arange(len(t)), 3)
    inc_k = np.tile(np.arange(3), len(t))
    order = np.lexsort((inc_t, inc_v))
    inc_v, inc_t, inc_k = inc_v[order], inc_t[order], inc_k[order]
    cnt = np.bincount(inc_v, minlength=n)
    ptr = np.concatenate([[0], np.cumsum(cnt)])

    def loads(a):
        r = np.zeros(n, dtype=np.float64)
        for k in range(int(cnt.max()) if len(t) else 0):
            rows = np.nonzero(cnt > k)[0]
            s = ptr[rows] + k
            r[rows] = r[rows] + a[inc_t[s], inc_k[s]]
        return r

    r = loads(a)
    rows = np.arange(len(t))
    for i in range(1, N + 1):
        g = _gamma64(i)
        one_minus = 1.0 - g
        x = tri_argmin(r[t]) if len(t) else np.zeros(0, np.int64)
        if record is not None:
            record.append(x.copy())
        ah = np.zeros(t.shape, dtype=np.float64)
        ah[rows, x] = 1.0
        a = (one_minus * a) + (g * ah)
        r = loads(a)
    return r, a


def snap_tri_weights(alpha, Dn3: int):
    """An exactly feasible integer solution W (|T|, 3) over the denominator Dn3
    from binary64 alphas (the snapping of the Def. 12 check's reading): every
    weight is rint(alpha * Dn3) except that the member with the largest alpha
    (the first one on ties) takes Dn3 minus the other two, so every row sums to
    Dn3 and no weight is negative."""
    a = np.asarray(alpha, dtype=np.float64).reshape(-1, 3)
    W = np.rint(a * float(Dn3)).astype(np.int64)
    if len(a):
        j = np.argmax(a, axis=1)
        rows = np.arange(len(a))
        W[rows, j] = Dn3 - (W.sum(axis=1) - W[rows, j])
    return W


# --------------------------------------------------------------------------
# binary32, recurrence form (alpha rebuilt exactly from the choices)
# --------------------------------------------------------------------------

def gamma32(i: int) -> np.float32:
    return np.float32(2.0) / np.float32(i + 2)


def fw_edge_fp32_step(r, i: int, u, v, n: int):
    """One binary32 recurrence step (iteration i) from loads r.  Returns
    (r_next float32[n], to_u bool[m])."""
    r = np.asarray(r, dtype=np.float32)
    to_u = r[u] < r[v]
    c = (np.bincount(u, weights=to_u, minlength=n) + np.bincount(v, weights=~to_u, minlength=n)).astype(np.float32)
    g = gamma32(i)
    one_minus = np.float32(1.0) - g
    r_next = (one_minus * r) + (g * c)
    return r_next.astype(np.float32), to_u


def fw_edge_fp32(n: int, u, v, N: int, record=None):
    """Returns (r float32[n], W int64[m], D_N) where W = D_N * alpha_{u,v} is
    rebuilt exactly from the binary32 run's choices (appended to ``record``
    when a list is given)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    r = (degrees(n, u, v).astype(np.float32) * np.float32(0.5)).astype(np.float32)
    W = np.ones(len(u), dtype=np.int64)
    for i in range(1, N + 1):
        r, to_u = fw_edge_fp32_step(r, i, u, v, n)
        if record is not None:
            record.append(to_u)
        W = W + 2 * (i + 1) * to_u
    return r, W, D(N)


def fw_tri_fp32_step(r, i: int, tris, n: int):
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    r = np.asarray(r, dtype=np.float32)
    x = tri_argmin(r[t]) if len(t) else np.zeros(0, np.int64)
    winners = t[np.arange(len(t)), x]
    c = np.bincount(winners, minlength=n).astype(np.float32)
    g = gamma32(i)
    one_minus = np.float32(1.0) - g
    return ((one_minus * r) + (g * c)).astype(np.float32), x


def fw_tri_fp32(n: int, tris, N: int):
    """Triangle analogue of fw_edge_fp32.  Returns (r float32[n], W (|T|,3),
    3 D_N)."""
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    r = (triangle_degrees(n, t).astype(np.float32) / np.float32(3.0)).astype(np.float32)
    W = np.full(t.shape, 2, dtype=np.int64)
    rows = np.arange(len(t))
    for i in range(1, N + 1):
        r, x = fw_tri_fp32_step(r, i, t, n)
        W[rows, x] += 6 * (i + 1)
    return r, W, 3 * D(N)


# --------------------------------------------------------------------------
# helpers shared by the oracle's later stages
# --------------------------------------------------------------------------

def edge_loads_from_W(n: int, u, v, W, Dn: int):
    """R_x = sum of x's scaled shares: u gets W, v gets D - W."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    W = np.asarray(W, dtype=np.int64)
    R = np.bincount(u, weights=W, minlength=n) + np.bincount(v, weights=Dn - W, minlength=n)
    return np.rint(R).astype(np.int64)


def tri_loads_from_W(n: int, tris, W):
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    R = np.zeros(n, dtype=np.int64)
    for k in range(3):
        np.add.at(R, t[:, k], np.asarray(W)[:, k])
    return R

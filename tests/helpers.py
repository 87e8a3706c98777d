"""Shared test helpers: golden fixtures and small random graphs."""
import os
from fractions import Fraction

import numpy as np

from paper_2504_10937_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_graph(name):
    u, v = [], []
    n = None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            if line.startswith("n "):
                n = int(line.split()[1])
                continue
            a, b = line.split()
            u.append(int(a))
            v.append(int(b))
    return n, np.array(u, dtype=np.int64), np.array(v, dtype=np.int64)


def load_expected(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            k, val = [s.strip() for s in line.split("=", 1)]
            out[k] = val
    return out


def frac(s):
    return Fraction(s)


def parse_sets(s):
    """'5/2:0,1,2 ; 2:9,10' -> [(Fraction(5,2), [0,1,2]), (Fraction(2), [9,10])]"""
    res = []
    for part in s.split(";"):
        d, vs = part.strip().split(":")
        res.append((Fraction(d.strip()), [int(x) for x in vs.split(",")]))
    return res


def parse_ids(s):
    return sorted(int(x) for x in s.split(","))


def random_graph(n, p, seed):
    n_, u, v, _ = synth.gnp_planted(n, p, seed=seed)
    return n_, u.astype(np.int64), v.astype(np.int64)


def random_planted(n, p, sizes, probs, seed):
    n_, u, v, blocks = synth.gnp_planted(n, p, sizes, probs, seed=seed)
    return n_, u.astype(np.int64), v.astype(np.int64), blocks

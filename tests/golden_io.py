"""Reader for the exact-rational fixtures in tests/golden/."""
from __future__ import annotations

import glob
import os
from fractions import Fraction

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(path):
    with open(path) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    it = iter(lines)
    hdr = {}
    for _ in range(3):
        key, val = next(it).split()
        hdr[key] = int(val)
    n, p, k = hdr["n"], hdr["p"], hdr["k"]

    def block(tag, rows):
        assert next(it) == tag
        return [next(it).split() for _ in range(rows)]

    M = np.array(block("M", n), dtype=np.float64)
    # rows of an empty X_L (p == 1) are blank lines, dropped above
    XL = np.array(block("XL", n if p > 1 else 0), dtype=np.float64).reshape(n, p - 1)
    y = np.array(block("y", 1)[0], dtype=np.float64)
    XR = np.array(block("XR", n), dtype=np.int8).reshape(n, k)
    Bf = [[Fraction(v) for v in row] for row in block("B", k)]
    B = np.array([[float(v) for v in row] for row in Bf], dtype=np.float64).T  # p x k
    return dict(n=n, p=p, k=k, M=M, XL=XL, y=y, XR=XR, B=B, B_exact=Bf)


def all_cases():
    return sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))

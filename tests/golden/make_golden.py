"""Writes the exact-rational fixtures in this folder.

Each fixture is a tiny integer instance of Eq. 1 with its b_i evaluated
exactly by ``oracle.exact`` (explicit M^{-1} by Gauss-Jordan over rationals).
The paper prints no worked example, so these exact values are the strongest
stored pin available.  Run from the repository root:

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import exact  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# (name, n, p, k, seed); M = A^T A + n I with small integer A
CASES = [
    ("tiny_n5_p3_k4", 5, 3, 4, 1),
    ("tiny_n8_p3_k6", 8, 3, 6, 2),
    ("tiny_n6_p1_k3", 6, 1, 3, 3),
    ("tiny_n7_p2_k5", 7, 2, 5, 4),
    ("tiny_n4_p4_k2", 4, 4, 2, 5),
    ("tiny_n8_p4_k3", 8, 4, 3, 6),
]


def make_case(n, p, k, seed):
    g = np.random.Generator(np.random.Philox(seed))
    A = g.integers(-3, 4, size=(n, n))
    M = A.T @ A + n * np.eye(n, dtype=np.int64)
    XL = np.empty((n, p - 1), dtype=np.int64)
    if p >= 2:
        XL[:, 0] = 1
        XL[:, 1:] = g.integers(-4, 5, size=(n, p - 2))
    y = g.integers(-9, 10, size=n)
    XR = g.integers(0, 3, size=(n, k))
    return M.astype(np.int64), XL, y.astype(np.int64), XR.astype(np.int64)


def write(name, n, p, k, M, XL, y, XR, B):
    lines = [
        "# Eq. 1, b_i = (X_i^T M^{-1} X_i)^{-1} X_i^T M^{-1} y with X_i = (X_L | x_Ri),",
        "# evaluated exactly over the rationals (explicit inverse, Gauss-Jordan)",
        "# by tests/golden/make_golden.py.  Matrices are listed row by row.",
        f"n {n}", f"p {p}", f"k {k}", "M",
    ]
    lines += [" ".join(str(int(v)) for v in row) for row in M]
    lines.append("XL")
    lines += [" ".join(str(int(v)) for v in row) for row in XL]
    lines.append("y")
    lines.append(" ".join(str(int(v)) for v in y))
    lines.append("XR")
    lines += [" ".join(str(int(v)) for v in row) for row in XR]
    lines.append("B")
    lines += [" ".join(f"{b.numerator}/{b.denominator}" for b in bi) for bi in B]
    with open(os.path.join(HERE, name + ".txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def main():
    for name, n, p, k, seed in CASES:
        M, XL, y, XR = make_case(n, p, k, seed)
        B = exact.gls_exact(M.tolist(), XL.tolist(), y.tolist(), XR.tolist())
        write(name, n, p, k, M, XL, y, XR, B)
        print("wrote", name)


if __name__ == "__main__":
    main()

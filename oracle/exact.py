"""Exact-rational brute force for Eq. 1 on tiny integer inputs.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

b_i = (X_i^T M^{-1} X_i)^{-1} X_i^T M^{-1} y is evaluated literally: M^{-1} is
formed explicitly by Gauss-Jordan elimination over ``fractions.Fraction`` and
every product is exact.  This is deliberately a different algorithm from the
FP64 oracle (no Cholesky, no triangular solves, no rounding), so agreement
between the two pins the FP64 oracle to the definition in Eq. 1.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Sequence

Matrix = List[List[Fraction]]


def _to_frac(a: Sequence[Sequence[int]]) -> Matrix:
    return [[Fraction(v) for v in row] for row in a]


def gauss_jordan_solve(A: Matrix, B: Matrix) -> Matrix:
    """Solve A X = B exactly (A square, nonsingular). Returns X."""
    n = len(A)
    m = len(B[0]) if B else 0
    aug = [list(A[i]) + list(B[i]) for i in range(n)]
    for col in range(n):
        piv = next((r for r in range(col, n) if aug[r][col] != 0), None)
        if piv is None:
            raise ZeroDivisionError("singular matrix")
        aug[col], aug[piv] = aug[piv], aug[col]
        pv = aug[col][col]
        aug[col] = [v / pv for v in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                f = aug[r][col]
                aug[r] = [a - f * b for a, b in zip(aug[r], aug[col])]
    return [row[n:n + m] for row in aug]


def inverse(A: Matrix) -> Matrix:
    n = len(A)
    eye = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    return gauss_jordan_solve(A, eye)


def matmul(A: Matrix, B: Matrix) -> Matrix:
    return [[sum((A[i][k] * B[k][j] for k in range(len(B))), Fraction(0))
             for j in range(len(B[0]))] for i in range(len(A))]


def transpose(A: Matrix) -> Matrix:
    return [list(r) for r in zip(*A)]


def gls_exact(M, XL, y, XR) -> List[List[Fraction]]:
    """Exact b_i for every SNP column of XR.

    M: n x n integers (symmetric positive definite)
    XL: n x (p-1) integers (rows), may have zero columns
    y: n integers
    XR: n x k integers (rows); column i is x_Ri
    Returns a list of k coefficient vectors (X_L coefficients first, SNP last).
    """
    Mf = _to_frac(M)
    n = len(Mf)
    Minv = inverse(Mf)
    yv = [[Fraction(v)] for v in y]
    k = len(XR[0]) if XR else 0
    out = []
    for i in range(k):
        X = [[Fraction(v) for v in XL[r]] + [Fraction(XR[r][i])] for r in range(n)]
        Xt = transpose(X)
        W = matmul(Xt, Minv)            # X_i^T M^{-1}
        A = matmul(W, X)                # X_i^T M^{-1} X_i
        r = matmul(W, yv)               # X_i^T M^{-1} y
        b = gauss_jordan_solve(A, r)
        out.append([row[0] for row in b])
    return out

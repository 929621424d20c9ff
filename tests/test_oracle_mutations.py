"""Planted mistakes: each mutation below is applied to a temporary copy of the
oracle's C source, which is compiled on the CPU; the exact-rational fixtures
must then fail.  This shows that the pins would catch a dropped term, a wrong
sign, a wrong index or a transposed operand anywhere in the oracle's steps.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from tests import golden_io

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTATIONS = {
    # Cholesky of M
    "potrf_dropped_term": ("for (int64_t k = 0; k < j; ++k) {\n      const double ljk",
                           "for (int64_t k = 1; k < j; ++k) {\n      const double ljk"),
    "potrf_transposed": ("v[i] -= COLMAJ(L, ldl, i, k) * ljk;", "v[i] -= COLMAJ(L, ldl, k, i) * ljk;"),
    "potrf_no_sqrt": ("const double ljj = sqrt(v[j]);", "const double ljj = v[j];"),
    # forward substitution
    "trsv_sign": ("x[i] -= COLMAJ(L, ldl, i, j) * xj;", "x[i] += COLMAJ(L, ldl, i, j) * xj;"),
    "trsv_transposed": ("x[i] -= COLMAJ(L, ldl, i, j) * xj;", "x[i] -= COLMAJ(L, ldl, j, i) * xj;"),
    "trsv_no_diag": ("const double xj = x[j] / COLMAJ(L, ldl, j, j);", "const double xj = x[j];"),
    # Gram / right-hand side
    "gram_dropped_row": ("for (int64_t t = 0; t < n; ++t) acc += ca[t] * cc[t];",
                         "for (int64_t t = 1; t < n; ++t) acc += ca[t] * cc[t];"),
    "rhs_wrong_operand": ("acc += ca[t] * jb->yt[t];", "acc += ca[t] * ca[t];"),
    "snp_column_index": ("const double* ca = (a < p - 1) ? jb->XLt + (size_t)a * (size_t)n : xt;",
                         "const double* ca = (a < p - 1) ? jb->XLt + (size_t)0 * (size_t)n : xt;"),
    # p x p solve
    "posv_sign": ("s -= COLMAJ(S, p, i, k) * b[k];", "s += COLMAJ(S, p, i, k) * b[k];"),
    "posv_back_transposed": ("s -= COLMAJ(S, p, k, i) * b[k];", "s -= COLMAJ(S, p, i, k) * b[k];"),
    "posv_dropped_pivot_term": ("for (int k = 0; k < j; ++k) d -= COLMAJ(S, p, j, k) * COLMAJ(S, p, j, k);",
                                "for (int k = 1; k < j; ++k) d -= COLMAJ(S, p, j, k) * COLMAJ(S, p, j, k);"),
    # whitening of the phenotype skipped
    "y_not_whitened": ("gls_oracle_trsv(n, L, n, yt);", "(void)0;"),
}


def golden_fails(lib):
    """True when at least one exact fixture disagrees with this oracle build."""
    for path in golden_io.all_cases():
        c = golden_io.load(path)
        try:
            B, status, info = oracle.gls(c["M"], c["XL"] if c["p"] > 1 else None, c["y"], c["XR"],
                                         library=lib)
        except Exception:
            return True
        if info != 0 or (status != 0).any():
            return True
        err = np.linalg.norm(B - c["B"], axis=0) / np.linalg.norm(c["B"], axis=0)
        if not np.all(err <= 1e-13):
            return True
    return False


def test_unmutated_copy_passes(tmp_path):
    so = oracle.build(src=SRC, out=str(tmp_path / "lib_ok.so"))
    assert not golden_fails(oracle.load_library(so))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    path = tmp_path / "oracle_mut.c"
    path.write_text(mutated)
    so = oracle.build(src=str(path), out=str(tmp_path / f"lib_{name}.so"))
    assert golden_fails(oracle.load_library(so)), f"pins did not catch mutation {name}"

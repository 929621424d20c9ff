"""Pins for the FP64 oracle, each against something other than the oracle itself.

Every check below comes from the mathematics of Eq. 1 or from an independent
library routine, never from re-running the oracle's own formula:
  * exact rational answers (explicit inverse) on tiny integer inputs;
  * the Cholesky residual and LAPACK's Cholesky;
  * M = I reduces GLS to ordinary least squares (QR/SVD lstsq);
  * b_i is invariant under M -> cM;
  * GLS equals OLS on whitened data (Alg. 1 reduction to gels);
  * planted exact solutions, closed forms for p = 1 and p = 2;
  * the normal-equation residual X_i^T M^{-1}(y - X_i b_i) = 0;
  * structure: permutations, duplicate columns, degenerate SNPs, threads.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1210_7325_gb300 import synth
from tests import golden_io


def relerr(B, Bref):
    """Per-SNP ||b_i - b_i^ref||_2 / ||b_i^ref||_2 (columns of p x k arrays)."""
    num = np.linalg.norm(B - Bref, axis=0)
    den = np.linalg.norm(Bref, axis=0)
    return num / den


def gls_lapack(M, XL, y, X):
    """Eq. 1 through LAPACK-backed numpy routines, explicitly via M^{-1} applied
    with an LU solve (a different algorithm from the oracle's Cholesky)."""
    Minv_y = np.linalg.solve(M, y)
    out = []
    for i in range(X.shape[1]):
        Xi = np.column_stack([XL, X[:, i].astype(np.float64)]) if XL.size else \
            X[:, i:i + 1].astype(np.float64)
        W = np.linalg.solve(M, Xi)
        out.append(np.linalg.solve(Xi.T @ W, Xi.T @ Minv_y))
    return np.array(out).T


@pytest.mark.parametrize("path", golden_io.all_cases(), ids=lambda p: p.split("/")[-1])
def test_exact_rational_golden(path):
    c = golden_io.load(path)
    B, status, info = oracle.gls(c["M"], c["XL"] if c["p"] > 1 else None, c["y"], c["XR"])
    assert info == 0
    assert (status == 0).all()
    assert relerr(B, c["B"]).max() <= 1e-13


def test_golden_fixture_count():
    assert len(golden_io.all_cases()) >= 5


@pytest.mark.parametrize("n", [1, 2, 7, 64, 129])
def test_potrf_residual_and_lapack(n):
    M = synth.kinship_M(n, 0.6, seed=11 + n, n_markers=50) if n > 1 else np.array([[2.25]])
    L, info = oracle.potrf(M)
    assert info == 0
    assert np.allclose(np.triu(L, 1), 0.0)
    res = np.linalg.norm(L @ L.T - M) / np.linalg.norm(M)
    assert res <= 4 * n * np.finfo(float).eps
    Lref = np.linalg.cholesky(M)
    assert np.abs(L - Lref).max() <= 1e-12 * np.abs(Lref).max()


def test_potrf_reads_lower_triangle_only():
    M = synth.kinship_M(40, 0.5, seed=3, n_markers=60)
    Mg = M.copy()
    Mg[np.triu_indices(40, 1)] = 1e300
    L1, _ = oracle.potrf(M)
    L2, _ = oracle.potrf(np.asfortranarray(Mg))
    assert np.array_equal(L1, L2)


def test_potrf_threads_bitwise():
    M = synth.kinship_M(150, 0.5, seed=4, n_markers=200)
    L1, _ = oracle.potrf(M, nthreads=1)
    L4, _ = oracle.potrf(M, nthreads=5)
    assert np.array_equal(L1, L4)


@pytest.mark.parametrize("M,pivot", [
    (np.diag([1.0, 2.0, -1.0, 3.0]), 3),
    (np.array([[4.0, 2.0], [2.0, 1.0]]), 2),          # second pivot exactly 0
    (np.array([[0.0, 0.0], [0.0, 1.0]]), 1),
    (np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]]), 2),
])
def test_potrf_not_spd_pivot(M, pivot):
    _, info = oracle.potrf(M)
    assert info == pivot
    B, status, info2 = oracle.gls(M, None, np.ones(M.shape[0]), np.ones((M.shape[0], 2), np.int8))
    assert info2 == pivot
    assert np.isnan(B).all()  # untouched output


def small_problem(n=60, p=4, k=25, h=0.5, seed=5):
    pr = synth.problem(n, p, k, h, seed, n_markers=80)
    return pr["M"], pr["XL"], pr["y"], pr["XR"]


def test_identity_M_reduces_to_ols():
    _, XL, y, XR = small_problem()
    n = XL.shape[0]
    B, status, _ = oracle.gls(np.eye(n), XL, y, XR)
    assert (status == 0).all()
    for i in range(XR.shape[1]):
        Xi = np.column_stack([XL, XR[:, i].astype(float)])
        ref = np.linalg.lstsq(Xi, y, rcond=None)[0]
        assert np.linalg.norm(B[:, i] - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("c", [3.7, 1e-3, 2.0 ** 40])
def test_scale_invariance(c):
    M, XL, y, XR = small_problem(seed=6)
    B1, _, _ = oracle.gls(M, XL, y, XR)
    B2, _, _ = oracle.gls(c * M, XL, y, XR)
    assert relerr(B2, B1).max() <= 1e-12
    if c == 2.0 ** 40:  # a power of two scales every rounded quantity exactly
        assert np.array_equal(B1, B2)


def test_whitened_ols_equals_gls():
    """Alg. 1: GLS -> potrf, trsv, trsm, gels.  LAPACK Cholesky + triangular
    solves + QR least squares."""
    M, XL, y, XR = small_problem(n=90, p=5, k=20, seed=7)
    B, _, _ = oracle.gls(M, XL, y, XR)
    L = sla.cholesky(M, lower=True)
    yw = sla.solve_triangular(L, y, lower=True)
    for i in range(XR.shape[1]):
        Xi = np.column_stack([XL, XR[:, i].astype(float)])
        Xw = sla.solve_triangular(L, Xi, lower=True)
        Q, R = np.linalg.qr(Xw)
        ref = sla.solve_triangular(R, Q.T @ yw)
        assert np.linalg.norm(B[:, i] - ref) <= 1e-11 * np.linalg.norm(ref)


def test_against_lu_explicit_solves():
    M, XL, y, XR = small_problem(n=70, p=3, k=15, seed=8)
    B, _, _ = oracle.gls(M, XL, y, XR)
    assert relerr(B, gls_lapack(M, XL, y, XR)).max() <= 1e-11


def test_planted_solution():
    """y = X_L beta_L + x_k beta_k exactly => b_k = (beta_L, beta_k) for any SPD M."""
    M, XL, _, XR = small_problem(n=80, p=4, k=12, seed=9)
    beta = np.array([0.5, -1.25, 2.0, 0.75])
    k0 = 5
    y = XL @ beta[:-1] + XR[:, k0].astype(float) * beta[-1]
    B, _, _ = oracle.gls(M, XL, y, XR)
    assert np.abs(B[:, k0] - beta).max() <= 1e-12


def test_closed_form_p1():
    """p = 1 (X_L empty): b_i = x^T M^{-1} y / x^T M^{-1} x."""
    M, _, y, XR = small_problem(n=50, p=1, k=9, seed=10)
    B, status, _ = oracle.gls(M, None, y, XR)
    assert B.shape == (1, 9)
    for i in range(9):
        x = XR[:, i].astype(float)
        ref = (x @ np.linalg.solve(M, y)) / (x @ np.linalg.solve(M, x))
        assert abs(B[0, i] - ref) <= 1e-12 * abs(ref)


def test_closed_form_p2_identity():
    """M = I, X_L = ones: slope = cov(x, y) / var(x), intercept = mean(y) - slope mean(x)."""
    n = 64
    g = np.random.Generator(np.random.Philox(12))
    y = g.standard_normal(n)
    XR = g.integers(0, 3, size=(n, 7)).astype(np.int8)
    B, _, _ = oracle.gls(np.eye(n), np.ones((n, 1)), y, XR)
    for i in range(7):
        x = XR[:, i].astype(float)
        slope = np.cov(x, y, bias=True)[0, 1] / np.var(x)
        icpt = y.mean() - slope * x.mean()
        assert abs(B[1, i] - slope) <= 1e-12 * max(1.0, abs(slope))
        assert abs(B[0, i] - icpt) <= 1e-12 * max(1.0, abs(icpt))


def test_normal_equation_residual():
    M, XL, y, XR = small_problem(n=100, p=6, k=10, seed=13)
    B, _, _ = oracle.gls(M, XL, y, XR)
    for i in range(XR.shape[1]):
        Xi = np.column_stack([XL, XR[:, i].astype(float)])
        r = Xi.T @ np.linalg.solve(M, y - Xi @ B[:, i])
        scale = np.abs(Xi.T @ np.linalg.solve(M, y)).max()
        assert np.abs(r).max() <= 1e-11 * scale


def test_structure_permutation_duplicates_threads():
    M, XL, y, XR = small_problem(n=60, p=4, k=30, seed=14)
    B, _, _ = oracle.gls(M, XL, y, XR)
    perm = np.random.Generator(np.random.Philox(1)).permutation(30)
    Bp, _, _ = oracle.gls(M, XL, y, XR[:, perm])
    assert np.array_equal(Bp, B[:, perm])
    XRd = np.column_stack([XR, XR[:, 3]])
    Bd, _, _ = oracle.gls(M, XL, y, XRd)
    assert np.array_equal(Bd[:, -1], Bd[:, 3])
    Bt, _, _ = oracle.gls(M, XL, y, XR, nthreads=7)
    assert np.array_equal(Bt, B)
    idx = np.array([29, 0, 3, 3, 17])
    Bs, _, _ = oracle.gls_sampled(M, XL, y, XR, idx)
    assert np.array_equal(Bs, B[:, idx])


def test_degenerate_snps_flagged():
    """A monomorphic SNP is collinear with the intercept; an all-zero SNP has
    S_BR = 0.  Both give NaN and status 1; the rest are unaffected."""
    M, XL, y, XR = small_problem(n=60, p=3, k=6, seed=15)
    XR = XR.copy()
    XR[:, 1] = 1
    XR[:, 4] = 0
    B, status, _ = oracle.gls(M, XL, y, XR)
    assert status.tolist() == [0, 1, 0, 0, 1, 0]
    assert np.isnan(B[:, [1, 4]]).all()
    assert np.isfinite(B[:, [0, 2, 3, 5]]).all()
    Bm, status_m, _ = oracle.gls(M, XL, y, XR, tau=oracle.TAU_MIXED)
    assert status_m.tolist() == [0, 1, 0, 0, 1, 0]
    assert np.array_equal(Bm[:, [0, 2, 3, 5]], B[:, [0, 2, 3, 5]])


def test_empty_sequence():
    M, XL, y, XR = small_problem(n=20, p=3, k=0, seed=16)
    B, status, info = oracle.gls(M, XL, y, XR[:, :0])
    assert info == 0 and B.shape == (3, 0) and status.shape == (0,)


def test_general_int8_values():
    """Any int8 genotype code is accepted (exactly representable); compare with LU."""
    M, XL, y, _ = small_problem(n=40, p=3, k=1, seed=17)
    g = np.random.Generator(np.random.Philox(2))
    XR = g.integers(-128, 128, size=(40, 6)).astype(np.int8)
    B, _, _ = oracle.gls(M, XL, y, XR)
    assert relerr(B, gls_lapack(M, XL, y, XR)).max() <= 1e-11

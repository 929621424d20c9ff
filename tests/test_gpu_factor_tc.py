"""The tensor-core binary64 factor (Cholesky of M, L^{-1}, whitening with exact
integer slices on tcgen05) against the FP64 oracle and against the plain
binary64 CUDA-core factor, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import oracle_ref, relerr, run_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


def factors(pr, flags, precision="fp64"):
    n = pr["M"].shape[0]
    p = pr["XL"].shape[1] + 1
    L = np.zeros((n, n), order="F")
    Z = np.zeros((n, n), order="F")
    with gls.Plan(n, p, 8, precision=precision, flags=flags) as plan:
        XL = np.asfortranarray(pr["XL"]) if p > 1 else None
        plan.factor(np.asfortranarray(pr["M"]), XL, np.ascontiguousarray(pr["y"]))
        plan.get_factor(L, Z)
    return L, Z


@pytest.mark.parametrize("n,p,m", [
    (1, 1, 3), (2, 2, 5), (63, 3, 17), (64, 4, 20), (65, 4, 129), (127, 5, 40), (129, 2, 70),
    (300, 20, 40), (640, 32, 33), (1000, 4, 300), (2049, 6, 64),
])
def test_fp64_plan_with_tensor_factor_matches_oracle(n, p, m):
    pr = synth.problem(n, p, m, 0.5, seed=200 + n + p, n_markers=max(2 * n, 20))
    B, st = run_gpu(pr, "fp64", flags=gls.GLS_FLAG_FACTOR_TENSOR)
    Bref, sref = oracle_ref(pr, oracle.TAU_FP64)
    assert np.array_equal(st, sref)
    ok = sref == 0
    e = relerr(B[:, ok], Bref[:, ok])
    assert e.max() <= TOL, f"max rel err {e.max():.3e}"


@pytest.mark.parametrize("n", [200, 1000, 2600])
def test_tensor_factor_agrees_with_binary64_factor(n):
    """L and L^{-1} of both implementations agree to a few binary64 ulps, and
    each satisfies L L^T = M and L^{-1} L = I to binary64 accuracy."""
    pr = synth.problem(n, 3, 4, 0.5, seed=300 + n, n_markers=max(2 * n, 20))
    Lt, Zt = factors(pr, gls.GLS_FLAG_FACTOR_TENSOR)
    Ln, Zn = factors(pr, 0)
    M = pr["M"]
    assert np.array_equal(np.triu(Lt, 1), np.zeros_like(Lt))
    assert np.array_equal(np.triu(Zt, 1), np.zeros_like(Zt))
    dL = np.abs(Lt - Ln).max() / np.abs(Ln).max()
    dZ = np.abs(Zt - Zn).max() / np.abs(Zn).max()
    assert dL <= 1e-12 and dZ <= 1e-12, (dL, dZ)
    eps = np.finfo(float).eps
    res = np.linalg.norm(Lt @ Lt.T - M) / np.linalg.norm(M)
    inv = np.abs(Zt @ Lt - np.eye(n)).max()
    assert res <= 4 * n * eps, res
    assert inv <= 4 * n * eps, inv
    # the plain binary64 factor meets the same bounds (same yardstick)
    assert np.linalg.norm(Ln @ Ln.T - M) / np.linalg.norm(M) <= 4 * n * eps


def test_tensor_factor_reports_not_spd_pivot():
    n = 300
    M = synth.kinship_M(n, 0.5, seed=3, n_markers=400)
    M[201, 201] = -1.0
    _, info = oracle.potrf(M)
    for prec, flags in (("fp64", gls.GLS_FLAG_FACTOR_TENSOR), ("bf16", 0)):
        with gls.Plan(n, 2, 8, precision=prec, flags=flags) as plan:
            with pytest.raises(gls.GlsError) as ei:
                plan.factor(np.asfortranarray(M), np.ones((n, 1), order="F"), np.ones(n))
            assert ei.value.status == 2 and ei.value.info == info == 202


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_mixed_path_with_native_factor_flag(prec):
    pr = synth.problem(700, 6, 300, 0.5, seed=17, n_markers=900)
    B, st = run_gpu(pr, prec, flags=gls.GLS_FLAG_FACTOR_NATIVE)
    Bt, stt = run_gpu(pr, prec)
    Bref, sref = oracle_ref(pr, oracle.TAU_MIXED)
    assert np.array_equal(st, sref) and np.array_equal(stt, sref)
    assert relerr(B, Bref).max() <= 1e-6
    assert relerr(Bt, Bref).max() <= 1e-6
    # the two factors differ by binary64 rounding only
    assert relerr(Bt, B).max() <= 2e-8


def test_conflicting_factor_flags_rejected():
    with pytest.raises(gls.GlsError) as ei:
        gls.Plan(100, 2, 8, flags=gls.GLS_FLAG_FACTOR_TENSOR | gls.GLS_FLAG_FACTOR_NATIVE)
    assert ei.value.status == 1

"""The split-factor autotuner: it picks the 2-slice split of L^{-1} only where
its measured error leaves the margin, and the split it picks meets the
tolerance against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import autotune, gls, synth
from tests.gpu_util import oracle_ref, relerr, run_gpu, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


@pytest.mark.parametrize("prec,tol,expect", [
    ("bf16", 1e-6, 3),   # the 2-slice BF16 split is near 2e-5 off: rejected
    ("bf16", 1e-2, 2),   # a loose tolerance admits it
    ("fp16", 1e-3, 2),
])
def test_tune_split_choice_and_accuracy(prec, tol, expect):
    pr = synth.problem(900, 5, 1200, 0.5, seed=91, n_markers=1800)
    n, m = pr["XR"].shape
    p = pr["XL"].shape[1] + 1
    M, XL, y, XR = to_device(pr)
    S, info = autotune.tune_split(n, p, prec, M, XL, y, XR[:256].t(), tol=tol)
    assert S == expect, info
    assert info["status_agree"]
    # the chosen split meets the tolerance on every SNP of the scan
    B, st = run_gpu(pr, prec, split_terms=S)
    Bref, sref = oracle_ref(pr, oracle.TAU_MIXED)
    assert np.array_equal(st, sref)
    assert relerr(B, Bref).max() <= tol

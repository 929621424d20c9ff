"""The paper's comparison algorithms (Alg. 3 black-box, Alg. 4 seq-gls,
Alg. 6 gwfgls) and the library's own Alg. 5 through gls_solve_variant: every
one computes Eq. 1, so b_i must match the FP64 oracle within 1e-10 and the
singular-SNP decisions must agree (a constant SNP is collinear with the
intercept, an all-zero one gives a zero row of S_i)."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import oracle_ref, relerr, to_device

pytestmark = pytest.mark.gpu
ALGS = ["black_box", "seq_gls", "hp_gwas", "gwfgls"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


def run_variant(pr, alg, kmax=None):
    import torch
    n, k = pr["XR"].shape
    p = pr["XL"].shape[1] + 1
    M, XL, y, XR = to_device(pr)
    B = torch.full((k, p), -3.0, dtype=torch.float64, device="cuda")
    st = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    with gls.Plan(n, p, kmax or k, precision="fp64") as plan:
        plan.solve_variant(alg, M, XL, y, XR.t(), B.t(), st, k=k)
        if alg != "hp_gwas":  # the comparison paths leave no factor behind
            with pytest.raises(gls.GlsError) as ei:
                plan.solve_block(XR.t(), B.t(), st, k=min(k, kmax or k))
            assert ei.value.status == 6
    return B.cpu().numpy().T, st.cpu().numpy()


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("n,p,k", [(300, 4, 40), (129, 1, 17), (500, 8, 70), (64, 2, 9)])
def test_variant_matches_oracle(alg, n, p, k):
    pr = synth.problem(n, p, k, 0.5, seed=700 + n + p, n_markers=max(2 * n, 200))
    pr["XR"] = pr["XR"].copy(order="F")
    pr["XR"][:, 3] = 1    # constant: collinear with the intercept when p > 1
    pr["XR"][:, 5] = 0    # monomorphic: S_i singular for every p
    B, st = run_variant(pr, alg, kmax=16 if alg == "hp_gwas" else None)
    Bref, sref = oracle_ref(pr, oracle.TAU_FP64)
    assert np.array_equal(st, sref), (st, sref)
    ok = sref == 0
    assert np.isnan(B[:, ~ok]).all()
    e = relerr(B[:, ok], Bref[:, ok])
    assert e.max() <= 1e-10, f"{alg}: max rel err {e.max():.3e}"


def test_variant_arguments():
    import torch
    pr = synth.problem(100, 9, 10, 0.5, seed=71, n_markers=200)   # p = 9 > 8
    M, XL, y, XR = to_device(pr)
    B = torch.zeros((10, 9), dtype=torch.float64, device="cuda")
    with gls.Plan(100, 9, 10, precision="fp64") as plan:
        with pytest.raises(gls.GlsError):
            plan.solve_variant("gwfgls", M, XL, y, XR.t(), B.t(), k=10)
        plan.solve_variant("hp_gwas", M, XL, y, XR.t(), B.t(), k=10)   # any p for Alg. 5
    Bref, _ = oracle_ref(pr, oracle.TAU_FP64)
    assert relerr(B.cpu().numpy().T, Bref).max() <= 1e-10
    pr2 = synth.problem(100, 2, 10, 0.5, seed=72, n_markers=200)
    M2, XL2, y2, XR2 = to_device(pr2)
    with gls.Plan(100, 2, 10, precision="bf16") as plan:
        with pytest.raises(gls.GlsError):
            plan.solve_variant("seq_gls", M2, XL2, y2, XR2.t(), B[:, :2].t(), k=10)

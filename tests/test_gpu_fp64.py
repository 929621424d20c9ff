"""FP64 GPU path against the FP64 oracle (tolerance 1e-10 relative on b_i),
through the C ABI.  Sizes span several 64-row/64-SNP tiles and ragged tails."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import oracle_ref, relerr, run_gpu, to_device

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


def check(pr, B, st, tau=oracle.TAU_FP64, tol=TOL):
    Bref, sref = oracle_ref(pr, tau)
    assert np.array_equal(st, sref)
    ok = sref == 0
    assert np.isnan(B[:, ~ok]).all()
    if not ok.any():
        return 0.0
    e = relerr(B[:, ok], Bref[:, ok])
    assert e.max() <= tol, f"max rel err {e.max():.3e}"
    return e.max()


def test_config0_full():
    """n = 1000, p = 4, m = 4096, h = 0.4 (the small FP64 workload), every SNP."""
    pr = synth.problem(1000, 4, 4096, 0.4, seed=synth.BASE_SEED + 0)
    B, st = run_gpu(pr, "fp64")
    check(pr, B, st)


@pytest.mark.parametrize("n,p,m,kmax", [
    (1, 1, 3, 3), (7, 2, 5, 2), (63, 3, 17, 17), (65, 4, 129, 64), (130, 5, 100, 33),
    (257, 1, 65, 65), (300, 20, 40, 40), (511, 32, 70, 70),
])
def test_ragged_shapes(n, p, m, kmax):
    pr = synth.problem(n, p, m, 0.5, seed=100 + n + p, n_markers=max(2 * n, 20))
    B, st = run_gpu(pr, "fp64", kmax=kmax)
    check(pr, B, st)


def test_host_pointers_match_device_pointers():
    pr = synth.problem(200, 4, 150, 0.5, seed=7, n_markers=300)
    Bd, sd = run_gpu(pr, "fp64", kmax=64)
    Bh, sh = run_gpu(pr, "fp64", kmax=64, host=True)
    assert np.array_equal(Bd, Bh) and np.array_equal(sd, sh)


def test_stream_matches_blocks_and_oracle():
    import torch
    pr = synth.problem(400, 4, 3000, 0.5, seed=8, n_markers=600)
    Bb, sb = run_gpu(pr, "fp64", kmax=1024)
    n, m, p = 400, 3000, 4
    with gls.Plan(n, p, 1024) as plan:
        plan.factor(np.asfortranarray(pr["M"]), np.asfortranarray(pr["XL"]), pr["y"])
        # pinned host input, pageable host output
        XR = torch.from_numpy(np.ascontiguousarray(pr["XR"].T)).pin_memory()
        B = np.zeros((p, m), order="F")
        st = np.zeros(m, np.int32)
        plan.solve_stream(XR.t(), B, st, m=m)
        assert np.array_equal(B, Bb) and np.array_equal(st, sb)
        # pageable input, pinned output
        Bp = torch.zeros((m, p), dtype=torch.float64).pin_memory()
        sp = torch.zeros(m, dtype=torch.int32).pin_memory()
        plan.solve_stream(np.asfortranarray(pr["XR"]), Bp.t(), sp, m=m)
        assert np.array_equal(Bp.numpy().T, Bb) and np.array_equal(sp.numpy(), sb)
    check(pr, Bb, sb)


def test_degenerate_snps_and_status():
    pr = synth.problem(256, 3, 10, 0.5, seed=9, n_markers=300)
    pr["XR"] = pr["XR"].copy(order="F")
    pr["XR"][:, 2] = 1   # collinear with the intercept
    pr["XR"][:, 7] = 0   # no variance at all
    B, st = run_gpu(pr, "fp64")
    assert st.tolist() == [0, 0, 1, 0, 0, 0, 0, 1, 0, 0]
    check(pr, B, st)


def test_not_spd_reports_pivot():
    n = 130
    M = synth.kinship_M(n, 0.5, seed=3, n_markers=200)
    M[70, 70] = -1.0
    with gls.Plan(n, 2, 8) as plan:
        with pytest.raises(gls.GlsError) as ei:
            plan.factor(np.asfortranarray(M), np.ones((n, 1), order="F"), np.ones(n))
        assert ei.value.status == 2
        _, info = oracle.potrf(M)
        assert ei.value.info == info == 71
        with pytest.raises(gls.GlsError) as ej:
            plan.solve_block(np.zeros((n, 1), np.int8, order="F"), np.zeros((2, 1), order="F"))
        assert ej.value.status == 6  # no valid factor


def test_collinear_covariates():
    n = 100
    M = synth.kinship_M(n, 0.5, seed=4, n_markers=150)
    XL = np.ones((n, 2), order="F")  # two identical columns
    with gls.Plan(n, 3, 8) as plan:
        with pytest.raises(gls.GlsError) as ei:
            plan.factor(np.asfortranarray(M), XL, np.ones(n))
        assert ei.value.status == 8 and ei.value.info == 2


def test_new_phenotype_keeps_factor():
    pr = synth.problem(300, 4, 64, 0.5, seed=10, n_markers=400)
    y2 = synth.phenotype(300, seed=99)
    n, m, p = 300, 64, 4
    with gls.Plan(n, p, m) as plan:
        plan.factor(np.asfortranarray(pr["M"]), np.asfortranarray(pr["XL"]), pr["y"])
        B1 = np.zeros((p, m), order="F")
        plan.solve_block(np.asfortranarray(pr["XR"]), B1)
        plan.factor(None, None, y2)
        B2 = np.zeros((p, m), order="F")
        plan.solve_block(np.asfortranarray(pr["XR"]), B2)
    pr2 = dict(pr, y=y2)
    Bref2, _ = oracle_ref(pr2, oracle.TAU_FP64)
    assert relerr(B2, Bref2).max() <= TOL
    assert not np.allclose(B1, B2)


def test_argument_errors():
    with gls.Plan(50, 2, 10) as plan:
        with pytest.raises(gls.GlsError) as ei:
            plan.solve_block(np.zeros((50, 1), np.int8, order="F"), np.zeros((2, 1), order="F"))
        assert ei.value.status == 6  # before factor
        pr = synth.problem(50, 2, 11, 0.5, seed=1, n_markers=60)
        plan.factor(np.asfortranarray(pr["M"]), np.asfortranarray(pr["XL"]), pr["y"])
        with pytest.raises(gls.GlsError) as ej:
            plan.solve_block(np.asfortranarray(pr["XR"]), np.zeros((2, 11), order="F"))
        assert ej.value.status == 1  # k = 11 > max_block_snps = 10
        plan.solve_block(np.asfortranarray(pr["XR"][:, :0]), np.zeros((2, 0), order="F"), k=0)


def test_general_int8_codes():
    pr = synth.problem(200, 3, 50, 0.5, seed=11, n_markers=300)
    g = np.random.Generator(np.random.Philox(5))
    pr["XR"] = np.asfortranarray(g.integers(-128, 128, size=(200, 50)).astype(np.int8))
    B, st = run_gpu(pr, "fp64")
    check(pr, B, st)

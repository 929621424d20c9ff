"""Several phenotypes per factor (Eq. 1 with its index j <= t): one pass of the
blocked solve over X_R serves t right-hand sides.  b_ij must match the oracle
run on phenotype j alone (1e-10 FP64, 1e-6 mixed); in binary64 it must equal
a single-phenotype plan's result bit for bit (every step treats the columns
of [X_L | Y] independently).  Covers a plan holding more phenotypes than a
call uses, new phenotypes for a kept factor, the double-buffered stream, a
batch of plans with different t, and degenerate SNPs."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import relerr, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


def phenotypes(n, t, seed):
    return np.column_stack([synth.phenotype(n, seed + 17 * j) for j in range(t)])


def oracle_each(pr, Y, tau):
    """The oracle once per phenotype: B (p, k, t), status (k,)."""
    XL = pr["XL"] if pr["XL"].shape[1] else None
    outs, st0 = [], None
    for j in range(Y.shape[1]):
        B, st, info = oracle.gls(pr["M"], XL, Y[:, j], pr["XR"], tau=tau,
                                 nthreads=oracle.default_threads())
        assert info == 0
        assert st0 is None or np.array_equal(st, st0)
        st0 = st
        outs.append(B)
    return np.stack(outs, axis=2), st0


def run_t(pr, Y, prec, kmax=None, capacity=None, flags=0):
    """Factor with all columns of Y; blocks of kmax SNPs; returns B (p, k, t), status."""
    import torch
    n, k = pr["XR"].shape
    p = pr["XL"].shape[1] + 1
    t = Y.shape[1]
    kmax = kmax or k
    M, XL, _, XR = to_device(pr)
    Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).to("cuda").t()
    with gls.Plan(n, p, kmax, precision=prec, phenotypes=capacity or t, flags=flags) as plan:
        plan.factor(M, XL, Yd)
        B = torch.empty((k * t, p), dtype=torch.float64, device="cuda")
        st = torch.empty(k, dtype=torch.int32, device="cuda")
        for s0 in range(0, k, kmax):
            kb = min(kmax, k - s0)
            plan.solve_block(XR[s0:s0 + kb].t(), B[s0 * t:(s0 + kb) * t].t(), st[s0:s0 + kb],
                             k=kb)
        plan.synchronize()
        Bh = B.cpu().numpy().reshape(k, t, p).transpose(2, 0, 1)   # (p, k, t)
        return Bh, st.cpu().numpy()


def check(B, st, Bref, sref, tol):
    assert np.array_equal(st, sref)
    ok = sref == 0
    assert np.isnan(B[:, ~ok, :]).all()
    for j in range(B.shape[2]):
        e = relerr(B[:, ok, j], Bref[:, ok, j])
        assert e.max() <= tol, f"phenotype {j}: max rel err {e.max():.3e}"


@pytest.mark.parametrize("prec,n,p,t,k,kmax,tol", [
    ("fp64", 700, 4, 3, 900, 256, 1e-10),
    ("fp64", 257, 1, 5, 300, 300, 1e-10),     # p = 1: no covariates
    ("fp16", 900, 6, 4, 700, 300, 1e-6),
    ("bf16", 2100, 20, 13, 400, 400, 1e-6),   # p - 1 + t = 32, BF16 slices
])
def test_phenotypes_match_oracle_each(prec, n, p, t, k, kmax, tol):
    pr = synth.problem(n, p, k, 0.5, seed=800 + n + t, n_markers=max(2 * n, 400))
    pr["XR"] = pr["XR"].copy(order="F")
    pr["XR"][:, 5] = 1                         # collinear with the intercept when p > 1
    Y = phenotypes(n, t, 900 + n)
    B, st = run_t(pr, Y, prec, kmax=kmax)
    tau = oracle.TAU_FP64 if prec == "fp64" else oracle.TAU_MIXED
    Bref, sref = oracle_each(pr, Y, tau)
    check(B, st, Bref, sref, tol)
    if prec == "fp64":  # each phenotype equals its own single-phenotype plan
        for j in (0, t - 1):
            Bj, sj = run_t(pr, Y[:, j:j + 1], prec, kmax=kmax)
            assert np.array_equal(Bj[:, :, 0], B[:, :, j], equal_nan=True)


def test_capacity_and_new_phenotypes_for_a_kept_factor():
    import torch
    n, p, k = 600, 3, 500
    pr = synth.problem(n, p, k, 0.4, seed=81, n_markers=700)
    Y = phenotypes(n, 5, 82)
    M, XL, _, XR = to_device(pr)
    with gls.Plan(n, p, k, precision="fp16", phenotypes=5) as plan:
        outs = []
        for cols, Mi, XLi in ((slice(0, 2), M, XL), (slice(2, 5), None, None),
                              (slice(4, 5), None, None)):
            Yj = Y[:, cols]
            plan.factor(Mi, XLi, torch.from_numpy(np.ascontiguousarray(Yj.T)).cuda().t())
            t = Yj.shape[1]
            B = torch.empty((k * t, p), dtype=torch.float64, device="cuda")
            st = torch.empty(k, dtype=torch.int32, device="cuda")
            plan.solve_block(XR.t(), B.t(), st, k=k)
            plan.synchronize()
            outs.append(B.cpu().numpy().reshape(k, t, p).transpose(2, 0, 1))
    Bref, sref = oracle_each(pr, Y, oracle.TAU_MIXED)
    check(outs[0], sref, Bref[:, :, 0:2], sref, 1e-6)
    check(outs[1], sref, Bref[:, :, 2:5], sref, 1e-6)
    check(outs[2], sref, Bref[:, :, 4:5], sref, 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_stream_with_phenotypes(prec):
    import torch
    n, p, t, m, kmax = 500, 4, 3, 2500, 1000
    pr = synth.problem(n, p, m, 0.5, seed=83, n_markers=700)
    Y = phenotypes(n, t, 84)
    Bb, sb = run_t(pr, Y, prec, kmax=kmax)
    with gls.Plan(n, p, kmax, precision=prec, phenotypes=t) as plan:
        plan.factor(np.asfortranarray(pr["M"]), np.asfortranarray(pr["XL"]),
                    np.asfortranarray(Y))
        XRh = torch.from_numpy(np.ascontiguousarray(pr["XR"].T)).pin_memory()
        for pinned in (True, False):
            B = torch.empty((m * t, p), dtype=torch.float64, pin_memory=pinned)
            st = torch.empty(m, dtype=torch.int32, pin_memory=pinned)
            plan.solve_stream(XRh.t(), B.t(), st, m=m)
            Bs = B.numpy().reshape(m, t, p).transpose(2, 0, 1)
            assert np.array_equal(Bs, Bb) and np.array_equal(st.numpy(), sb)


def test_batch_of_plans_with_different_t():
    import torch
    specs = [(700, 3, 400, 2), (1300, 5, 300, 4), (400, 2, 500, 1)]
    plans, XRs, Bs, sts, refs = [], [], [], [], []
    for i, (n, p, k, t) in enumerate(specs):
        pr = synth.problem(n, p, k, 0.5, seed=850 + i, n_markers=max(2 * n, 400))
        Y = phenotypes(n, t, 860 + i)
        M, XL, _, XR = to_device(pr)
        pl = gls.Plan(n, p, k, precision="fp16", phenotypes=t)
        pl.factor(M, XL, torch.from_numpy(np.ascontiguousarray(Y.T)).cuda().t())
        plans.append(pl)
        XRs.append(XR.t())
        Bs.append(torch.empty((k * t, p), dtype=torch.float64, device="cuda"))
        sts.append(torch.empty(k, dtype=torch.int32, device="cuda"))
        refs.append((pr, Y))
    with gls.Batch(plans) as batch:
        batch.solve(XRs, [B.t() for B in Bs], sts)
    for (n, p, k, t), B, st, (pr, Y) in zip(specs, Bs, sts, refs):
        Bh = B.cpu().numpy().reshape(k, t, p).transpose(2, 0, 1)
        Bref, sref = oracle_each(pr, Y, oracle.TAU_MIXED)
        check(Bh, st.cpu().numpy(), Bref, sref, 1e-6)
        Bsingle, _ = run_t(pr, Y, "fp16")
        assert np.array_equal(Bh, Bsingle, equal_nan=True)
    for pl in plans:
        pl.close()


def test_phenotype_bounds_rejected():
    with pytest.raises(gls.GlsError):
        gls.Plan(100, 20, 10, precision="fp64", phenotypes=14)   # 19 + 14 > 32
    with gls.Plan(100, 3, 10, precision="fp64", phenotypes=2) as plan:
        M = np.eye(100, order="F")
        with pytest.raises(gls.GlsError):
            plan.factor(M, np.ones((100, 2), order="F"), np.ones((100, 3), order="F"))

"""2-bit packed genotype input (gls_solve_block_packed, gls_solve_stream_packed)
against the int8 entry points on the same codes (identical results: the block
is unpacked on the device into the same int8 staging) and against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import oracle_ref, relerr, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


def plan_for(pr, prec, kmax):
    import torch
    n, m = pr["XR"].shape
    p = pr["XL"].shape[1] + 1
    plan = gls.Plan(n, p, kmax, precision=prec)
    M, XL, y, _ = to_device(pr)
    plan.factor(M, XL, y)
    return plan


@pytest.mark.parametrize("prec,n,m,kmax", [("bf16", 1001, 700, 256), ("fp64", 403, 300, 300),
                                           ("fp16", 514, 129, 64)])
def test_packed_block_equals_int8(prec, n, m, kmax):
    import torch
    pr = synth.problem(n, 4, m, 0.5, seed=500 + n, n_markers=2 * n)
    p = pr["XL"].shape[1] + 1
    XR = np.asfortranarray(pr["XR"])
    XP = gls.pack_genotypes(XR)
    Bref, sref = oracle_ref(pr, oracle.TAU_FP64 if prec == "fp64" else oracle.TAU_MIXED)
    with plan_for(pr, prec, kmax) as plan:
        outs = {}
        for where in ("int8", "packed_host", "packed_dev"):
            B = np.full((p, m), -7.0, order="F")
            st = np.full(m, -1, np.int32)
            for s0 in range(0, m, kmax):
                k = min(kmax, m - s0)
                if where == "int8":
                    plan.solve_block(XR[:, s0:s0 + k], B[:, s0:s0 + k], st[s0:s0 + k], k=k)
                elif where == "packed_host":
                    plan.solve_block_packed(XP[:, s0:s0 + k], B[:, s0:s0 + k], st[s0:s0 + k],
                                            k=k)
                else:
                    XPd = torch.from_numpy(np.ascontiguousarray(XP[:, s0:s0 + k].T)).cuda().t()
                    plan.solve_block_packed(XPd, B[:, s0:s0 + k], st[s0:s0 + k], k=k)
            outs[where] = (B, st)
    B8, s8 = outs["int8"]
    for where in ("packed_host", "packed_dev"):
        Bp, sp = outs[where]
        assert np.array_equal(B8, Bp) and np.array_equal(s8, sp), where
    assert np.array_equal(s8, sref)
    tol = 1e-10 if prec == "fp64" else 1e-6
    ok = sref == 0
    assert relerr(B8[:, ok], Bref[:, ok]).max() <= tol


@pytest.mark.parametrize("prec,source", [("bf16", "pinned"), ("bf16", "pageable"),
                                         ("bf16", "device"), ("fp16", "pinned"),
                                         ("fp64", "pinned")])
def test_packed_stream_equals_int8(prec, source):
    import torch
    pr = synth.problem(777, 5, 3000, 0.4, seed=77, n_markers=1500)
    n, m = pr["XR"].shape
    p = pr["XL"].shape[1] + 1
    XR = np.asfortranarray(pr["XR"])
    # a wider leading dimension than ceil(n/4) bytes: the packed columns of a larger array
    XPw = np.zeros((gls.packed_rows(n) + 5, m), dtype=np.uint8, order="F")
    XPw[:gls.packed_rows(n)] = gls.pack_genotypes(XR)
    if source == "pinned":
        XPt = torch.from_numpy(np.ascontiguousarray(XPw.T)).pin_memory().t()[:gls.packed_rows(n)]
    elif source == "device":
        XPt = torch.from_numpy(np.ascontiguousarray(XPw.T)).cuda().t()[:gls.packed_rows(n)]
    else:  # pageable host memory
        XPt = torch.from_numpy(np.ascontiguousarray(XPw.T)).t()[:gls.packed_rows(n)]
    with plan_for(pr, prec, 512) as plan:
        B8 = np.zeros((p, m), order="F")
        s8 = np.zeros(m, np.int32)
        plan.solve_stream(XR, B8, s8, m=m)
        Bp = np.full((p, m), -7.0, order="F")
        sp = np.full(m, -1, np.int32)
        plan.solve_stream_packed(XPt, Bp, sp, m=m)
    assert np.array_equal(B8, Bp) and np.array_equal(s8, sp)
    fp64 = prec == "fp64"
    Bref, sref = oracle_ref(pr, oracle.TAU_FP64 if fp64 else oracle.TAU_MIXED)
    assert np.array_equal(sp, sref)
    assert relerr(Bp, Bref).max() <= (1e-10 if fp64 else 1e-6)


def test_packed_rejects_short_leading_dimension():
    pr = synth.problem(100, 2, 8, 0.5, seed=3, n_markers=200)
    p = pr["XL"].shape[1] + 1
    with plan_for(pr, "bf16", 8) as plan:
        XP = np.zeros((gls.packed_rows(100) - 1, 8), dtype=np.uint8, order="F")
        B = np.zeros((p, 8), order="F")
        with pytest.raises(gls.GlsError) as ei:
            plan.solve_block_packed(XP, B, k=8)
        assert ei.value.status == 1

"""Batched uneven scans: several independent problems (own M, n, p, block size)
in one persistent launch of the mixed-precision solve.  Each problem's result
must equal its own single-plan solve bit for bit (an item's arithmetic does not
depend on which CTA runs it) and the FP64 oracle within 1e-6."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import oracle_ref, relerr, run_gpu, to_device

pytestmark = pytest.mark.gpu

SCANS = [  # n, p, m, h
    (1500, 6, 700, 0.3),
    (513, 2, 300, 0.8),
    (2048, 20, 257, 0.5),
    (130, 4, 1000, 0.6),
    (1001, 12, 1, 0.2),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_batch_matches_single_and_oracle(prec):
    import torch
    probs, plans, XRs, Bs, sts = [], [], [], [], []
    for i, (n, p, m, h) in enumerate(SCANS):
        pr = synth.problem(n, p, m, h, seed=500 + i, n_markers=max(2 * n, 200))
        probs.append(pr)
        M, XL, y, XR = to_device(pr)
        pl = gls.Plan(n, p, m, precision=prec)
        pl.factor(M, XL, y)
        plans.append(pl)
        XRs.append(XR.t())
        B = torch.full((m, p), -7.0, dtype=torch.float64, device="cuda")
        Bs.append(B)
        st = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        sts.append(st)
    with gls.Batch(plans) as batch:
        for group in (0, 3):
            batch.solve(XRs, [B.t() for B in Bs], sts, group=group)
            for i, pr in enumerate(probs):
                Bb = Bs[i].cpu().numpy().T
                Bs_single, st_single = run_gpu(pr, prec)
                assert np.array_equal(Bb, Bs_single), f"scan {i} group {group}"
                assert np.array_equal(sts[i].cpu().numpy(), st_single)
    if prec == "bf16":  # n = 2048 keeps BF16 slices, the rest run on FP16 ones
        assert [pl.operand_precision for pl in plans] == ["fp16"] * 2 + ["bf16"] + ["fp16"] * 2
    for i, pr in enumerate(probs):
        Bref, sref = oracle_ref(pr, oracle.TAU_MIXED)
        ok = sref == 0
        assert relerr(Bs[i].cpu().numpy().T[:, ok], Bref[:, ok]).max() <= 1e-6
    for pl in plans:
        pl.close()


def test_batch_rejects_mixed_configurations():
    a = gls.Plan(200, 3, 10, precision="fp16")
    b = gls.Plan(200, 3, 10, precision="fp16", split_terms=2)
    c = gls.Plan(200, 3, 10, precision="fp64")
    d = gls.Plan(2100, 3, 10, precision="bf16")
    with pytest.raises(gls.GlsError):
        gls.Batch([a, b])
    with pytest.raises(gls.GlsError):
        gls.Batch([a, c])
    gls.Batch([a, d]).close()  # BF16 and FP16 operands share a launch
    for pl in (a, b, c, d):
        pl.close()

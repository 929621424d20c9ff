"""CUDA-graph replay of repeated launch sequences (the factor of M, one block of
the SNP loop, one batched round) against eager launches of the same kernels
and against the FP64 oracle, through the C ABI."""
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


def solve_rounds(prs, precision, flags, rounds=3, kmax=None, timing=False):
    """Factors and solves every problem `rounds` times with the same device
    pointers (eager, captured, replayed); returns the B of each round."""
    import torch
    out = []
    pr0 = prs[0]
    n, m = pr0["XR"].shape
    p = pr0["XL"].shape[1] + 1
    kmax = kmax or m
    with gls.Plan(n, p, kmax, precision=precision, flags=flags) as plan:
        if timing:
            plan.set_timing(True)
        B = torch.empty((m, p), dtype=torch.float64, device="cuda:0")
        st = torch.empty(m, dtype=torch.int32, device="cuda:0")
        dev = [to_device(pr) for pr in prs]
        for r in range(rounds):
            M, XL, y, XR = dev[r % len(dev)]
            plan.factor(M, XL, y)
            B.fill_(-7.0)
            for s0 in range(0, m, kmax):
                k = min(kmax, m - s0)
                plan.solve_block(XR[s0:s0 + k].t(), B[s0:s0 + k].t(), st[s0:s0 + k], k=k)
            plan.synchronize()
            out.append((B.cpu().numpy().T.copy(order="F"), st.cpu().numpy()))
        stats = plan.stats()
    return out, stats


@pytest.mark.parametrize("precision,flags", [("bf16", 0), ("fp64", 0),
                                             ("fp64", gls.GLS_FLAG_FACTOR_TENSOR),
                                             ("bf16", gls.GLS_FLAG_FACTOR_NATIVE)])
def test_replayed_rounds_equal_eager(precision, flags):
    pr = synth.problem(700, 5, 700, 0.5, seed=41, n_markers=1400)
    eager, _ = solve_rounds([pr], precision, flags | gls.GLS_FLAG_EAGER)
    graph, _ = solve_rounds([pr], precision, flags)
    tau = oracle.TAU_FP64 if precision == "fp64" else oracle.TAU_MIXED
    Bref, sref = oracle_ref(pr, tau)
    tol = 1e-10 if precision == "fp64" else 1e-6
    for (Be, se), (Bg, sg) in zip(eager, graph):
        # the same kernels with the same arguments: identical bits
        assert np.array_equal(Be, Bg) and np.array_equal(se, sg)
        assert np.array_equal(sg, sref)
        assert relerr(Bg, Bref).max() <= tol


def test_replayed_factor_sees_new_matrix():
    """Round 3 replays the graph captured in round 2 on a different M and y:
    the graph reads the plan's buffers, so the new data flows through."""
    prs = [synth.problem(600, 4, 300, h, seed=s, n_markers=1200)
           for h, s in ((0.5, 51), (0.2, 52), (0.8, 53))]
    out, _ = solve_rounds(prs, "bf16", 0, rounds=3)
    for (B, st), pr in zip(out, prs):
        Bref, sref = oracle_ref(pr, oracle.TAU_MIXED)
        assert np.array_equal(st, sref)
        assert relerr(B, Bref).max() <= 1e-6


def test_replay_keeps_timing_and_launch_counts():
    pr = synth.problem(500, 3, 600, 0.5, seed=61, n_markers=1000)
    _, se = solve_rounds([pr], "bf16", gls.GLS_FLAG_EAGER, rounds=4, kmax=256, timing=True)
    _, sg = solve_rounds([pr], "bf16", 0, rounds=4, kmax=256, timing=True)
    assert sg["launches"] == se["launches"] > 0
    for key in ("trsm_launches", "convert_launches", "solve_launches", "factor_calls"):
        assert sg[key] == se[key] > 0, key
    for key in ("trsm_ms", "convert_ms", "solve_ms", "factor_ms"):
        assert sg[key] > 0.0, key


def test_replayed_stream_from_pinned_host():
    import torch
    pr = synth.problem(800, 4, 5000, 0.5, seed=71, n_markers=1600)
    n, m = pr["XR"].shape
    p = pr["XL"].shape[1] + 1
    XRh = torch.from_numpy(np.ascontiguousarray(pr["XR"].T)).pin_memory()
    res = {}
    for flags in (gls.GLS_FLAG_EAGER, 0):
        with gls.Plan(n, p, 1024, precision="bf16", flags=flags) as plan:
            M, XL, y, _ = to_device(pr)
            plan.factor(M, XL, y)
            outs = []
            for _ in range(3):
                Bh = torch.full((m, p), -7.0, dtype=torch.float64).pin_memory()
                sh = torch.full((m,), -1, dtype=torch.int32).pin_memory()
                plan.solve_stream(XRh.t(), Bh.t(), sh, m=m)
                outs.append((Bh.numpy().T.copy(), sh.numpy().copy()))
        res[flags] = outs
    Bref, sref = oracle_ref(pr, oracle.TAU_MIXED)
    for (Be, se), (Bg, sg) in zip(res[gls.GLS_FLAG_EAGER], res[0]):
        assert np.array_equal(Be, Bg) and np.array_equal(se, sg)
        assert np.array_equal(sg, sref)
        assert relerr(Bg, Bref).max() <= 1e-6


def test_replayed_batch_rounds_equal_eager():
    import torch
    specs = [(900, 5, 700, 0.5, 81), (400, 2, 1500, 0.3, 82), (1300, 8, 300, 0.7, 83)]
    prs = [synth.problem(n, p, m, h, seed=s, n_markers=2 * n) for n, p, m, h, s in specs]
    results = {}
    for flags in (gls.GLS_FLAG_EAGER, 0):
        plans, XRs, Bs, sts = [], [], [], []
        for pr in prs:
            n, m = pr["XR"].shape
            p = pr["XL"].shape[1] + 1
            pl = gls.Plan(n, p, m, precision="bf16", flags=flags)
            M, XL, y, XR = to_device(pr)
            pl.factor(M, XL, y)
            plans.append(pl)
            XRs.append(XR.t())
            Bs.append(torch.full((m, p), -7.0, dtype=torch.float64, device="cuda"))
            sts.append(torch.full((m,), -1, dtype=torch.int32, device="cuda"))
        outs = []
        with gls.Batch(plans) as batch:
            for _ in range(3):
                for B in Bs:
                    B.fill_(-7.0)
                batch.solve(XRs, [B.t() for B in Bs], sts)
                outs.append([(B.cpu().numpy().T.copy(), s.cpu().numpy()) for B, s in zip(Bs, sts)])
        for pl in plans:
            pl.close()
        results[flags] = outs
    refs = [oracle_ref(pr, oracle.TAU_MIXED) for pr in prs]
    for re_, rg in zip(results[gls.GLS_FLAG_EAGER], results[0]):
        for (Be, se), (Bg, sg), (Bref, sref) in zip(re_, rg, refs):
            assert np.array_equal(Be, Bg) and np.array_equal(se, sg)
            assert np.array_equal(sg, sref)
            assert relerr(Bg, Bref).max() <= 1e-6

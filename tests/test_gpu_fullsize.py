"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times, on sampled SNPs the oracle computes one by one: the FP64 method at
n = 1500, p = 4, m = 2.5M streamed from pinned host memory in blocks of 16384,
and one round of the 48 uneven scans in one persistent batched launch."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import autotune, gls, synth
from tests.gpu_util import relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


def test_fp64_streamed_2_5M_sampled():
    import torch
    import bench
    wl = bench.WORKLOADS["n1500_p4_m2500000_fp64"]
    n, p, m, kmax = wl["n"], wl["p"], wl["m"], wl["block"]
    seed = synth.BASE_SEED + wl["seed_offset"]
    M = synth.kinship_M(n, wl["h"], seed, device="cuda")
    XL = synth.covariates(n, p, seed)
    y = synth.phenotype(n, seed)
    XRh = torch.empty((m, n), dtype=torch.int8, pin_memory=True)
    synth.genotypes_torch(n, m, seed, device="cuda", out=XRh)  # drawn on the GPU, stored on the host
    Bh = torch.empty((m, p), dtype=torch.float64, pin_memory=True)
    sh = torch.empty(m, dtype=torch.int32, pin_memory=True)
    with gls.Plan(n, p, kmax, precision="fp64") as plan:
        plan.factor(np.asfortranarray(M), np.asfortranarray(XL), y)
        plan.solve_stream(XRh.t(), Bh.t(), sh, m=m)
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 5])))
    idx = np.unique(np.concatenate([[0, kmax - 1, kmax, m - 1], g.integers(0, m, 60)]))
    cols = np.asfortranarray(XRh[torch.from_numpy(idx)].numpy().T)  # n x len(idx)
    Bref, sref, info = oracle.gls_sampled(M, XL, y, cols, np.arange(idx.size),
                                          tau=oracle.TAU_FP64, nthreads=oracle.default_threads())
    assert info == 0
    B = Bh.numpy().T[:, idx]
    assert np.array_equal(sh.numpy()[idx], sref)
    e = relerr(B, Bref)
    print(f"fp64 n=1500 m=2.5M streamed: max rel err {e.max():.3e} over {idx.size} SNPs")
    assert e.max() <= 1e-10


def test_batch48_round_sampled():
    import torch
    import bench
    bw = bench.BATCH_WORKLOADS["batch48_uneven_bf16"]
    specs = bench.batch_specs(bw)
    plans, inputs, XRs, Bs, sts, ks = [], [], [], [], [], []
    for (n, p, m, h, seed) in specs:
        kb = autotune.choose_block(m, bw["block"])
        Mt = synth.kinship_M_torch(n, h, seed, device="cuda")
        XL = synth.covariates(n, p, seed)
        y = synth.phenotype(n, seed)
        XR = synth.genotypes_torch(n, kb, seed, device="cuda")  # the first block of the scan
        pl = gls.Plan(n, p, kb, precision="bf16")
        pl.factor(Mt.t(), torch.from_numpy(np.ascontiguousarray(XL.T)).cuda().t(),
                  torch.from_numpy(y).cuda())
        plans.append(pl)
        inputs.append((Mt, XL, y, XR))
        XRs.append(XR.t())
        B = torch.empty((kb, p), dtype=torch.float64, device="cuda")
        st = torch.empty(kb, dtype=torch.int32, device="cuda")
        Bs.append(B.t())
        sts.append(st)
        ks.append(kb)
    with gls.Batch(plans) as batch:
        batch.solve(XRs, Bs, sts, ks)
    torch.cuda.synchronize()
    order = np.argsort([s[0] for s in specs])
    for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        n, p, m, h, seed = specs[i]
        Mt, XL, y, XR = inputs[i]
        kb = ks[i]
        idx = np.unique(np.concatenate([[0, kb - 1], np.linspace(0, kb - 1, 14).astype(np.int64)]))
        cols = np.asfortranarray(XR[torch.from_numpy(idx).cuda()].cpu().numpy().T)
        Bref, sref, info = oracle.gls_sampled(Mt.cpu().numpy(), XL, y, cols, np.arange(idx.size),
                                              tau=oracle.TAU_MIXED,
                                              nthreads=oracle.default_threads())
        assert info == 0
        B = Bs[i].cpu().numpy()[:, idx]
        assert np.array_equal(sts[i].cpu().numpy()[idx], sref)
        e = relerr(B, Bref)
        print(f"batch48 scan {i}: n={n} p={p} block={kb}: max rel err {e.max():.3e}")
        assert e.max() <= 1e-6
    for pl in plans:
        pl.close()

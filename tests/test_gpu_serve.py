"""Serving with continuous batching: requests that arrive while others run are
admitted as memory frees up, their blocks share batched launches, repeated
M's reuse the resident factor, and every result equals the same request
solved alone (same kernels: bit for bit) and the oracle within 1e-6."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import gls, serve, synth
from tests.gpu_util import relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


def make_factory():
    import torch

    def make(req, torch_mod, reuse):
        seed = 900 + req.mkey
        M = XL = None
        if not reuse:
            M = torch.from_numpy(synth.kinship_M(req.n, req.h, seed, n_markers=400)).cuda().t()
            XL = torch.from_numpy(np.ascontiguousarray(synth.covariates(req.n, req.p, seed).T))
            XL = XL.cuda().t()
        y = torch.from_numpy(synth.phenotype(req.n, req.y_seed)).cuda()
        XR = torch.from_numpy(np.ascontiguousarray(synth.genotypes_np(req.n, req.m, seed).T))
        return serve.Inputs(M, XL, XR.cuda(), y)
    return make


def alone(req, prec, block):
    """The same request on its own plan, block by block."""
    import torch
    seed = 900 + req.mkey
    M = synth.kinship_M(req.n, req.h, seed, n_markers=400)
    XL = synth.covariates(req.n, req.p, seed)
    y = synth.phenotype(req.n, req.y_seed)
    XR = synth.genotypes_np(req.n, req.m, seed)
    with gls.Plan(req.n, req.p, block, precision=prec) as plan:
        plan.factor(np.asfortranarray(M), np.asfortranarray(XL), y)
        B = np.zeros((req.p, req.m), order="F")
        st = np.zeros(req.m, np.int32)
        for s0 in range(0, req.m, block):
            k = min(block, req.m - s0)
            plan.solve_block(np.asfortranarray(XR[:, s0:s0 + k]), B[:, s0:s0 + k],
                             st[s0:s0 + k], k=k)
    return B, st, (M, XL, y, XR)


@pytest.mark.parametrize("prec,budget", [("fp16", 100e9), ("fp16", 2.5e8), ("bf16", 100e9),
                                         ("fp64", 100e9)])
def test_served_equals_alone(prec, budget):
    reqs = serve.poisson_requests(10, 60.0, 1234, (150, 1400), (2, 6), (300, 2500), 0.3)
    assert any(r.reuse for r in reqs)
    block = 1024
    srv = serve.Server(make_factory(), prec, hbm_budget=budget, block=block)
    res = srv.run(reqs, time_cap=300.0, keep_outputs=True)
    assert not srv.rejected
    srv.close()
    assert len(res) == len(reqs)
    for r in reqs:
        got = res[r.rid]
        B = got["B"].cpu().numpy().T
        st = got["status"].cpu().numpy()
        Ba, sa, (M, XL, y, XR) = alone(r, prec, block)
        assert np.array_equal(st, sa)
        assert np.array_equal(B, Ba), f"request {r.rid} differs alone vs in the mix"
        if r.rid < 3:
            tau = oracle.TAU_FP64 if prec == "fp64" else oracle.TAU_MIXED
            Bref, sref, _ = oracle.gls(M, XL, y, XR, tau=tau, nthreads=oracle.default_threads())
            ok = sref == 0
            assert relerr(B[:, ok], Bref[:, ok]).max() <= (1e-10 if prec == "fp64" else 1e-6)
    summ = serve.latency_summary(res)
    assert summ["completed"] == len(reqs) and summ["p99_s"] >= summ["p50_s"] > 0

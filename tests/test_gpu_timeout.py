"""Bounded waits end in GLS_ERR_TIMEOUT, not a hang, and leave the GPU usable.

Device side: with a 1 microsecond limit (wait_limit_us) the pipeline waits of
the tensor-core solve run out while a working pipeline is still filling; the
kernel lets its in-flight copies and products finish, frees its tensor memory
and returns, and gls_synchronize reports the timeout.  A plan with the default
limit on the same device then matches the oracle.

Host side: with a 1 ms deadline (host_wait_ms) a binary64 factor of n = 4096
(tens of ms) returns GLS_ERR_TIMEOUT with its work still queued; waiting again
drains it, and a plan without the deadline matches the oracle.

No wait here is endless: every device wait has a limit, and the host waits
either have one or wait for kernels that have one."""
import time

import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import oracle_ref, relerr, run_gpu, to_device

pytestmark = pytest.mark.gpu
TIMEOUT = 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


def test_device_wait_limit_gives_timeout_then_gpu_is_usable():
    import torch
    n, p, k = 2048, 4, 8192
    pr = synth.problem(n, p, k, 0.5, seed=61, n_markers=600)
    M, XL, y, XR = to_device(pr)
    B = torch.zeros((k, p), dtype=torch.float64, device="cuda")
    st = torch.zeros(k, dtype=torch.int32, device="cuda")
    with gls.Plan(n, p, k, precision="fp16", wait_limit_us=1) as plan:
        plan.factor(M, XL, y)          # the factor's own waits keep their limit
        plan.solve_block(XR.t(), B.t(), st, k=k)
        with pytest.raises(gls.GlsError) as ei:
            plan.synchronize()
        assert ei.value.status == TIMEOUT
        assert "bounded device wait" in str(ei.value)
        # the error stays until the next factor clears it
        plan.factor(M, XL, y)
    torch.cuda.synchronize()           # the context is still usable
    assert float(torch.ones(4, device="cuda").sum()) == 4.0
    Bg, sg = run_gpu(pr, "fp16")       # a plan with the default limit
    Bref, sref = oracle_ref(pr, oracle.TAU_MIXED)
    assert np.array_equal(sg, sref)
    ok = sref == 0
    assert relerr(Bg[:, ok], Bref[:, ok]).max() <= 1e-6


def test_host_wait_deadline_gives_timeout_with_work_queued():
    n, p, k = 4096, 3, 256
    pr = synth.problem(n, p, k, 0.5, seed=62, n_markers=300)
    M, XL, y, XR = to_device(pr)
    plan = gls.Plan(n, p, k, precision="fp64", host_wait_ms=1)
    with pytest.raises(gls.GlsError) as ei:
        plan.factor(M, XL, y)
    assert ei.value.status == TIMEOUT and "still queued" in str(ei.value)
    t0 = time.perf_counter()
    while True:                        # the queued factor ends: its kernels are finite
        try:
            plan.synchronize()
            break
        except gls.GlsError as e:
            assert e.status == TIMEOUT
            assert time.perf_counter() - t0 < 60.0
    plan.close()
    Bg, sg = run_gpu(pr, "fp64")
    Bref, sref = oracle_ref(pr, oracle.TAU_FP64)
    assert np.array_equal(sg, sref)
    ok = sref == 0
    assert relerr(Bg[:, ok], Bref[:, ok]).max() <= 1e-10

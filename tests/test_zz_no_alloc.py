"""The allocation-free FP64 block solve (gls_solve_block_fp64_static).

Callers that cannot call cudaMalloc pass their own device buffers; the only
scratch is a fixed 4 MiB array inside the library.  Two calls in a row must
each agree with the plan-based gls_solve_block and with the oracle within the
FP64 tolerance (1e-10 relative on b_i), including p = 1 (no covariates, NULL
R_TL and z_T) and a block that fills the scratch exactly; sizes beyond the
scratch must be rejected, and a call leaves the device's free memory as it
was.  This file is collected last so that a failure here leaves every other
test already run; it also passes on its own in a fresh process.
"""
import ctypes
import gc

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import oracle_ref, relerr, run_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    from paper_1210_7325_gb300 import build
    build.build()
    lib = gls.load()
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    f = lib.gls_solve_block_fp64_static
    f.argtypes = [i64, i32, vp, i64, vp, i64, vp, vp, vp, i64, i64, vp, i64, vp, vp]
    f.restype = i32
    return lib


def factor_products(pr):
    """L^{-1}, [X~_L | y~], R_TL and z_T of the setup phase, on the host."""
    M, XL, y = pr["M"], pr["XL"], pr["y"]
    n = M.shape[0]
    p = XL.shape[1] + 1
    L = sla.cholesky(M, lower=True)
    Z = sla.solve_triangular(L, np.eye(n), lower=True)
    W = Z @ np.column_stack([XL, y])
    S = W[:, :p - 1].T @ W[:, :p - 1]
    R = sla.cholesky(S, lower=True) if p > 1 else np.zeros((0, 0))
    zT = sla.solve_triangular(R, W[:, :p - 1].T @ W[:, p - 1], lower=True) if p > 1 \
        else np.zeros(0)
    return Z, W, R, zT


@pytest.mark.parametrize("n,p,k", [
    (300, 5, 400),
    (200, 1, 300),      # p = 1: X_L empty, R_TL and z_T passed as NULL
    (512, 3, 16384),    # n a multiple of 64 and ceil(n/64) (p+1) k = 524288 exactly
])
def test_static_entry_point_matches_plan_and_oracle_twice(lib, n, p, k):
    import torch
    pr = synth.problem(n, p, k, 0.5, seed=77 + n + p, n_markers=max(400, 2 * n))
    Bplan, splan = run_gpu(pr, "fp64")
    Bora, sora = oracle_ref(pr, oracle.TAU_FP64)
    Z, W, R, zT = factor_products(pr)
    dev = "cuda:0"
    # row-major storage of the transposes = column-major storage of Z, W, R
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev)
    Wd = torch.from_numpy(np.ascontiguousarray(W.T)).to(dev)
    Rd = torch.from_numpy(np.ascontiguousarray(R.T)).to(dev) if p > 1 else None
    zd = torch.from_numpy(np.ascontiguousarray(zT)).to(dev) if p > 1 else None
    XR = torch.from_numpy(np.ascontiguousarray(pr["XR"].T)).to(dev)     # (k, n)
    stream = torch.cuda.current_stream().cuda_stream
    outs = [(torch.empty((k, p), dtype=torch.float64, device=dev),
             torch.empty((k,), dtype=torch.int32, device=dev)) for _ in range(2)]
    for call, (B, st) in enumerate(outs):
        B.fill_(-1.0)
        st.fill_(-1)
        gc.collect()  # so that no unrelated tensor is freed during the call
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        held0 = torch.cuda.memory_allocated()
        rc = lib.gls_solve_block_fp64_static(
            n, p, Zd.data_ptr(), n, Wd.data_ptr(), n,
            Rd.data_ptr() if Rd is not None else None, zd.data_ptr() if zd is not None else None,
            XR.data_ptr(), n, k, B.data_ptr(), p, st.data_ptr(), stream)
        assert rc == 0, gls.last_error()
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the kernels' module; later ones allocate nothing
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() <= held0  # nothing from torch's pool either
        Bh = B.cpu().numpy().T
        sh = st.cpu().numpy()
        assert np.array_equal(sh, splan) and np.array_equal(sh, sora)
        ok = sora == 0
        assert relerr(Bh, Bplan).max() <= TOL, f"call {call}: against the plan"
        assert relerr(Bh[:, ok], Bora[:, ok]).max() <= TOL, f"call {call}: against the oracle"


def test_static_entry_point_rejects_oversize(lib):
    # ceil(n/64) * (p+1) * k must fit 524288 doubles
    n, p, k = 4096, 20, 1000
    rc = lib.gls_solve_block_fp64_static(n, p, 1, n, 1, n, 1, 1, 1, n, k, 1, p, None, None)
    assert rc == 1
    assert "static scratch" in gls.last_error()
    # one SNP past the exact fit of the parity case above
    rc = lib.gls_solve_block_fp64_static(512, 3, 1, 512, 1, 512, 1, 1, 1, 512, 16385, 1, 3,
                                         None, None)
    assert rc == 1 and "static scratch" in gls.last_error()
    rc = lib.gls_solve_block_fp64_static(n, 0, 1, n, 1, n, 1, 1, 1, n, k, 1, p, None, None)
    assert rc == 1

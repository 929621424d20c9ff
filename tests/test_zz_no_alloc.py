"""The allocation-free FP64 block solve (gls_solve_block_fp64_static).

Callers that cannot call cudaMalloc pass their own device buffers; the only
scratch is a fixed 4 MiB array inside the library.  Two calls in a row must
each agree with the plan-based gls_solve_block within the FP64 tolerance
(1e-10 relative on b_i), and sizes beyond the scratch must be rejected.
This file is collected last so that a failure here leaves every other test
already run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import scipy.linalg as sla

from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import relerr, run_gpu

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


def test_static_entry_point_matches_plan_twice(lib):
    import torch
    n, p, k = 300, 5, 400
    pr = synth.problem(n, p, k, 0.5, seed=77, n_markers=400)
    Bref, sref = run_gpu(pr, "fp64")
    Z, W, R, zT = factor_products(pr)
    dev = "cuda:0"
    # row-major storage of the transposes = column-major storage of Z, W, R
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev)
    Wd = torch.from_numpy(np.ascontiguousarray(W.T)).to(dev)
    Rd = torch.from_numpy(np.ascontiguousarray(R.T)).to(dev)
    zd = torch.from_numpy(np.ascontiguousarray(zT)).to(dev)
    XR = torch.from_numpy(np.ascontiguousarray(pr["XR"].T)).to(dev)     # (k, n)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        B = torch.full((k, p), -1.0, dtype=torch.float64, device=dev)
        st = torch.full((k,), -1, dtype=torch.int32, device=dev)
        rc = lib.gls_solve_block_fp64_static(
            n, p, Zd.data_ptr(), n, Wd.data_ptr(), n, Rd.data_ptr(), zd.data_ptr(),
            XR.data_ptr(), n, k, B.data_ptr(), p, st.data_ptr(), stream)
        assert rc == 0, gls.last_error()
        torch.cuda.synchronize()
        Bh = B.cpu().numpy().T
        assert np.array_equal(st.cpu().numpy(), sref)
        assert relerr(Bh, Bref).max() <= TOL, f"call {call}"


def test_static_entry_point_rejects_oversize(lib):
    # ceil(n/64) * (p+1) * k must fit 524288 doubles
    n, p, k = 4096, 20, 1000
    rc = lib.gls_solve_block_fp64_static(n, p, 1, n, 1, n, 1, 1, 1, n, k, 1, p, None, None)
    assert rc == 1
    assert "static scratch" in gls.last_error()
    rc = lib.gls_solve_block_fp64_static(n, 0, 1, n, 1, n, 1, 1, 1, n, k, 1, p, None, None)
    assert rc == 1

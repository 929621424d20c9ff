"""Helpers shared by the GPU parity tests: device staging of a problem and one
call path through the C ABI."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1210_7325_gb300 import gls


def relerr(B, Bref):
    num = np.linalg.norm(B - Bref, axis=0)
    den = np.linalg.norm(Bref, axis=0)
    return num / den


def to_device(pr, dev="cuda:0"):
    import torch
    M = torch.from_numpy(np.ascontiguousarray(pr["M"].T)).to(dev).t()  # column-major
    XL = pr["XL"]
    XLd = torch.from_numpy(np.ascontiguousarray(XL.T)).to(dev).t() if XL.shape[1] else None
    y = torch.from_numpy(np.ascontiguousarray(pr["y"])).to(dev)
    XR = torch.from_numpy(np.ascontiguousarray(pr["XR"].T)).to(dev)  # (m, n)
    return M, XLd, y, XR


def run_gpu(pr, precision="fp64", kmax=None, split_terms=0, flags=0, host=False):
    """Factor + one block on the GPU; returns (B p x m numpy, status numpy)."""
    import torch
    n, m = pr["XR"].shape
    p = pr["XL"].shape[1] + 1
    kmax = kmax or max(m, 1)
    with gls.Plan(n, p, kmax, precision=precision, split_terms=split_terms,
                  flags=flags) as plan:
        if host:
            XL = np.asfortranarray(pr["XL"]) if p > 1 else None
            plan.factor(np.asfortranarray(pr["M"]), XL, np.ascontiguousarray(pr["y"]))
            B = np.zeros((p, m), order="F")
            st = np.zeros(m, np.int32)
            for s0 in range(0, m, kmax):
                k = min(kmax, m - s0)
                plan.solve_block(np.asfortranarray(pr["XR"][:, s0:s0 + k]),
                                 B[:, s0:s0 + k], st[s0:s0 + k], k=k)
            return B, st
        M, XL, y, XR = to_device(pr)
        plan.factor(M, XL, y)
        B = torch.empty((m, p), dtype=torch.float64, device="cuda:0")
        st = torch.empty(m, dtype=torch.int32, device="cuda:0")
        for s0 in range(0, m, kmax):
            k = min(kmax, m - s0)
            plan.solve_block(XR[s0:s0 + k].t(), B[s0:s0 + k].t(), st[s0:s0 + k], k=k)
        plan.synchronize()
        return B.cpu().numpy().T.copy(order="F"), st.cpu().numpy()


def oracle_ref(pr, tau):
    XL = pr["XL"] if pr["XL"].shape[1] else None
    B, st, info = oracle.gls(pr["M"], XL, pr["y"], pr["XR"], tau=tau,
                             nthreads=oracle.default_threads())
    assert info == 0
    return B, st

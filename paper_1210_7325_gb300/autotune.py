"""Autotuner for the batched mixed-precision solve.

Two knobs do not change results (each work item's arithmetic is the same
whichever CTA runs it), only speed:
  * group  -- row-block pairs per L2 rasterization group of a launch;
  * block  -- SNPs per plan per launch (bounded by max_block_snps).
One trades accuracy for speed and is gated by a measured error:
  * split  -- 16-bit slices of L^{-1} (2 or 3), ``tune_split``.
``tune_group`` times each candidate group on the caller's real launch with CUDA
events on the launching stream and keeps the fastest; results are cached in a
small JSON file keyed by device name and a signature of the batch, so later
runs with the same shapes skip the trials.
"""
from __future__ import annotations

import json
import os
import threading

DEFAULT_GROUPS = (1, 2, 3, 4, 6, 8)
_lock = threading.Lock()


def cache_path() -> str:
    base = os.environ.get("GLS_GB300_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "gls_gb300")
    return os.path.join(base, "autotune.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only loses the cache


def signature(plans, ks) -> str:
    """Shapes that determine the launch: (n, p, k) per plan, sorted, and precision."""
    shapes = sorted((p.n, p.p, int(k)) for p, k in zip(plans, ks))
    prec = plans[0].precision if plans else "?"
    return f"{prec}:" + ";".join(f"{n}x{p}x{k}" for n, p, k in shapes)


def device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


def tune_group(batch, XRs, Bs, statuses=None, ks=None, candidates=DEFAULT_GROUPS, reps: int = 2,
               use_cache: bool = True) -> tuple[int, dict]:
    """Returns (best group, {group: seconds}) for this batch launch."""
    import torch
    if ks is None:
        ks = [X.shape[1] for X in XRs]
    key = device_name() + "|" + signature(batch.plans, ks)
    if use_cache:
        with _lock:
            hit = _load().get(key)
        if hit:
            return int(hit["group"]), {int(g): t for g, t in hit["times"].items()}
    stream = torch.cuda.ExternalStream(batch.plans[0].stream)
    times = {}
    for g in candidates:
        batch.solve(XRs, Bs, statuses, ks, group=g)  # warm-up (also validates)
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.solve(XRs, Bs, statuses, ks, group=g)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        times[int(g)] = best
    group = min(times, key=times.get)
    if use_cache:
        with _lock:
            d = _load()
            d[key] = {"group": group, "times": {str(g): t for g, t in times.items()}}
            _store(d)
    return group, times


def choose_block(m: int, kmax: int, rounds_hint: int = 0) -> int:
    """SNPs per launch for a scan of m SNPs: the largest block up to kmax that
    splits m into equal rounds (fewer ragged tails across the batch)."""
    if m <= kmax:
        return max(m, 1)
    rounds = max(rounds_hint, -(-m // kmax))
    return -(-m // rounds)


def tune_split(n, p, precision, M, XL, y, XR_sample, tol: float = 1e-6, margin: float = 8.0,
               device: int = 0) -> tuple[int, dict]:
    """Operand split of L^{-1} (2 or 3 16-bit slices) for one scan of the mixed
    paths: the 2-slice split does two thirds of the tensor work, and is chosen
    only when its b_i on a sample of the scan's SNPs stay within tol / margin
    of the 3-slice b_i (relative 2-norm per SNP).  The 3-slice error is far
    below the 2-slice one (BF16: about 1/100 of it; FP16: about 1/10), so
    that difference bounds the 2-slice error to within the margin.  The
    caller's tolerance is for the whole scan; the margin covers SNPs outside
    the sample.  Arrays are device tensors in the layouts of ``gls.Plan``
    (M and XL column-major, XR_sample n x k column-major); returns
    (split_terms, {"err_2_vs_3": max relative difference, "threshold": ...}).
    """
    import numpy as np
    import torch
    from . import gls
    k = XR_sample.shape[1]
    outs = {}
    for S in (3, 2):
        with gls.Plan(n, p, k, precision=precision, device=device, split_terms=S) as pl:
            pl.factor(M, XL, y)
            B = torch.empty((k, p), dtype=torch.float64, device=XR_sample.device)
            st = torch.empty(k, dtype=torch.int32, device=XR_sample.device)
            pl.solve_block(XR_sample, B.t(), st, k=k)
            pl.synchronize()
            outs[S] = (B.cpu().numpy(), st.cpu().numpy())
    (B3, s3), (B2, s2) = outs[3], outs[2]
    ok = (s3 == 0) & (s2 == 0)
    num = np.linalg.norm(B2[ok] - B3[ok], axis=1)
    den = np.linalg.norm(B3[ok], axis=1)
    err = float((num / np.where(den > 0, den, 1.0)).max()) if ok.any() else float("inf")
    thr = tol / margin
    same_status = bool(np.array_equal(s2, s3))
    S = 2 if (err <= thr and same_status) else 3
    return S, {"err_2_vs_3": err, "threshold": thr, "status_agree": same_status}

#!/usr/bin/env python
"""Benchmark: GLS solves/s for the GWAS sequence b_i = (X_i^T M^{-1} X_i)^{-1} X_i^T M^{-1} y.

Default workload (the headline configuration): n = 10^4 individuals,
p = 20 (intercept + 18 covariates + the SNP), m = 10^6 int8 SNPs, h = 0.5,
mixed-precision path (BF16 slices of L^{-1}, tcgen05 tensor cores).  One step
is the whole hot path over the batch: gls_factor (Cholesky of M, L^{-1},
whitening, fixed Gram) + gls_solve_block over every SNP block, inputs resident
in HBM.  Inputs (10 GB of genotypes) are far larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line on rank 0.  ``--impl reference`` times the plain FP64
CPU oracle on the host cores instead (bounded sample of the same workload).
Multi-GPU runs are independent replicas (the method needs no exchange between
SNP ranges): value = all ranks' solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLS solves/s at n=1e4 (mixed vs FP64 @1e-6 rel err); serve p50/p99 latency"
UNIT = "solves/s"

WORKLOADS = {
    # name: n, p, m, h, precision, block
    "n10000_p20_m1000000_bf16": dict(n=10000, p=20, m=1_000_000, h=0.5, precision="bf16",
                                     block=65536, seed_offset=2),
    "n10000_p20_m1000000_fp16": dict(n=10000, p=20, m=1_000_000, h=0.5, precision="fp16",
                                     block=65536, seed_offset=2),
    # the headline scan on the binary64 path, in full (about 85 s per step)
    "n10000_p20_m1000000_fp64": dict(n=10000, p=20, m=1_000_000, h=0.5, precision="fp64",
                                     block=65536, seed_offset=2),
    # the headline n with two SNP blocks: profiler captures of the solve kernel (~6 GB)
    "n10000_p20_m131072_bf16": dict(n=10000, p=20, m=131072, h=0.5, precision="bf16",
                                    block=65536, seed_offset=2),
    # mid-size case for profiler captures: genotypes 268 MB (> L2), ~2 GB on the device
    "n4096_p20_m65536_bf16": dict(n=4096, p=20, m=65536, h=0.5, precision="bf16",
                                  block=65536, seed_offset=2),
    # a mid-size scan, the middle of the serving mix
    "n2000_p12_m131072_bf16": dict(n=2000, p=12, m=131072, h=0.5, precision="bf16",
                                   block=65536, seed_offset=4),
    "n1000_p4_m4096_fp64": dict(n=1000, p=4, m=4096, h=0.4, precision="fp64", block=4096,
                                seed_offset=0),
    "n1500_p4_m2500000_fp64": dict(n=1500, p=4, m=2_500_000, h=0.5, precision="fp64",
                                   block=16384, seed_offset=1),
}
DEFAULT_WORKLOAD = "n10000_p20_m1000000_bf16"

# DRAM bytes (read + write) of one launch of the mixed blocked-solve kernel, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the current
# kernel at that launch size: (precision, n, SNPs per launch) -> bytes.
TRSM_TRAFFIC = {("bf16", 10000, 65536): 13.476e9 + 0.0501e9}

# Batched uneven scans: each scan its own kinship, h ~ U(0.1, 0.9); one persistent
# launch per round serves one block of every scan.
BATCH_WORKLOADS = {
    "batch48_uneven_bf16": dict(scans=48, n=(500, 8000), p=(2, 20), m=(10_000, 500_000),
                                h=(0.1, 0.9), precision="bf16", block=65536, seed_offset=3),
    "batch48_uneven_fp16": dict(scans=48, n=(500, 8000), p=(2, 20), m=(10_000, 500_000),
                                h=(0.1, 0.9), precision="fp16", block=65536, seed_offset=3),
    # The FP64 path needs about 4 minutes per step at full m (2.8e14 FP64 flops),
    # so the FP64 comparison runs every scan's first m/32 SNPs, beside the mixed
    # path on the same reduced scans.
    "batch48_uneven_m32_fp64": dict(scans=48, n=(500, 8000), p=(2, 20), m=(10_000, 500_000),
                                    h=(0.1, 0.9), precision="fp64", block=16384, seed_offset=3,
                                    m_div=32),
    "batch48_uneven_m32_bf16": dict(scans=48, n=(500, 8000), p=(2, 20), m=(10_000, 500_000),
                                    h=(0.1, 0.9), precision="bf16", block=65536, seed_offset=3,
                                    m_div=32),
}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
        "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


# ----------------------------------------------------------------------------- inputs
def make_inputs(wl, rank, torch):
    from paper_1210_7325_gb300 import synth
    seed = synth.BASE_SEED + wl["seed_offset"] + 1000 * rank
    n, p, m = wl["n"], wl["p"], wl["m"]
    M = synth.kinship_M(n, wl["h"], seed, device="cuda")
    XL = synth.covariates(n, p, seed)
    y = synth.phenotype(n, seed)
    XR = synth.genotypes_torch(n, m, seed, device="cuda")  # (m, n) int8 = column-major n x m
    return M, XL, y, XR


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args, wl, rank, world, torch, dist):
    import numpy as np
    from paper_1210_7325_gb300 import gls

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    n, p, m, kmax, prec = wl["n"], wl["p"], wl["m"], wl["block"], wl["precision"]
    M, XL, y, XR = make_inputs(wl, rank, torch)
    Md = torch.from_numpy(np.ascontiguousarray(M.T)).to(dev).t()  # column-major
    XLd = torch.from_numpy(np.ascontiguousarray(XL.T)).to(dev).t()
    yd = torch.from_numpy(y).to(dev)
    B = torch.empty((m, p), dtype=torch.float64, device=dev)
    st = torch.empty(m, dtype=torch.int32, device=dev)
    split, split_info = 0, None
    if prec != "fp64":
        from paper_1210_7325_gb300 import autotune
        split, split_info = autotune.tune_split(n, p, prec, Md, XLd, yd, XR[:512].t(),
                                                tol=1e-6, device=dev.index)
    plan = gls.Plan(n, p, kmax, precision=prec, device=dev.index, split_terms=split,
                    flags=launch_flags(args, gls))
    stream = torch.cuda.ExternalStream(plan.stream, device=dev)

    def step():
        # the scan held in HBM, in blocks of kmax SNPs
        plan.factor(Md, XLd, yd)
        plan.solve_stream(XR.t(), B.t(), st, m=m)

    for _ in range(args.warmup):
        step()
    plan.synchronize()
    plan.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id_for(torch, dev)) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t = e0.elapsed_time(e1) / 1e3
    stats = plan.stats()
    bad = int((st != 0).sum().item())
    nan = int(torch.isnan(B).any().item())
    res = dict(time=t, stats=stats, clocks=clk.summary(), bad_status=bad, nan=nan,
               split=split or None, split_info=split_info)
    # the oracle leg solves a seeded sample of the timed run's own SNP columns
    cols = sample_columns(m, args.cpu_snps, seed=rank)
    ci = torch.as_tensor(cols, device=dev)
    res["sample"] = dict(cols=cols, XR=np.asfortranarray(XR[ci].cpu().numpy().T),
                         B=B[ci].cpu().numpy().T.copy(), st=st[ci].cpu().numpy(),
                         M=M, XL=XL, y=y)

    # end to end through the public API with host buffers (pinned); per-kernel
    # timing is instrumentation a user would not run with, so it is off here
    if not args.skip_e2e:
        plan.set_timing(False)
        XRh = torch.empty((m, n), dtype=torch.int8, pin_memory=True)
        XRh.copy_(XR)
        # the same genotypes packed four to a byte (the usual GWAS storage form)
        XPd = gls.pack_genotypes(XR.t())                  # (ceil(n/4), m) column-major
        XPh = torch.empty((m, XPd.shape[0]), dtype=torch.uint8, pin_memory=True)
        XPh.copy_(XPd.t())
        del XPd
        Mh = torch.from_numpy(np.ascontiguousarray(M.T)).pin_memory().t()
        XLh = torch.from_numpy(np.ascontiguousarray(XL.T)).pin_memory().t()
        yh = torch.from_numpy(y).pin_memory()
        Bh = torch.empty((m, p), dtype=torch.float64, pin_memory=True)
        sh = torch.empty(m, dtype=torch.int32, pin_memory=True)
        del XR
        torch.cuda.empty_cache()

        def e2e_int8():
            plan.factor(Mh, XLh, yh)
            plan.solve_stream(XRh.t(), Bh.t(), sh, m=m)

        def e2e_step():
            plan.factor(Mh, XLh, yh)
            plan.solve_stream_packed(XPh.t(), Bh.t(), sh, m=m)

        def timed(fn):
            for _ in range(max(1, min(args.warmup, 2))):
                fn()
            if dist:
                dist.barrier()
            marks = [time.perf_counter()]
            for _ in range(args.steps):
                fn()
                marks.append(time.perf_counter())
            return marks[-1] - marks[0], [round((b - a) * 1e3, 2)
                                          for a, b in zip(marks, marks[1:])]

        res["e2e_int8_time"], res["e2e_int8_step_ms"] = timed(e2e_int8)
        te, res["e2e_step_ms"] = timed(e2e_step)
        res["e2e_time"] = te
        # one more step of each with per-kernel device timing and every block
        # copy timed on its side stream while overlapped (not in the figures):
        # does the step's time go to the kernels or to waiting on the host link?
        def diag(fn):
            plan.set_timing(True)
            t1 = time.perf_counter()
            fn()
            t2 = time.perf_counter()
            sd = plan.stats()
            plan.set_timing(False)
            return {"wall_ms": round((t2 - t1) * 1e3, 2),
                    "factor_ms": round(sd["factor_ms"], 2),
                    "trsm_ms": round(sd["trsm_ms"], 2),
                    "convert_ms": round(sd["convert_ms"], 2),
                    "solve_pxp_ms": round(sd["solve_ms"], 2),
                    "h2d_copies": sd["h2d_copies"], "h2d_ms": round(sd["h2d_ms"], 2),
                    "h2d_gbps_overlapped": (sd["h2d_bytes"] / (sd["h2d_ms"] / 1e3) / 1e9
                                            if sd["h2d_ms"] > 0 else None),
                    "d2h_ms": round(sd["d2h_ms"], 2),
                    "d2h_gbps_overlapped": (sd["d2h_bytes"] / (sd["d2h_ms"] / 1e3) / 1e9
                                            if sd["d2h_ms"] > 0 else None)}
        res["e2e_diag"] = diag(e2e_step)
        res["e2e_int8_diag"] = diag(e2e_int8)
        # the int8 stream through the copy engine (the pre-existing staged path) on a
        # plan of its own, for comparison with the in-place reads above
        plan_st = gls.Plan(n, p, kmax, precision=prec, device=dev.index, split_terms=split,
                           flags=launch_flags(args, gls) | gls.GLS_FLAG_STAGED_INPUT)

        def e2e_int8_staged():
            plan_st.factor(Mh, XLh, yh)
            plan_st.solve_stream(XRh.t(), Bh.t(), sh, m=m)

        e2e_int8_staged()  # warm-up
        steps_st = min(args.steps, 3)
        marks = [time.perf_counter()]
        for _ in range(steps_st):
            e2e_int8_staged()
            marks.append(time.perf_counter())
        res["e2e_int8_staged"] = {
            "steps": steps_st, "value": m * steps_st / (marks[-1] - marks[0]),
            "step_ms": [round((b - a) * 1e3, 2) for a, b in zip(marks, marks[1:])]}
        plan_st.close()
        # context for the end-to-end figure: this box's pinned host -> device copy rate
        # ... over every block of the pinned genotype buffer (placement of its
        # pages can differ along the buffer), best of 3 per block
        probe = torch.empty((min(m, kmax), n), dtype=torch.int8, device=dev)
        rates = []
        for s0 in range(0, m, kmax):
            k = min(kmax, m - s0)
            best = float("inf")
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                probe[:k].copy_(XRh[s0:s0 + k], non_blocking=True)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            rates.append(k * n / best / 1e9)
        # and the device -> host return of b into the pinned output buffer
        bdev = torch.empty((min(m, kmax), p), dtype=torch.float64, device=dev)
        best = float("inf")
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            Bh[:bdev.shape[0]].copy_(bdev, non_blocking=True)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        res["d2h_gbps"] = bdev.numel() * 8 / best / 1e9
        del bdev
        res["h2d_gbps"] = rates[0]
        res["h2d_gbps_blocks"] = {"min": min(rates), "median": float(np.median(rates)),
                                  "max": max(rates), "blocks": len(rates)}
        del probe
        res["e2e_h2d"] = n * n * 8 + n * (p - 1) * 8 + n * 8 + gls.packed_rows(n) * m
        res["e2e_int8_h2d"] = n * n * 8 + n * (p - 1) * 8 + n * 8 + n * m
        res["e2e_d2h"] = p * m * 8 + 4 * m
    plan.close()
    return res


def run_factor_only(args, wl, torch):
    """gls_factor alone (Cholesky of M, L^{-1}, whitening, fixed Gram), timed
    with CUDA events on the plan's stream; a profiling and tuning aid."""
    import numpy as np
    from paper_1210_7325_gb300 import gls
    n, p, prec = wl["n"], wl["p"], wl["precision"]
    M, XL, y, _ = make_inputs(dict(wl, m=1), 0, torch)
    Md = torch.from_numpy(np.ascontiguousarray(M.T)).cuda().t()
    XLd = torch.from_numpy(np.ascontiguousarray(XL.T)).cuda().t()
    yd = torch.from_numpy(y).cuda()
    flags = gls.GLS_FLAG_FACTOR_NATIVE if (args.factor_native and prec != "fp64") else 0
    plan = gls.Plan(n, p, 1024, precision=prec, flags=flags | launch_flags(args, gls))
    for _ in range(args.warmup):
        plan.factor(Md, XLd, yd)
    plan.synchronize()
    plan.set_timing(True)
    for _ in range(args.steps):
        plan.factor(Md, XLd, yd)
    s = plan.stats()
    plan.close()
    return {"metric": "gls_factor time", "value": s["factor_ms"] / args.steps, "unit": "ms",
            "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": args.workload, "n": n, "p": p, "precision": prec,
                       "factor": "binary64 CUDA cores" if flags else
                       ("tensor-core exact slices" if prec != "fp64" else "binary64 CUDA cores")},
            "gpu_launches_per_call": s["launches"] / args.steps}


def fp64_sample(wl, torch, m_sample=16384):
    """FP64 GPU path on the same n, p over one block of SNPs (its full m would
    take minutes at the binary64 rate of this part)."""
    import numpy as np
    from paper_1210_7325_gb300 import gls, synth
    n, p = wl["n"], wl["p"]
    seed = synth.BASE_SEED + wl["seed_offset"]
    M = synth.kinship_M(n, wl["h"], seed, device="cuda")
    XL = synth.covariates(n, p, seed)
    y = synth.phenotype(n, seed)
    XR = synth.genotypes_torch(n, m_sample, seed, device="cuda")
    dev = torch.device("cuda")
    Md = torch.from_numpy(np.ascontiguousarray(M.T)).to(dev).t()
    XLd = torch.from_numpy(np.ascontiguousarray(XL.T)).to(dev).t()
    yd = torch.from_numpy(y).to(dev)
    B = torch.empty((m_sample, p), dtype=torch.float64, device=dev)
    plan = gls.Plan(n, p, m_sample, precision="fp64")
    plan.factor(Md, XLd, yd)
    plan.solve_block(XR.t(), B.t(), None, k=m_sample)
    plan.synchronize()
    plan.set_timing(True)
    plan.factor(Md, XLd, yd)
    plan.solve_block(XR.t(), B.t(), None, k=m_sample)
    s = plan.stats()
    plan.close()
    solve_s = (s["trsm_ms"] + s["solve_ms"]) / 1e3
    factor_s = s["factor_ms"] / 1e3
    return dict(m_sample=m_sample, factor_s=factor_s, solve_s=solve_s,
                steady_solves_per_s=m_sample / solve_s,
                trsm_fp64_tflops=n * n * m_sample / (s["trsm_ms"] / 1e3) / 1e12,
                whole_job_solves_per_s_projected=wl["m"] / (factor_s + wl["m"] / m_sample * solve_s))


def fp64_dgemm_tflops(torch):
    a = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(3):
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2 * 8192 ** 3 / best / 1e12


# ----------------------------------------------------------------------------- CPU oracle
def sample_columns(m, count, seed=0):
    """SNP columns checked against the oracle: the first half of `count` in
    order, the rest seeded uniform over the whole scan (sorted, distinct)."""
    import numpy as np
    count = min(count, m)
    head = np.arange(count // 2)
    rest = np.random.Generator(np.random.Philox(20121030 + seed)).choice(
        np.arange(count // 2, m), size=count - count // 2, replace=False)
    return np.sort(np.concatenate([head, rest])).astype(np.int64)


def oracle_sample(wl, nthreads, M, XL, y, XR):
    """Times the oracle as it stands on the host: the Cholesky of M once, then
    the per-SNP loop on the columns of XR (n x s int8).  Returns the timings,
    the projected whole-job rate for the workload's m, and the oracle's b_i."""
    import oracle
    s_snps = XR.shape[1]
    t0 = time.perf_counter()
    L, info = oracle.potrf(M, nthreads=nthreads)
    t1 = time.perf_counter()
    tau = oracle.TAU_FP64 if wl["precision"] == "fp64" else oracle.TAU_MIXED
    B, st = oracle.gls_factored(L, XL, y, XR, tau=tau, nthreads=nthreads)
    t2 = time.perf_counter()
    assert info == 0
    tf, ts = t1 - t0, t2 - t1
    whole = wl["m"] / (tf + wl["m"] / s_snps * ts)
    return dict(factor_s=tf, snp_s=ts, s_snps=s_snps, value=whole,
                steady=s_snps / ts, cores=nthreads, B=B, st=st)


def error_summary(B, st, Bref, sref, tol):
    """Relative 2-norm error of b_i against the oracle's on the same SNPs."""
    import numpy as np
    ok = sref == 0
    e = np.linalg.norm(B[:, ok] - Bref[:, ok], axis=0) / np.linalg.norm(Bref[:, ok], axis=0)
    return {"max": float(e.max()) if e.size else None,
            "p99": float(np.quantile(e, 0.99)) if e.size else None,
            "n_sampled": int(B.shape[1]), "status_mismatches": int((st != sref).sum()),
            "tolerance": tol, "reference": "FP64 oracle on the same SNP columns"}


def run_reference(args, wl):
    """--impl reference: the FP64 oracle on the host cores, same metric/config."""
    import numpy as np  # noqa: F401
    import oracle
    from paper_1210_7325_gb300 import synth
    nthreads = oracle.default_threads()
    n, p = wl["n"], wl["p"]
    seed = synth.BASE_SEED + wl["seed_offset"]
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
    except Exception:
        dev = "cpu"
    M = synth.kinship_M(n, wl["h"], seed, device=dev)
    XL = synth.covariates(n, p, seed)
    y = synth.phenotype(n, seed)
    s_snps = args.ref_snps
    XR = synth.genotypes_np(n, s_snps, seed)
    for _ in range(args.warmup):
        oracle_sample(wl, nthreads, M, XL, y, XR)
    vals, steps = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle_sample(wl, nthreads, M, XL, y, XR)
        steps.append(r)
        vals.append(r["value"])
    total = time.perf_counter() - t0
    value = statistics.median(vals)
    sample = (f"per step: oracle Cholesky of M (n={n}) + per-SNP loop on {s_snps} SNPs; "
              f"value = m / (t_factor + m/{s_snps} * t_snps) for m={wl['m']}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_for(wl, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                         "sample": sample,
                         "factor_s": statistics.median(r["factor_s"] for r in steps),
                         "snp_s": statistics.median(r["snp_s"] for r in steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_specs(bw):
    """Seeded (n, p, m, h, seed) per scan."""
    import numpy as np
    from paper_1210_7325_gb300 import synth
    g = synth.rng(synth.BASE_SEED + bw["seed_offset"], 99)
    out = []
    for i in range(bw["scans"]):
        n = int(g.integers(bw["n"][0], bw["n"][1] + 1))
        p = int(g.integers(bw["p"][0], bw["p"][1] + 1))
        m = int(g.integers(bw["m"][0], bw["m"][1] + 1))
        h = float(g.uniform(*bw["h"]))
        m = max(1, m // bw.get("m_div", 1))
        out.append((n, p, m, h, synth.BASE_SEED + bw["seed_offset"] * 1000 + i))
    return out


def run_batch_workload(args, bw, torch):
    """Config: 48 uneven scans.  One step = every scan's gls_factor (concurrent
    streams) + rounds until every scan is solved.  A mixed-precision round is ONE
    batched persistent launch over the next block of every scan; an FP64 round
    launches every scan's block on its own plan stream (they overlap)."""
    import concurrent.futures as cf
    import numpy as np
    from paper_1210_7325_gb300 import autotune, gls, synth
    specs = batch_specs(bw)
    plans, inputs, outs, blocks = [], [], [], []
    fp64 = bw["precision"] == "fp64"
    t_setup = time.perf_counter()
    for (n, p, m, h, seed) in specs:
        Md = synth.kinship_M_torch(n, h, seed, device="cuda").t()
        XL = synth.covariates(n, p, seed)
        y = synth.phenotype(n, seed)
        XR = synth.genotypes_torch(n, m, seed, device="cuda")
        XLd = torch.from_numpy(np.ascontiguousarray(XL.T)).cuda().t()
        yd = torch.from_numpy(y).cuda()
        inputs.append((Md, XLd, yd, XR))
    # split factor: one batch shares one split, so the first scan that needs
    # the 3-slice split settles it (2 slices only if every scan admits it)
    split, split_trials = 3, []
    if not fp64:
        split = 2
        for (n, p, m, h, seed), (Md, XLd, yd, XR) in zip(specs, inputs):
            S, info = autotune.tune_split(n, p, bw["precision"], Md, XLd, yd,
                                          XR[:min(m, 512)].t(), tol=1e-6)
            split_trials.append(dict(info, n=n, p=p, split=S))
            if S == 3:
                split = 3
                break
    for (n, p, m, h, seed) in specs:
        kb = autotune.choose_block(m, bw["block"])
        plans.append(gls.Plan(n, p, kb, precision=bw["precision"],
                              split_terms=0 if fp64 else split, flags=launch_flags(args, gls)))
        outs.append((torch.empty((m, p), dtype=torch.float64, device="cuda"),
                     torch.empty(m, dtype=torch.int32, device="cuda")))
        blocks.append(kb)
    rounds = max(-(-m // kb) for (_, _, m, _, _), kb in zip(specs, blocks))
    pool = cf.ThreadPoolExecutor(max_workers=8)

    def factor_all():
        list(pool.map(lambda i: plans[i].factor(*inputs[i][:3]), range(len(plans))))

    def round_args(r):
        XRs, Bs, sts, ks = [], [], [], []
        for i, (n, p, m, h, seed) in enumerate(specs):
            s0 = min(r * blocks[i], m)
            k = min(blocks[i], m - s0)
            XRs.append(inputs[i][3][s0:s0 + k].t())
            Bs.append(outs[i][0][s0:s0 + k].t())
            sts.append(outs[i][1][s0:s0 + k])
            ks.append(k)
        return XRs, Bs, sts, ks

    factor_all()
    if fp64:
        batch, group, tune_times = None, None, None
    else:
        batch = gls.Batch(plans)
        group, tune_times = autotune.tune_group(batch, *round_args(0))
    rargs = [round_args(r) for r in range(rounds)]
    t_setup = time.perf_counter() - t_setup

    def step():
        factor_all()
        for r in range(rounds):
            if fp64:
                XRs, Bs, sts, ks = rargs[r]
                for i, pl in enumerate(plans):
                    if ks[i] > 0:
                        pl.solve_block(XRs[i], Bs[i], sts[i], k=ks[i])
            else:
                batch.solve(*rargs[r], group=group)
        for pl in plans:
            pl.synchronize()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # timing of phases: on plan 0 for the batch (it carries every batched
    # launch); on every plan for FP64 (each runs on its own stream)
    for i, pl in enumerate(plans):
        pl.set_timing(fp64 or i == 0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    sts = [pl.stats() for pl in plans]
    st0 = {key: (sum(s[key] for s in sts) if fp64 else sts[0][key]) for key in sts[0]}
    total_m = sum(sp[2] for sp in specs)
    unit_flops = 1 if fp64 else split
    tensor_flops = sum(unit_flops * n * n * m for (n, p, m, h, seed) in specs) * args.steps
    bad = sum(int((o[1] != 0).sum().item()) for o in outs)
    peaks, peak_src = load_peaks()
    trsm_s = st0["trsm_ms"] / 1e3
    achieved = tensor_flops / trsm_s / 1e12 if trsm_s > 0 else None
    if fp64:
        fpk = fp64_dgemm_tflops(torch)
        roof = {"bound": "fp64", "achieved": achieved, "peak": fpk, "unit": "TFLOP/s",
                "frac": achieved / fpk if achieved else None, "traffic": None,
                "peak_source": "measured torch.matmul float64 8192^3 in this run",
                "per_unit": "n^2 FP64 flops per SNP; achieved uses the summed kernel time of "
                            "the 48 streams, so overlap makes it a lower bound"}
    else:
        roof = {"bound": "tensor", "achieved": achieved,
                "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                "frac": achieved / peaks["bf16_tflops_sustained"] if achieved else None,
                "traffic": None, "peak_source": f"{peak_src} bf16_tflops_sustained",
                "per_unit": "3 slices x n^2 tensor flops per SNP"}
    line = {
        "metric": METRIC, "value": total_m * args.steps / t, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp16": "f16", "fp64": "f64"}[bw["precision"]],
        "data": "synthetic (48 seeded scans, own kinship each)",
        "config": {"workload": args.workload, "scans": bw["scans"], "total_snps": total_m,
                   "n_range": bw["n"], "p_range": bw["p"], "m_range": bw["m"],
                   "m_divisor": bw.get("m_div", 1),
                   "rounds": rounds, "group_autotuned": group,
                   "group_trials_s": tune_times,
                   "split_terms_autotuned": None if fp64 else split,
                   "split_trials": split_trials,
                   "launch": "eager" if args.eager else "CUDA-graph replay of repeated sequences",
                   "parallelism": "replicas1"},
        "gpu_launches": None,
        "phase_ms_per_step": {"solve_kernels": st0["trsm_ms"] / args.steps,
                              "convert": st0["convert_ms"] / args.steps,
                              "solve_pxp": st0["solve_ms"] / args.steps},
        "roofline": roof,
        "check": {"bad_status": bad},
    }
    line["gpu_launches"] = int(sum(s["launches"] for s in sts))
    line["config"]["setup_s"] = round(t_setup, 2)
    line["config"]["operand_precision"] = sorted({pl.operand_precision for pl in plans})
    line["error"] = batch_error(specs, inputs, outs, fp64)
    if batch is not None:
        batch.close()
    for pl in plans:
        pl.close()
    return line


def batch_error(specs, inputs, outs, fp64, max_scans=6, n_max=3000, snps=48):
    """b_i of the batched run against the oracle: every scan with n <= n_max
    (up to max_scans, smallest n first), `snps` seeded SNP columns each."""
    import numpy as np
    import torch

    import oracle
    order = sorted((sp[0], i) for i, sp in enumerate(specs) if sp[0] <= n_max)[:max_scans]
    tau = oracle.TAU_FP64 if fp64 else oracle.TAU_MIXED
    errs, mism, nsnp, scans = [], 0, 0, []
    for n, i in order:
        m = specs[i][2]
        Md, XLd, yd, XR = inputs[i]
        cols = sample_columns(m, snps, seed=i)
        ci = torch.as_tensor(cols, device=XR.device)
        Bref, sref, info = oracle.gls(Md.cpu().numpy(), XLd.cpu().numpy(), yd.cpu().numpy(),
                                      np.asfortranarray(XR[ci].cpu().numpy().T), tau=tau,
                                      nthreads=oracle.default_threads())
        if info != 0:
            continue
        B = outs[i][0][ci].cpu().numpy().T
        st = outs[i][1][ci].cpu().numpy()
        ok = sref == 0
        errs.append(np.linalg.norm(B[:, ok] - Bref[:, ok], axis=0)
                    / np.linalg.norm(Bref[:, ok], axis=0))
        mism += int((st != sref).sum())
        nsnp += len(cols)
        scans.append(int(n))
    if not errs:
        return {"max": None, "p99": None, "n_sampled": 0}
    e = np.concatenate(errs)
    return {"max": float(e.max()), "p99": float(np.quantile(e, 0.99)), "n_sampled": nsnp,
            "status_mismatches": mism, "tolerance": 1e-10 if fp64 else 1e-6,
            "reference": "FP64 oracle on the same SNP columns", "scans_n": scans}


SERVE_WORKLOADS = {
    "serve2000_bf16": dict(requests=2000, rate=20.0, n=(1000, 10000), p=(2, 12),
                           m=(10_000, 200_000), reuse=0.3, precision="bf16", block=32768,
                           seed_offset=4, budget=200e9, time_cap=420.0),
    "serve2000_fp64": dict(requests=2000, rate=20.0, n=(1000, 10000), p=(2, 12),
                           m=(10_000, 200_000), reuse=0.3, precision="fp64", block=32768,
                           seed_offset=4, budget=200e9, time_cap=120.0),
}


def serve_inputs_factory(bank, seed_base):
    """Request inputs as slices of a pre-drawn bank (synth.ServingBank): the
    server's latency then excludes synthesizing them."""
    from paper_1210_7325_gb300 import serve

    def make_inputs(req, torch, reuse):
        M, XL, y, XR = bank.request(req.n, req.p, req.m, req.h, seed_base + req.mkey,
                                    req.y_seed, with_factor_inputs=not reuse)
        return serve.Inputs(M, XL, XR, y)
    return make_inputs


def serve_kept(reqs, count=6, n_max=3000):
    """Request ids whose outputs the serving run keeps for the oracle check:
    `count` requests with n <= n_max spread over the stream (new and reused)."""
    small = [r for r in reqs if r.n <= n_max]
    if not small:
        return set()
    step = max(1, len(small) // count)
    return {r.rid for r in small[::step][:count]}


def serve_error(bank, seed_base, reqs, results, tau, snps=48):
    """Relative error of served b_i against the oracle: for every kept request,
    `snps` seeded SNP columns solved by the oracle from the same inputs."""
    import numpy as np
    import torch

    import oracle
    errs, nreq = [], 0
    for r in reqs:
        got = results.get(r.rid)
        if got is None or "B" not in got:
            continue
        M, XL, y, XR = bank.request(r.n, r.p, r.m, r.h, seed_base + r.mkey, r.y_seed)
        cols = np.sort(np.random.default_rng(r.rid).choice(r.m, size=min(snps, r.m),
                                                           replace=False))
        ci = torch.as_tensor(cols, device=XR.device)
        Xs = np.asfortranarray(XR[ci].cpu().numpy().T)
        Bref, sref, info = oracle.gls(M.cpu().numpy(), None if XL is None else XL.cpu().numpy(),
                                      y.cpu().numpy(), Xs, tau=tau,
                                      nthreads=oracle.default_threads())
        B = got["B"][ci].cpu().numpy().T
        st = got["status"][ci].cpu().numpy()
        if info != 0 or not np.array_equal(st, sref):
            errs.append(float("inf"))
            continue
        ok = sref == 0
        e = np.linalg.norm(B[:, ok] - Bref[:, ok], axis=0) / np.linalg.norm(Bref[:, ok], axis=0)
        errs.extend(float(v) for v in e)
        nreq += 1
    if not errs:
        return {"max": None, "p99": None, "n_sampled": 0, "requests": 0}
    a = np.array(errs)
    return {"max": float(a.max()), "p99": float(np.quantile(a, 0.99)), "n_sampled": int(a.size),
            "requests": nreq, "reference": "FP64 oracle on the same inputs",
            "tolerance": 1e-10 if tau == 2.0 ** -30 else 1e-6}


def run_serve_workload(args, sw, torch, time_cap=None):
    """Config: Poisson stream of scan requests served with continuous batching.
    Request inputs are slices of banks drawn before the clock starts; a sample
    of requests is checked against the oracle after the run."""
    import oracle
    from paper_1210_7325_gb300 import serve, synth
    seed = synth.BASE_SEED + sw["seed_offset"]
    count = getattr(args, "requests", 0) or sw["requests"]
    reqs = serve.poisson_requests(count, sw["rate"], seed, sw["n"], sw["p"], sw["m"],
                                  sw["reuse"])
    t_bank = time.perf_counter()
    bank = synth.ServingBank(sw["n"][1], sw["m"][1], seed * 7, device="cuda")
    torch.cuda.synchronize()
    t_bank = time.perf_counter() - t_bank
    make = serve_inputs_factory(bank, seed * 10)
    # warm-up: load kernels and encode maps on a few small requests (not timed)
    warm = serve.poisson_requests(4, 100.0, seed + 1, (1000, 1200), (2, 4), (2000, 4000), 0.0)
    srv = serve.Server(make, sw["precision"], sw["budget"], sw["block"])
    srv.run(warm)
    srv.close()
    kept = serve_kept(reqs)
    srv = serve.Server(make, sw["precision"], sw["budget"], sw["block"], keep=kept,
                       trace=getattr(args, "serve_trace", None))
    cap = time_cap or getattr(args, "time_cap", 0) or sw["time_cap"]
    t0 = time.perf_counter()
    results = srv.run(reqs, time_cap=cap)
    wall = time.perf_counter() - t0
    summ = serve.latency_summary(results)
    depth = [d[1] for d in srv.queue_depth]
    srv.close()
    tau = oracle.TAU_FP64 if sw["precision"] == "fp64" else oracle.TAU_MIXED
    err = serve_error(bank, seed * 10, [r for r in reqs if r.rid in kept], results, tau)
    line = {
        "metric": METRIC, "value": summ.get("solves_per_s", 0.0), "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": wall * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp16": "f16", "fp64": "f64"}[sw["precision"]],
        "data": "synthetic Poisson request stream (seeded); inputs sliced from banks drawn "
                "before the clock",
        "config": {"workload": getattr(args, "workload", None), "requests": count,
                   "rate_per_s": sw["rate"], "n_range": sw["n"], "p_range": sw["p"],
                   "m_range": sw["m"], "reuse_fraction": sw["reuse"],
                   "hbm_budget_bytes": sw["budget"], "block_snps": sw["block"],
                   "time_cap_s": cap, "bank_build_s": round(t_bank, 2),
                   "parallelism": "replicas1"},
        "latency": {k: v for k, v in summ.items() if k.endswith("_s")},
        "completed": summ.get("completed", 0), "reused_factors": summ.get("reused", 0),
        "error": err,
        "loop_breakdown": srv.breakdown,
        "queue_depth_max": max(depth) if depth else 0,
        "queue_depth_last": depth[-1] if depth else 0,
        "wall_s": wall,
    }
    del bank
    torch.cuda.empty_cache()
    return line


def sub_phenotypes(args, torch, ts=(1, 4, 13), steps=3, warmup=1):
    """The headline scan with t phenotypes per factor (Eq. 1's index j <= t):
    one pass over X_R serves t right-hand sides, so GLS solves (b_ij) per
    second grow with t while the step's time barely moves.  b_ij of three
    phenotypes of the largest t are checked against the oracle on sampled SNPs."""
    import numpy as np

    import oracle
    from paper_1210_7325_gb300 import gls, synth
    wl = WORKLOADS[DEFAULT_WORKLOAD]
    n, p, m, kmax, prec = wl["n"], wl["p"], wl["m"], wl["block"], wl["precision"]
    dev = torch.device("cuda")
    M, XL, y, XR = make_inputs(wl, 0, torch)
    Md = torch.from_numpy(np.ascontiguousarray(M.T)).to(dev).t()
    XLd = torch.from_numpy(np.ascontiguousarray(XL.T)).to(dev).t()
    tmax = max(ts)
    Y = np.column_stack([synth.phenotype(n, synth.BASE_SEED + 50 + j) for j in range(tmax)])
    rows, last = [], None
    for t in ts:
        Yd = torch.from_numpy(np.ascontiguousarray(Y[:, :t].T)).to(dev).t()
        B = torch.empty((m * t, p), dtype=torch.float64, device=dev)
        st = torch.empty(m, dtype=torch.int32, device=dev)
        plan = gls.Plan(n, p, kmax, precision=prec, phenotypes=t, flags=launch_flags(args, gls))
        stream = torch.cuda.ExternalStream(plan.stream, device=dev)

        def step():
            plan.factor(Md, XLd, Yd)
            for s0 in range(0, m, kmax):
                k = min(kmax, m - s0)
                plan.solve_block(XR[s0:s0 + k].t(), B[s0 * t:(s0 + k) * t].t(), st[s0:s0 + k],
                                 k=k)

        for _ in range(warmup):
            step()
        plan.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        rows.append({"phenotypes": t, "value": m * t * steps / sec,
                     "ms_per_step": sec / steps * 1e3, "bad_status": int((st != 0).sum())})
        plan.close()
        last = (t, B, st)
    base = rows[0]["value"]
    for r in rows:
        r["vs_t1"] = r["value"] / base
    # oracle check of the largest t: three phenotypes on 256 seeded SNPs
    t, B, st = last
    cols = sample_columns(m, 256, seed=7)
    ci = torch.as_tensor(cols, device=dev)
    Xs = np.asfortranarray(XR[ci].cpu().numpy().T)
    L, info = oracle.potrf(M, nthreads=oracle.default_threads())
    Bg = B.view(m, t, p)[ci].cpu().numpy()          # (s, t, p)
    sg = st[ci].cpu().numpy()
    errs, mism = [], 0
    for j in (0, t // 2, t - 1):
        Bref, sref = oracle.gls_factored(L, XL, Y[:, j], Xs, tau=oracle.TAU_MIXED,
                                         nthreads=oracle.default_threads())
        ok = sref == 0
        Bj = Bg[:, j, :].T
        errs.append(np.linalg.norm(Bj[:, ok] - Bref[:, ok], axis=0)
                    / np.linalg.norm(Bref[:, ok], axis=0))
        mism += int((sg != sref).sum())
    e = np.concatenate(errs)
    return {"workload": DEFAULT_WORKLOAD, "unit": "solves/s (one solve = one b_ij)",
            "steps": steps, "warmup": warmup, "rows": rows,
            "error": {"max": float(e.max()), "p99": float(np.quantile(e, 0.99)),
                      "n_sampled": int(e.size), "status_mismatches": mism, "tolerance": 1e-6,
                      "phenotypes_checked": [0, t // 2, t - 1],
                      "reference": "FP64 oracle on the same SNP columns, per phenotype"}}


def run_variants(torch, n=2000, p=4, h=0.5):
    """Table 2 on GB300: the marginal cost per GLS problem of the paper's four
    algorithms (binary64), each timed at two numbers of SNPs so that its
    one-time setup (Cholesky, inverse) drops out, and its ratio to Alg. 5
    beside the table's asymptotic ratio.  b_i of every algorithm is compared
    with Alg. 5's on the SNPs both solved."""
    import numpy as np
    from paper_1210_7325_gb300 import gls, synth
    sizes = {"black_box": (2, 6), "seq_gls": (64, 320), "hp_gwas": (16384, 65536),
             "gwfgls": (4096, 16384)}
    table2 = {"black_box": n, "seq_gls": p, "hp_gwas": 1, "gwfgls": 2}
    mmax = max(m2 for _, m2 in sizes.values())
    seed = synth.BASE_SEED + 5
    dev = torch.device("cuda")
    M = torch.from_numpy(synth.kinship_M(n, h, seed)).to(dev).t()  # symmetric: column-major view
    XL = torch.from_numpy(np.ascontiguousarray(synth.covariates(n, p, seed).T)).to(dev).t()
    y = torch.from_numpy(synth.phenotype(n, seed)).to(dev)
    XR = synth.genotypes_torch(n, mmax, seed, device=dev)          # (m, n)
    B = torch.empty((mmax, p), dtype=torch.float64, device=dev)
    st = torch.empty(mmax, dtype=torch.int32, device=dev)
    rows, ref = {}, None
    with gls.Plan(n, p, 16384, precision="fp64") as plan:
        plan.solve_variant("hp_gwas", M, XL, y, XR[:256].t(), B[:256].t(), st[:256], k=256)
        for alg in ("hp_gwas", "black_box", "seq_gls", "gwfgls"):
            times = []
            for m in sizes[alg]:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                plan.solve_variant(alg, M, XL, y, XR[:m].t(), B[:m].t(), st[:m], k=m)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            (m1, m2), (t1, t2) = sizes[alg], times
            per = (t2 - t1) / (m2 - m1)
            got = B[:sizes["black_box"][1]].cpu().numpy().T.copy()
            if alg == "hp_gwas":
                ref = got
            diff = float(np.max(np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)))
            rows[alg] = {"m": [m1, m2], "seconds": [round(t1, 4), round(t2, 4)],
                         "per_problem_us": per * 1e6,
                         "setup_ms": max(t1 - m1 * per, 0.0) * 1e3,
                         "max_rel_diff_vs_hp_gwas": diff}
    for alg, r in rows.items():
        r["ratio_vs_hp_gwas"] = r["per_problem_us"] / rows["hp_gwas"]["per_problem_us"]
        r["table2_ratio"] = table2[alg]
    return {"workload": f"variants_n{n}_p{p}", "n": n, "p": p, "precision": "fp64",
            "algorithms": rows,
            "note": "per_problem_us = marginal cost (two sizes); Table 2 gives the asymptotic "
                    "ratios n, p, 1, 2 for Alg. 3, 4, 5, 6"}


FILE_WORKLOADS = {
    # the motivating scan's size (n = 1500, p = 4, binary64) at the paper's out-of-core scale
    "file_n1500_p4_m10000000_fp64": dict(n=1500, p=4, m=10_000_000, h=0.5, precision="fp64",
                                         block=65536, seed_offset=1),
}


def run_file_workload(args, fw, torch):
    """Disk tier of Alg. 8: the genotypes (int8, or 2-bit with --packed) are
    written to a file, then gls_factor + gls_solve_file stream them back through
    the pinned ring, timed end to end.  The same plan's rate on the same
    genotypes held in HBM (gls_solve_stream on device memory) is the reference
    the file rate is compared with.  Reads after the write may be served by the
    page cache; the line reports the read rate the ring sustained."""
    import tempfile

    import numpy as np
    from paper_1210_7325_gb300 import gls, synth
    n, p, m, prec, kmax = fw["n"], fw["p"], fw["m"], fw["precision"], fw["block"]
    seed = synth.BASE_SEED + fw["seed_offset"]
    width = gls.packed_rows(n) if args.packed else n
    d = args.file_dir or tempfile.gettempdir()
    path = os.path.join(d, f"gls_genotypes_n{n}_m{m}_{'2bit' if args.packed else 'int8'}.bin")
    dev = torch.device("cuda")
    XRd = synth.genotypes_torch(n, m, seed, device="cuda")             # (m, n) int8 in HBM
    t0 = time.perf_counter()
    with open(path, "wb") as f:
        for s0 in range(0, m, 1 << 20):
            blk = XRd[s0:s0 + (1 << 20)]
            if args.packed:
                blk = gls.pack_genotypes(blk.t()).t()
            f.write(blk.contiguous().cpu().numpy().tobytes())
    t_write = time.perf_counter() - t0
    M = synth.kinship_M(n, fw["h"], seed)
    XL = np.asfortranarray(synth.covariates(n, p, seed))
    y = synth.phenotype(n, seed)
    Bh = torch.empty((m, p), dtype=torch.float64, pin_memory=True)
    sh = torch.empty(m, dtype=torch.int32, pin_memory=True)
    plan = gls.Plan(n, p, kmax, precision=prec, flags=launch_flags(args, gls))
    Mf = np.asfortranarray(M)
    # in HBM: the same stream on device-resident genotypes (one warm pass)
    plan.factor(Mf, XL, y)
    plan.solve_stream(XRd.t(), Bh.t(), sh, m=min(m, 4 * kmax))
    t0 = time.perf_counter()
    plan.factor(Mf, XL, y)
    plan.solve_stream(XRd.t(), Bh.t(), sh, m=m)
    t_hbm = time.perf_counter() - t0
    B_hbm = Bh[:: max(1, m // 4096)].clone()
    del XRd
    torch.cuda.empty_cache()
    plan.set_timing(True)
    t0 = time.perf_counter()
    plan.factor(Mf, XL, y)
    plan.solve_file(path, m, Bh.t(), sh, packed=args.packed)
    t_file = time.perf_counter() - t0
    st = plan.stats()
    plan.close()
    same = bool(torch.equal(Bh[:: max(1, m // 4096)], B_hbm))
    try:
        os.unlink(path)
    except OSError:
        pass
    return {"metric": METRIC, "value": m / t_file, "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": t_file * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16": "bf16", "fp16": "f16", "fp64": "f64"}[prec],
            "data": "synthetic genotypes written to a file, then streamed back",
            "config": {"workload": args.workload, "n": n, "p": p, "m": m, "block_snps": kmax,
                       "file_format": "2-bit packed" if args.packed else "int8",
                       "file_bytes": width * m, "file_dir": d, "parallelism": "replicas1"},
            "in_hbm": {"value": m / t_hbm, "unit": UNIT, "seconds": t_hbm},
            "file_vs_in_hbm": t_hbm / t_file,
            "write_s": t_write, "read_gbps_overall": width * m / t_file / 1e9,
            "file_results_equal_in_hbm_results": same,
            "phase_ms": {"factor": st["factor_ms"], "solve_kernels": st["trsm_ms"] + st["solve_ms"],
                         "h2d": st["h2d_ms"]},
            "e2e": {"value": m / t_file, "unit": UNIT,
                    "h2d_bytes_per_step": width * m + n * n * 8 + n * p * 8,
                    "d2h_bytes_per_step": m * (p * 8 + 4)}}


def sub_batch(args, torch, name="batch48_uneven_bf16", steps=2, warmup=1):
    """The batched uneven-scan workload as a sub-object of the default line."""
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup, sub.workload = steps, warmup, name
    try:
        ln = run_batch_workload(sub, BATCH_WORKLOADS[name], torch)
    except Exception as ex:  # reported, not fatal to the headline line
        return {"workload": name, "error_raised": repr(ex)}
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "roofline",
            "phase_ms_per_step", "error", "gpu_launches", "check")
    out = {"workload": name}
    out.update({k: ln[k] for k in keep if k in ln})
    out["config"] = {k: ln["config"][k] for k in ("scans", "total_snps", "rounds",
                                                  "group_autotuned", "split_terms_autotuned",
                                                  "operand_precision", "setup_s")
                     if k in ln["config"]}
    return out


def sub_serve(args, torch, name="serve2000_bf16", time_cap=180.0):
    """The serving workload as a sub-object of the default line (time-capped)."""
    try:
        ln = run_serve_workload(argparse.Namespace(workload=name, requests=0, time_cap=0,
                                                   serve_trace=args.serve_trace),
                                SERVE_WORKLOADS[name], torch, time_cap=time_cap)
    except Exception as ex:  # reported, not fatal to the headline line
        return {"workload": name, "error_raised": repr(ex)}
    keep = ("value", "unit", "latency", "completed", "reused_factors", "error",
            "queue_depth_max", "queue_depth_last", "wall_s", "dtype")
    out = {"workload": name}
    out.update({k: ln[k] for k in keep if k in ln})
    out["config"] = {k: ln["config"][k] for k in ("requests", "rate_per_s", "time_cap_s",
                                                  "bank_build_s", "hbm_budget_bytes")}
    out["loop_breakdown"] = {k: round(v, 3) if isinstance(v, float) else v
                             for k, v in ln["loop_breakdown"].items()}
    return out


def launch_flags(args, gls):
    return gls.GLS_FLAG_EAGER if getattr(args, "eager", False) else 0


def config_for(wl, args):
    return {"workload": args.workload, "n": wl["n"], "p": wl["p"], "m": wl["m"], "h": wl["h"],
            "precision": wl["precision"], "block_snps": wl["block"],
            "l2": "inputs larger than L2 (int8 genotypes n*m bytes)",
            "launch": "eager" if args.eager else "CUDA-graph replay of repeated sequences",
            "parallelism": f"replicas{args.gpus}"}


# ----------------------------------------------------------------------------- ranks
def max_over_ranks(t_local, e2e_local, dist, torch, device):
    """The slowest rank's timed-region and end-to-end times (replicas run in
    parallel, so the job takes as long as its slowest replica)."""
    if not dist:
        return t_local, e2e_local
    tt = torch.tensor([t_local, e2e_local or 0.0], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt[0]), (float(tt[1]) or None)


def whole_job_rate(world, m, steps, t):
    """Solves/s of the whole job: every rank solves its own m SNPs per step."""
    return world * m * steps / t


# ----------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload",
                    choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) + sorted(SERVE_WORKLOADS)
                    + sorted(FILE_WORKLOADS),
                    default=DEFAULT_WORKLOAD)
    ap.add_argument("--file-dir", default=None,
                    help="file workloads: directory of the genotype file (default: the temp dir)")
    ap.add_argument("--packed", action="store_true",
                    help="file workloads: write and read 2-bit packed genotypes")
    ap.add_argument("--requests", type=int, default=0, help="serving: number of requests")
    ap.add_argument("--time-cap", type=float, default=0.0, help="serving: wall-time cap (s)")
    ap.add_argument("--factor-only", action="store_true",
                    help="time gls_factor alone on the workload's M (setup phase, Alg. 5 lines 1-6)")
    ap.add_argument("--factor-native", action="store_true",
                    help="with --factor-only on a mixed workload: the binary64 CUDA-core factor")
    ap.add_argument("--eager", action="store_true",
                    help="launch every kernel directly (no CUDA-graph replay of repeated sequences)")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-sub", action="store_true",
                    help="default workload: skip the batched-scan and serving legs")
    ap.add_argument("--serve-trace", default=None,
                    help="serving: append one line per admission, round and eviction to this file")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--cpu-snps", type=int, default=2048)
    ap.add_argument("--ref-snps", type=int, default=1024)
    args = ap.parse_args()
    if args.workload in SERVE_WORKLOADS:
        import torch
        from paper_1210_7325_gb300 import build as gbuild
        gbuild.build()
        print(json.dumps(run_serve_workload(args, SERVE_WORKLOADS[args.workload], torch)),
              flush=True)
        return
    if args.workload in FILE_WORKLOADS:
        import torch
        from paper_1210_7325_gb300 import build as gbuild
        gbuild.build()
        print(json.dumps(run_file_workload(args, FILE_WORKLOADS[args.workload], torch)),
              flush=True)
        return
    if args.workload in BATCH_WORKLOADS:
        import torch
        from paper_1210_7325_gb300 import build as gbuild
        gbuild.build()
        print(json.dumps(run_batch_workload(args, BATCH_WORKLOADS[args.workload], torch)),
              flush=True)
        return
    wl = WORKLOADS[args.workload]
    args.warmup = max(args.warmup, 3) if args.impl == "gb300" else args.warmup
    if args.factor_only:
        import torch
        from paper_1210_7325_gb300 import build as gbuild
        gbuild.build()
        print(json.dumps(run_factor_only(args, wl, torch)), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist

    from paper_1210_7325_gb300 import build as gbuild
    if rank == 0:
        gbuild.build()
    if dist:
        dist.barrier()

    res = run_gpu(args, wl, rank, world, torch, dist)
    t_max, e2e_max = max_over_ranks(res["time"], res.get("e2e_time"), dist, torch, "cuda")
    e8_max, _ = max_over_ranks(res.get("e2e_int8_time") or 0.0, None, dist, torch, "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks, peak_src = load_peaks()
    n, p, m = wl["n"], wl["p"], wl["m"]
    K = args.steps
    value = whole_job_rate(world, m, K, t_max)
    s = res["stats"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": t_max / K * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if wl["precision"] == "bf16" else ("f16" if wl["precision"] == "fp16"
                                                          else "f64"),
        "data": "synthetic (seeded kinship, covariates, phenotype, Binomial(2,f) genotypes)",
        "config": config_for(wl, args),
        "gpu_launches": int(s["launches"]),
        "clocks": res["clocks"],
        "steady_state": {"value": m * K / (t_max - s["factor_ms"] / 1e3),
                         "unit": UNIT, "note": "the step without its factor (the SNP loop)"},
        "phase_ms_per_step": {"factor": s["factor_ms"] / K, "trsm_gram": s["trsm_ms"] / K,
                              "convert": s["convert_ms"] / K, "solve_pxp": s["solve_ms"] / K},
        "check": {"bad_status": res["bad_status"], "nan": res["nan"]},
    }
    # roofline of the dominant kernel (the blocked solve + Gram epilogue)
    trsm_avg_s = s["trsm_ms"] / 1e3 / max(s["trsm_launches"], 1)
    snps_per_launch = m * K / max(s["trsm_launches"], 1)
    if wl["precision"] == "fp64":
        dgemm = fp64_dgemm_tflops(torch)
        flops = n * n * snps_per_launch
        achieved = flops / trsm_avg_s / 1e12
        line["roofline"] = {"bound": "fp64", "achieved": achieved, "peak": dgemm,
                            "unit": "TFLOP/s", "frac": achieved / dgemm, "traffic": None,
                            "peak_source": "measured torch.matmul float64 8192^3 in this run",
                            "flops_per_launch": flops}
    else:
        S = res.get("split") or 3
        line["config"]["split_terms_autotuned"] = S
        line["config"]["split_trial"] = res.get("split_info")
        flops = S * n * n * snps_per_launch
        achieved = flops / trsm_avg_s / 1e12
        peak = peaks["bf16_tflops_sustained"]
        line["roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak,
                            "unit": "TFLOP/s", "frac": achieved / peak,
                            "traffic": TRSM_TRAFFIC.get((wl["precision"], n, wl["block"])),
                            "peak_source": f"{peak_src} bf16_tflops_sustained",
                            "flops_per_launch": flops,
                            "per_unit": f"{S} slices x n^2 tensor flops per SNP"}
    if e2e_max:
        line["e2e"] = {"value": whole_job_rate(world, m, K, e2e_max), "unit": UNIT,
                       "h2d_bytes_per_step": res["e2e_h2d"], "d2h_bytes_per_step": res["e2e_d2h"],
                       "h2d_gbps_measured": res.get("h2d_gbps"),
                       "h2d_gbps_per_block": res.get("h2d_gbps_blocks"),
                       "d2h_gbps_measured": res.get("d2h_gbps"),
                       "genotype_input": "2-bit packed (gls_solve_stream_packed)",
                       "step_ms": res.get("e2e_step_ms"),
                       "diagnostic_step": res.get("e2e_diag")}
        if e8_max:
            line["e2e_int8"] = {"value": whole_job_rate(world, m, K, e8_max), "unit": UNIT,
                                "h2d_bytes_per_step": res["e2e_int8_h2d"],
                                "d2h_bytes_per_step": res["e2e_d2h"],
                                "genotype_input": "int8 (gls_solve_stream), pinned blocks "
                                                  "read in place, block j+1 converted on 8 "
                                                  "SMs beside block j's solve",
                                "step_ms": res.get("e2e_int8_step_ms"),
                                "diagnostic_step": res.get("e2e_int8_diag"),
                                "staged_copy_engine": res.get("e2e_int8_staged")}
    if not args.skip_fp64 and wl["precision"] != "fp64":
        try:
            line["fp64"] = fp64_sample(wl, torch)
            line["fp64"]["dgemm_tflops_measured"] = fp64_dgemm_tflops(torch)
        except Exception as ex:  # reported, not fatal
            line["fp64"] = {"error": repr(ex)}
    if not args.skip_cpu and world == 1:
        import oracle
        smp = res["sample"]
        r = oracle_sample(wl, oracle.default_threads(), smp["M"], smp["XL"], smp["y"], smp["XR"])
        line["cpu_baseline"] = {
            "value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
            "sample": (f"oracle Cholesky of M (n={n}, {r['factor_s']:.1f} s) + per-SNP loop on "
                       f"{r['s_snps']} of the timed run's SNP columns ({r['snp_s']:.1f} s), "
                       f"projected to m={m}"),
            "steady_state": r["steady"]}
        line["error"] = error_summary(smp["B"], smp["st"], r["B"], r["st"],
                                      1e-10 if wl["precision"] == "fp64" else 1e-6)
    del res
    if world == 1 and not args.skip_sub and args.workload == DEFAULT_WORKLOAD:
        # each leg reports its own failure; the headline line is printed regardless
        for key, leg in (("batch", lambda: sub_batch(args, torch)),
                         ("serve", lambda: sub_serve(args, torch)),
                         ("phenotypes", lambda: sub_phenotypes(args, torch)),
                         ("variants", lambda: run_variants(torch))):
            try:
                torch.cuda.empty_cache()
                line[key] = leg()
            except Exception as ex:
                line[key] = {"error_raised": repr(ex)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

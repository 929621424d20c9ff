"""Continuous-batching server for GLS scan requests.

Each request is one GWAS scan (its own n, p, m, M, X_L, y, X_R).  The server
  * admits waiting requests in arrival order while the device bytes of the
    plans it holds plus the new request's inputs stay within an HBM budget,
    evicting idle cached factors (least recently used) to make room;
  * keeps each factor of M (L, L^{-1}, its operand slices and X~_L) resident
    after its request finishes, so a later request with the same M and
    covariates and a new phenotype only re-whitens y (gls_factor with M = NULL);
  * factors newly admitted requests on worker threads (each plan has its own
    stream) while the main loop keeps the GPU busy with solves;
  * admits waiting requests that share one M (and X_L, X_R) together, up to
    the plans' phenotype capacity: their phenotypes join one factor call
    (gls_factor_y) and every solve pass over X_R serves all of them;
  * solves in rounds: every round runs ONE batched launch (gls_batch_solve)
    over the next block of every active request (mixed precision), or one
    block per active request on their own streams (FP64), so requests that
    arrive while others are running join the next round.
Latency of a request = completion time - arrival time.

Ordering and lifetime of request inputs.  ``make_inputs`` enqueues whatever
device work makes a request's tensors on the calling thread's current stream.
The server records an event on that stream right after it returns and makes
the request's plan wait for the event (gls_plan_wait_event) before the factor
and every solve read the tensors on the plan's stream; a batched round runs
after the work queued on each of its plans' streams, so it is ordered too.
The tensors stay referenced until the request's last synchronous round has
returned and its factor has ended; run() waits for every outstanding factor
before it returns, even when it stops at its time cap.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import gls

MAX_BATCH = 64


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float           # seconds after the start of the run
    n: int
    p: int
    m: int
    mkey: int                # identifies (M, X_L, X_R); equal keys share a factor
    y_seed: int
    h: float = 0.5
    reuse: bool = False


@dataclasses.dataclass
class Inputs:
    M: object                # device tensors (column-major views)
    XL: object
    XR: object               # (m, n) int8, i.e. the column-major n x m matrix
    y: object


class _Slot:
    """A resident factor (plan) and the request currently using it."""

    def __init__(self, plan, key, n, p, nbytes):
        self.plan = plan
        self.key = key
        self.n, self.p = n, p
        self.nbytes = nbytes
        self.busy = False
        self.last_used = 0.0


class _Active:
    """Requests being served on one plan: the leader and the requests that
    share its M and joined as further phenotypes (b_ij of phenotype j in
    row i t + j of B)."""

    def __init__(self, reqs, slot, inputs, B, st, t_admit):
        self.reqs = reqs
        self.req = reqs[0]
        self.slot = slot
        self.inputs = inputs
        self.B = B
        self.st = st
        self.next = 0
        self.t_admit = t_admit
        self.factored: Optional[cf.Future] = None


class Server:
    def __init__(self, make_inputs, precision="bf16", hbm_budget=150e9, block=32768,
                 factor_workers=4, group=0, device="cuda", streams=None, keep=None,
                 phenotypes=4, trace=None):
        """make_inputs(req, torch, reuse) -> Inputs (device tensors for the request,
        made by work on the current stream; with reuse=True the factor of M is
        cached, so M and X_L may be None).  ``streams`` supplies
        current_stream() and Event() (torch.cuda by default on a GPU device,
        none on the CPU); ``keep`` is a set of request ids whose outputs run()
        keeps (every request's with keep_outputs=True); ``trace`` a file that
        gets one flushed line per admission, round, eviction and batch."""
        import torch
        self.torch = torch
        self.device = device
        if streams is None and str(device).startswith("cuda"):
            streams = torch.cuda
        self.streams = streams
        self.keep = set(keep or ())
        self.make_inputs = make_inputs
        self.precision = precision
        self.budget = float(hbm_budget)
        self.block = int(block)
        self.group = int(group)
        self.phenotypes = max(1, int(phenotypes))  # phenotype capacity of every plan
        self._trace = open(trace, "a", buffering=1) if trace else None
        self._t0 = time.perf_counter()
        self.slots: Dict[int, _Slot] = {}
        self.used = 0.0
        self.pool = cf.ThreadPoolExecutor(max_workers=factor_workers)
        self.batches: "collections.OrderedDict[tuple, gls.Batch]" = collections.OrderedDict()
        self.results: Dict[int, dict] = {}
        self.queue_depth: List[tuple] = []
        self.rejected: List[tuple] = []   # (rid, reason): larger than the whole budget
        self.peak_used = 0.0
        self._lock = threading.Lock()
        # wall-time breakdown of the serving loop (seconds) and factor wall time
        self.breakdown = {"admit_s": 0.0, "rounds_s": 0.0, "idle_s": 0.0, "rounds": 0,
                          "round_requests": 0, "factor_s": 0.0, "factors": 0,
                          "plan_create_s": 0.0, "evict_s": 0.0, "inputs_s": 0.0}

    def _log(self, *fields):
        if self._trace:
            self._trace.write(f"{time.perf_counter() - self._t0:.4f} " +
                              " ".join(str(f) for f in fields) + "\n")

    # ------------------------------------------------------------ memory
    def _plan_bytes(self, n, p):
        return gls.footprint_bytes(n, p, self.block, self.precision,
                                   phenotypes=min(self.phenotypes, 33 - p))

    def _input_bytes(self, req):
        return req.n * req.m + req.m * req.p * 8 + req.m * 4 + req.n * req.n * 8

    def _evict(self, need):
        idle = sorted((s for s in self.slots.values() if not s.busy), key=lambda s: s.last_used)
        for s in idle:
            if self.used + need <= self.budget:
                break
            t = time.perf_counter()
            self._log("evict", s.key, id(s.plan), s.n, s.p)
            self._drop_batches_with(s.plan)
            s.plan.close()
            self.breakdown["evict_s"] += time.perf_counter() - t
            self.used -= s.nbytes
            del self.slots[s.key]

    def _drop_batches_with(self, plan):
        for key in [k for k in self.batches if id(plan) in k]:
            self._log("batch_close", key)
            self.batches.pop(key).close()

    # ------------------------------------------------------------ admission
    def _try_admit(self, req, now, companions=()):
        """Admits req and, as further phenotypes of the same factor, the waiting
        requests in `companions` (same mkey) that fit the plan's capacity."""
        slot = self.slots.get(req.mkey)
        if slot is not None and slot.busy:
            return None  # the resident factor is serving another phenotype
        reqs = [req] + list(companions)[:min(self.phenotypes, 33 - req.p) - 1]
        in_bytes = sum(self._input_bytes(r) for r in reqs)
        need = in_bytes + (0 if slot is not None else self._plan_bytes(req.n, req.p))
        if need > self.budget:
            raise MemoryError(f"request {req.rid} needs {need:.3g} B, above the HBM budget")
        if self.used + need > self.budget:
            if slot is not None:
                slot.busy = True  # the factor this request reuses is not evicted
            self._evict(need)
            if slot is not None:
                slot.busy = False
            if self.used + need > self.budget:
                return None
        reuse = slot is not None
        t = time.perf_counter()
        inputs = self.make_inputs(req, self.torch, reuse)
        if len(reqs) > 1:  # the companions' phenotypes: Y = [y_1 ... y_g], column-major
            ys = [inputs.y] + [self.make_inputs(r, self.torch, True).y for r in reqs[1:]]
            inputs.y = self.torch.stack(ys, dim=0).t()
        ready = self._inputs_ready()
        self.breakdown["inputs_s"] += time.perf_counter() - t
        if not reuse:
            t = time.perf_counter()
            plan = gls.Plan(req.n, req.p, self.block, precision=self.precision,
                            phenotypes=min(self.phenotypes, 33 - req.p))
            self.breakdown["plan_create_s"] += time.perf_counter() - t
            slot = _Slot(plan, req.mkey, req.n, req.p, self._plan_bytes(req.n, req.p))
            self.slots[req.mkey] = slot
            self.used += slot.nbytes
        slot.busy = True
        self.used += in_bytes
        self.peak_used = max(self.peak_used, self.used)
        torch = self.torch
        B = torch.empty((req.m * len(reqs), req.p), dtype=torch.float64, device=self.device)
        st = torch.empty(req.m, dtype=torch.int32, device=self.device)
        act = _Active(reqs, slot, inputs, B, st, now)
        if len(reqs) > 1:
            self.breakdown["grouped"] = self.breakdown.get("grouped", 0) + len(reqs) - 1
        self._log("admit", [r.rid for r in reqs], req.mkey, id(slot.plan), req.n, req.p, req.m,
                  "reuse" if reuse else "new")
        if ready is not None:
            # the plan's stream reads the inputs only after their producer wrote them
            slot.plan.wait_event(ready)
        if reuse:
            act.factored = self.pool.submit(self._timed_factor, slot.plan, None, None, inputs.y)
        else:
            act.factored = self.pool.submit(self._timed_factor, slot.plan, inputs.M, inputs.XL,
                                            inputs.y)
        return act

    def _inputs_ready(self):
        """An event on the current stream after make_inputs' work (None on the CPU)."""
        if self.streams is None:
            return None
        ev = self.streams.Event()
        ev.record(self.streams.current_stream())
        return ev

    def _timed_factor(self, plan, M, XL, y):
        t = time.perf_counter()
        plan.factor(M, XL, y)
        with self._lock:
            self.breakdown["factor_s"] += time.perf_counter() - t
            self.breakdown["factors"] += 1

    # ------------------------------------------------------------ solving
    def _batch_for(self, acts):
        key = tuple(id(a.slot.plan) for a in acts)
        b = self.batches.get(key)
        if b is None:
            b = gls.Batch([a.slot.plan for a in acts])
            self._log("batch_new", key)
            self.batches[key] = b
            while len(self.batches) > 32:
                old_key, old = self.batches.popitem(last=False)
                self._log("batch_close", old_key)
                old.close()
        else:
            self.batches.move_to_end(key)
        return b

    def _round(self, ready):
        parts = []
        for a in ready:
            s0 = a.next
            k = min(self.block, a.req.m - s0)
            parts.append((a, s0, k))
        # logged before the launch, so that a trace cut short by a failure names it
        self._log("round", [(a.req.rid, id(a.slot.plan), s0, k, len(a.reqs)) for a, s0, k in parts])
        if self.precision == "fp64":
            for a, s0, k in parts:
                g = len(a.reqs)
                a.slot.plan.solve_block(a.inputs.XR[s0:s0 + k].t(),
                                        a.B[s0 * g:(s0 + k) * g].t(), a.st[s0:s0 + k], k=k)
            for a, s0, k in parts:
                a.slot.plan.synchronize()
        else:
            acts = [a for a, _, _ in parts]
            batch = self._batch_for(acts)
            batch.solve([a.inputs.XR[s0:s0 + k].t() for a, s0, k in parts],
                        [a.B[s0 * len(a.reqs):(s0 + k) * len(a.reqs)].t() for a, s0, k in parts],
                        [a.st[s0:s0 + k] for a, s0, k in parts],
                        [k for _, _, k in parts], group=self.group)
        for a, s0, k in parts:
            a.next = s0 + k

    def _finish(self, a, now):
        a.slot.busy = False
        a.slot.last_used = now
        g = len(a.reqs)
        Bg = a.B.view(a.req.m, g, a.req.p)
        for j, r in enumerate(a.reqs):
            self.used -= self._input_bytes(r)
            self.results[r.rid] = dict(
                rid=r.rid, arrival=r.arrival, admitted=a.t_admit, done=now,
                latency=now - r.arrival, n=r.n, p=r.p, m=r.m, reuse=r.reuse,
                B=Bg[:, j, :] if g > 1 else a.B, status=a.st, phenotypes_in_call=g)

    # ------------------------------------------------------------ main loop
    def run(self, requests: List[Request], time_cap: float = float("inf"), keep_outputs=False):
        """Serves the requests in real time (arrivals are offsets from now)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: collections.deque = collections.deque()
        active: List[_Active] = []
        try:
            self._serve(pending, waiting, active, time_cap, keep_outputs)
        finally:
            # a factor still running (time cap, or another request's error)
            # reads its request's inputs: they stay referenced until it ends
            cf.wait([a.factored for a in active if a.factored is not None])
        return self.results

    def _serve(self, pending, waiting, active, time_cap, keep_outputs):
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            if now > time_cap:
                break
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # admission in arrival order; a blocked request does not block others
            still = collections.deque()
            t_adm = time.perf_counter()
            while waiting:
                req = waiting.popleft()
                if len(active) >= MAX_BATCH:
                    still.append(req)
                    continue
                same = [r for r in waiting if r.mkey == req.mkey]
                try:
                    act = self._try_admit(req, time.perf_counter() - t0, same)
                except MemoryError as e:
                    self.rejected.append((req.rid, str(e)))
                    continue
                if act is None:
                    still.append(req)
                else:
                    active.append(act)
                    for r in act.reqs[1:]:
                        waiting.remove(r)
            waiting = still
            self.breakdown["admit_s"] += time.perf_counter() - t_adm
            self.queue_depth.append((now, len(waiting), len(active)))
            ready = [a for a in active if a.factored.done()]
            for a in ready:
                a.factored.result()  # re-raises a factor error
            ready = [a for a in ready if a.next < a.req.m]
            if ready:
                t_r = time.perf_counter()
                self._round(ready[:MAX_BATCH])
                self.breakdown["rounds_s"] += time.perf_counter() - t_r
                self.breakdown["rounds"] += 1
                self.breakdown["round_requests"] += min(len(ready), MAX_BATCH)
            else:
                # nothing to solve yet: wait for a factor or the next arrival
                nxt = pending[0].arrival if pending else now + 0.01
                t_i = time.perf_counter()
                time.sleep(max(0.0, min(0.002, nxt - now)))
                self.breakdown["idle_s"] += time.perf_counter() - t_i
            done_now = time.perf_counter() - t0
            for a in [a for a in active if a.factored.done() and a.next >= a.req.m]:
                self._finish(a, done_now)
                active.remove(a)
                for r in a.reqs:
                    if not keep_outputs and r.rid not in self.keep:
                        self.results[r.rid].pop("B")
                        self.results[r.rid].pop("status")

    def close(self):
        # a run cut off by its time cap can leave factors running on the
        # workers: they finish before any plan is destroyed
        self.pool.shutdown(wait=True)
        if self._trace:
            self._trace.close()
            self._trace = None
        for b in self.batches.values():
            b.close()
        self.batches.clear()
        for s in self.slots.values():
            s.plan.close()
        self.slots.clear()


def poisson_requests(count, rate, seed, n_range, p_range, m_range, reuse_frac=0.3, h=0.5):
    """Seeded Poisson stream; a reusing request repeats an earlier request's
    (n, p, m, M, X_L, X_R) with a new phenotype."""
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 77])))
    t = 0.0
    reqs: List[Request] = []
    for i in range(count):
        t += g.exponential(1.0 / rate)
        if reqs and g.uniform() < reuse_frac:
            src = reqs[int(g.integers(0, len(reqs)))]
            reqs.append(Request(i, t, src.n, src.p, src.m, src.mkey, seed * 100003 + i, src.h,
                                True))
        else:
            n = int(g.integers(n_range[0], n_range[1] + 1))
            p = int(g.integers(p_range[0], p_range[1] + 1))
            m = int(g.integers(m_range[0], m_range[1] + 1))
            reqs.append(Request(i, t, n, p, m, i, seed * 100003 + i, h, False))
    return reqs


def latency_summary(results):
    lat = np.array([r["latency"] for r in results.values()])
    if lat.size == 0:
        return {"completed": 0}
    done = max(r["done"] for r in results.values())
    first = min(r["arrival"] for r in results.values())
    snps = sum(r["m"] for r in results.values())
    return {"completed": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "max_s": float(lat.max()),
            "solves_per_s": snps / max(done - first, 1e-9),
            "reused": int(sum(r["reuse"] for r in results.values()))}

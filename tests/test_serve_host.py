"""Host logic of the serving loop (admission by memory budget, LRU eviction of
idle factors, reuse of a resident factor for a new phenotype, continuous
batching), run on the CPU against a fake of the GLS binding that records
every call.  The GPU behaviour is covered by tests/test_gpu_serve.py."""
import threading
import time

import numpy as np
import pytest
import torch

from paper_1210_7325_gb300 import serve


class FakeStreams:
    """current_stream() / Event() of a fake device.  Work is not run, only
    logged: make_inputs tags each tensor with the stream it was made on and the
    position of that work in the log, and an event remembers where it was
    recorded."""

    def __init__(self):
        self.lock = threading.Lock()
        self.log = []
        self.current = "s0"

    def current_stream(self):
        return self.current

    def produce(self, *tensors):
        with self.lock:
            self.log.append(("produce", self.current))
            pos = len(self.log)
        for t in tensors:
            if t is not None:
                t.made_on, t.made_at = self.current, pos

    def Event(self):
        streams = self

        class Event:
            stream = at = None

            def record(self, stream):
                with streams.lock:
                    streams.log.append(("record", stream))
                    self.stream, self.at = stream, len(streams.log)
        return Event()


class FakeGls:
    def __init__(self):
        self.lock = threading.Lock()
        self.factors = []      # (plan id, with_M)
        self.batches = []      # number of plans per batched launch
        self.closed_use = 0
        self.inflight = 0      # factors running now
        self.groups = []       # phenotypes per factor call
        self.factor_s = 0.002
        self.unordered = []    # reads of inputs the plan was not ordered after

    def footprint_bytes(self, n, p, block, precision, phenotypes=1):
        return 8 * n * n + 1000

    def make(self):
        fake = self

        class Plan:
            ids = iter(range(10**6))

            def __init__(self, n, p, block, precision="fp64", phenotypes=1):
                self.n, self.p, self.block, self.precision = n, p, block, precision
                self.capacity = phenotypes
                self.id = next(Plan.ids)
                self.closed = False
                self.yv = None
                self.waited = None

            def wait_event(self, ev):
                self.waited = ev

            def check_ordered(self, *tensors):
                # every input was made before an event that this plan waited
                # for, on the stream that made it
                for t in tensors:
                    if t is None or not hasattr(t, "made_on"):
                        continue
                    ev = self.waited
                    if ev is None or ev.stream != t.made_on or ev.at <= t.made_at:
                        fake.unordered.append((self.id, getattr(t, "made_on", None)))

            def factor(self, M, XL, y):
                with fake.lock:
                    fake.inflight += 1
                self.check_ordered(M, XL, y)
                time.sleep(fake.factor_s)
                with fake.lock:
                    fake.inflight -= 1
                    if self.closed:
                        fake.closed_use += 1
                        raise RuntimeError("factor on a closed plan")
                    fake.factors.append((self.id, M is not None))
                    fake.groups.append(1 if y.dim() == 1 else y.shape[1])
                assert (1 if y.dim() == 1 else y.shape[1]) <= self.capacity
                self.yv = y.sum(dim=0).reshape(-1)  # one sum per phenotype

            def _fill(self, XR, B, st):
                # b_ij := (sum of the SNP column + sum of phenotype j) in every row of
                # column i t + j: a function of the request's own data only
                t = self.yv.numel()
                v = XR.t().double().sum(dim=1)[:, None] + self.yv[None, :]   # (k, t)
                B.t()[:] = v.reshape(-1)[:, None]
                st[:] = 0

            def solve_block(self, XR, B, st, k=None):
                if self.closed:
                    fake.closed_use += 1
                self.check_ordered(XR._base if XR._base is not None else XR)
                self._fill(XR, B, st)

            def synchronize(self):
                pass

            def close(self):
                self.closed = True

        class Batch:
            def __init__(self, plans):
                self.plans = plans

            def solve(self, XRs, Bs, sts, ks, group=0):
                fake.batches.append(len(self.plans))
                for pl, X, B, s in zip(self.plans, XRs, Bs, sts):
                    if pl.closed:
                        fake.closed_use += 1
                    pl.check_ordered(X._base if X._base is not None else X)
                    pl._fill(X, B, s)

            def close(self):
                pass

        self.Plan, self.Batch = Plan, Batch
        return self


def make_inputs(req, torch_mod, reuse):
    g = torch.Generator().manual_seed(req.mkey)
    XR = torch.randint(0, 3, (req.m, req.n), generator=g, dtype=torch.int8)
    y = torch.full((req.n,), float(req.y_seed % 97), dtype=torch.float64)
    M = None if reuse else torch.eye(req.n, dtype=torch.float64)
    XL = None if reuse else torch.ones((req.n, max(req.p - 1, 0)), dtype=torch.float64)
    return serve.Inputs(M, XL, XR, y)


def expected(req):
    g = torch.Generator().manual_seed(req.mkey)
    XR = torch.randint(0, 3, (req.m, req.n), generator=g, dtype=torch.int8)
    return XR.double().sum(dim=1) + float(req.y_seed % 97) * req.n


@pytest.fixture
def fake(monkeypatch):
    f = FakeGls().make()
    monkeypatch.setattr(serve, "gls", f)
    return f


@pytest.mark.parametrize("prec", ["bf16", "fp64"])
@pytest.mark.parametrize("budget", [1e9, 2.2e6])
def test_every_request_served_once_within_budget(fake, prec, budget):
    reqs = serve.poisson_requests(40, 400.0, 5, (100, 300), (2, 5), (50, 700), 0.4)
    srv = serve.Server(make_inputs, prec, hbm_budget=budget, block=128, device="cpu")
    res = srv.run(reqs, time_cap=60.0, keep_outputs=True)
    srv.close()
    assert not srv.rejected
    assert sorted(res) == [r.rid for r in reqs]
    assert srv.peak_used <= budget
    assert fake.closed_use == 0
    for r in reqs:
        B = res[r.rid]["B"]
        assert torch.equal(B[:, 0], expected(r)), r.rid
        assert torch.equal(B[:, -1], expected(r))
    # every phenotype is in exactly one factor call; a resident factor serves
    # new phenotypes with M = None
    assert sum(fake.groups) == len(reqs)
    distinct = len({r.mkey for r in reqs})
    with_m = sum(1 for _, m in fake.factors if m)
    if budget >= 1e9:
        assert with_m == distinct                 # nothing evicted: one factor per M
    else:
        assert with_m > distinct                  # evictions forced re-factoring
    if prec != "fp64":
        assert max(fake.batches) > 1               # requests shared launches


def test_request_larger_than_budget_is_rejected(fake):
    reqs = [serve.Request(0, 0.0, 2000, 3, 100, 0, 1), serve.Request(1, 0.0, 100, 3, 100, 1, 2)]
    srv = serve.Server(make_inputs, "bf16", hbm_budget=1e6, block=128, device="cpu")
    res = srv.run(reqs, time_cap=30.0)
    srv.close()
    assert [rid for rid, _ in srv.rejected] == [0]
    assert list(res) == [1]


def test_latency_summary():
    res = {i: dict(latency=float(i), done=float(i) + 1, arrival=0.0, m=10, reuse=i % 2 == 0)
           for i in range(1, 101)}
    s = serve.latency_summary(res)
    assert s["completed"] == 100 and s["reused"] == 50
    assert s["p50_s"] == pytest.approx(50.5) and s["p99_s"] == pytest.approx(99.01)
    assert s["solves_per_s"] == pytest.approx(1000 / 101)


def tagged_inputs(streams):
    """make_inputs that logs its work on the current fake stream."""
    def make(req, torch_mod, reuse):
        inp = make_inputs(req, torch_mod, reuse)
        streams.produce(inp.M, inp.XL, inp.y, inp.XR)
        return inp
    return make


@pytest.mark.parametrize("prec", ["bf16", "fp64"])
def test_inputs_ordered_before_the_plan_reads_them(fake, prec):
    """The invariant whose absence let a plan's stream read request inputs made
    on another stream: after make_inputs the server records an event on the
    stream that made them, and the plan waits for it before its factor and
    every solve read them (checked for reused factors too)."""
    streams = FakeStreams()
    streams.current = "side"   # inputs made on a stream other than the default
    reqs = serve.poisson_requests(30, 400.0, 9, (100, 300), (2, 5), (50, 700), 0.4)
    assert any(r.reuse for r in reqs)
    srv = serve.Server(tagged_inputs(streams), prec, hbm_budget=1e9, block=128,
                       device="cpu", streams=streams)
    res = srv.run(reqs, time_cap=60.0)
    srv.close()
    assert sorted(res) == [r.rid for r in reqs]
    assert fake.unordered == []
    # and a server that forgets the event is caught by the same check
    fake.unordered.clear()
    bad = serve.Server(tagged_inputs(streams), prec, hbm_budget=1e9, block=128, device="cpu",
                       streams=None)
    bad.run(reqs[:3], time_cap=60.0)
    bad.close()
    assert fake.unordered


def test_time_cap_waits_for_running_factors(fake):
    """run() stopped by its time cap returns only after every factor it started
    has ended, so no factor reads inputs that were already released."""
    fake.factor_s = 0.3
    reqs = serve.poisson_requests(6, 1000.0, 3, (100, 200), (2, 4), (50, 100), 0.0)
    srv = serve.Server(make_inputs, "bf16", hbm_budget=1e9, block=128, device="cpu",
                       factor_workers=6)
    t0 = time.perf_counter()
    srv.run(reqs, time_cap=0.02)
    assert fake.inflight == 0
    assert time.perf_counter() - t0 >= 0.25
    srv.close()


def test_kept_outputs(fake):
    reqs = serve.poisson_requests(8, 400.0, 4, (100, 200), (2, 4), (50, 300), 0.0)
    srv = serve.Server(make_inputs, "bf16", hbm_budget=1e9, block=128, device="cpu",
                       keep={0, 3})
    res = srv.run(reqs, time_cap=60.0)
    srv.close()
    assert "B" in res[0] and "B" in res[3] and "B" not in res[1]
    assert torch.equal(res[3]["B"][:, 0], expected(reqs[3]))


@pytest.mark.parametrize("prec", ["bf16", "fp64"])
def test_requests_sharing_an_m_join_one_factor(fake, prec):
    """A burst of requests on one M (new phenotypes) waiting together is
    served by factor calls with several phenotypes, up to the capacity, and
    every request still gets its own b."""
    base = serve.Request(0, 0.0, 150, 3, 200, 7, 100)
    reqs = [base] + [serve.Request(i, 0.0, 150, 3, 200, 7, 100 + i, reuse=True)
                     for i in range(1, 7)]
    reqs += [serve.Request(7, 0.0, 120, 2, 100, 8, 300)]
    srv = serve.Server(make_inputs, prec, hbm_budget=1e9, block=64, device="cpu", phenotypes=4)
    res = srv.run(reqs, time_cap=60.0, keep_outputs=True)
    srv.close()
    assert sorted(res) == list(range(8))
    assert max(fake.groups) == 4 and sum(fake.groups) == 8
    assert srv.breakdown["grouped"] >= 3
    for r in reqs:
        B = res[r.rid]["B"]
        assert torch.equal(B[:, 0], expected(r)), r.rid
        assert torch.equal(B[:, -1], expected(r))

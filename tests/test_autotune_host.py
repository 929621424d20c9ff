"""Host logic of the autotuner on the CPU: the error gate of the split factor
(against a fake of the GLS binding whose 2- and 3-slice results differ by a
chosen amount), the block-size rule and the group cache."""
import numpy as np
import pytest
import torch

from paper_1210_7325_gb300 import autotune


class FakePlan:
    """Stands in for gls.Plan: solve_block writes B = base * (1 + rel[S]) and
    the status vector given for S."""
    rel = {3: 0.0, 2: 0.0}
    status = {3: None, 2: None}
    made = []

    def __init__(self, n, p, k, precision="bf16", device=0, split_terms=0):
        self.p, self.S = p, split_terms
        FakePlan.made.append(split_terms)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def factor(self, M, XL, y):
        pass

    def solve_block(self, XR, Bt, st, k=None):
        base = torch.arange(1, k * self.p + 1, dtype=torch.float64).reshape(k, self.p)
        Bt.t().copy_(base * (1.0 + FakePlan.rel[self.S]))
        s = FakePlan.status[self.S]
        st.copy_(torch.zeros(k, dtype=torch.int32) if s is None else torch.as_tensor(s))

    def synchronize(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    from paper_1210_7325_gb300 import gls
    monkeypatch.setattr(gls, "Plan", FakePlan)
    FakePlan.rel = {3: 0.0, 2: 0.0}
    FakePlan.status = {3: None, 2: None}
    FakePlan.made = []
    return FakePlan


def run(k=16):
    XR = torch.zeros((100, k), dtype=torch.int8)
    return autotune.tune_split(100, 4, "bf16", None, None, None, XR, tol=1e-6, margin=8.0)


def test_two_slices_within_margin(fake):
    fake.rel[2] = 1e-7          # below tol / 8 = 1.25e-7
    S, info = run()
    assert S == 2 and info["err_2_vs_3"] == pytest.approx(1e-7, rel=1e-6)
    assert sorted(fake.made) == [2, 3]


def test_two_slices_beyond_margin(fake):
    fake.rel[2] = 2e-7          # within tol, but not within tol / 8
    S, info = run()
    assert S == 3 and info["threshold"] == pytest.approx(1.25e-7)


def test_status_disagreement_keeps_three(fake):
    fake.status[2] = np.array([0] * 15 + [1], dtype=np.int32)
    S, info = run()
    assert S == 3 and not info["status_agree"]


def test_all_degenerate_sample_keeps_three(fake):
    fake.status[2] = np.ones(16, dtype=np.int32)
    fake.status[3] = np.ones(16, dtype=np.int32)
    S, info = run()
    assert S == 3 and info["err_2_vs_3"] == float("inf")


@pytest.mark.parametrize("m,kmax,expect", [
    (10, 100, 10), (100, 100, 100), (101, 100, 51), (250, 100, 84), (0, 100, 1),
])
def test_choose_block(m, kmax, expect):
    kb = autotune.choose_block(m, kmax)
    assert kb == expect
    if m > kmax:
        rounds = -(-m // kb)
        assert kb <= kmax and rounds == -(-m // kmax)


def test_group_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("GLS_GB300_CACHE", str(tmp_path))
    assert autotune._load() == {}
    autotune._store({"k": {"group": 3, "times": {"3": 0.1}}})
    assert autotune._load()["k"]["group"] == 3
    assert autotune.cache_path().startswith(str(tmp_path))

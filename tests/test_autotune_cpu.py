"""Host logic of the batch autotuner (solver.autotune_batch) with the GPU
timing replaced by a fake batch whose step time depends on the configured
pipeline depth: the fastest depth wins, is cached under the workload's
signature and reused without timing, and depths the library refuses are
skipped."""
import json

import pytest

from paper_2609_23057_b300 import _lib, solver


class _FakeSolver:
    def __init__(self, n):
        self.n = n
        self.precision = "bf16"


class _FakeBatch:
    """Stands in for solver.Batch: configure() may refuse a depth; each step
    'takes' the time of the current depth."""

    def __init__(self, ms_per_stage, refuse=(), ns=(8, 16, 32)):
        self.solvers = [_FakeSolver(n) for n in ns]
        self.site_direction_updates_per_step = 187203584
        self.ms_per_stage = ms_per_stage
        self.refuse = set(refuse)
        self.stages = None
        self.steps = 0
        self.configured = []

    def configure(self, st):
        if st in self.refuse:
            raise _lib.RtlbError(4, "stages must be 2, 4, 6 or 8 and fit in shared memory")
        self.stages = st
        self.configured.append(st)

    def step(self, k):
        self.steps += k
        _Clock.now += k * self.ms_per_stage[self.stages]


class _Clock:
    now = 0.0


class _FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self):
        self.t = _Clock.now

    def elapsed_time(self, other):
        return other.t - self.t


@pytest.fixture
def fake_cuda(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)


def test_picks_fastest_and_caches(tmp_path, fake_cuda):
    path = str(tmp_path / "tune.json")
    b = _FakeBatch({2: 3.0, 4: 1.0, 6: 1.5, 8: 2.0})
    assert solver.autotune_batch(b, cache_path=path) == 4
    assert b.stages == 4 and b.steps > 0
    with open(path) as f:
        cache = json.load(f)
    (key, val), = cache.items()
    sig = json.loads(key)
    assert sig == {"device": "FakeGPU", "precision": "bf16", "n": [8, 16, 32], "channels": 3,
                   "sdu_per_step_log2": 27}
    assert val["stages"] == 4 and val["ms_per_step"] == pytest.approx(1.0)

    # same signature: the cached depth is applied without timing anything
    b2 = _FakeBatch({2: 0.1, 4: 9.0, 6: 9.0, 8: 9.0})
    assert solver.autotune_batch(b2, cache_path=path) == 4
    assert b2.steps == 0 and b2.configured == [4]

    # another signature (different direction counts) is tuned afresh
    b3 = _FakeBatch({2: 0.5, 4: 1.0, 6: 1.5, 8: 2.0}, ns=(8, 8))
    assert solver.autotune_batch(b3, cache_path=path) == 2
    with open(path) as f:
        assert len(json.load(f)) == 2


def test_refused_depths_are_skipped(tmp_path, fake_cuda):
    path = str(tmp_path / "tune.json")
    b = _FakeBatch({2: 3.0, 4: 2.0, 6: 1.0, 8: 0.5}, refuse=(8,))
    assert solver.autotune_batch(b, cache_path=path) == 6
    assert 8 not in b.configured[:-1] and b.stages == 6


def test_unreadable_cache_is_ignored(tmp_path, fake_cuda):
    path = tmp_path / "tune.json"
    path.write_text("not json")
    b = _FakeBatch({2: 1.0, 4: 2.0, 6: 3.0, 8: 4.0})
    assert solver.autotune_batch(b, cache_path=str(path)) == 2
    assert json.loads(path.read_text())

"""Host logic of the batch autotuner (solver.autotune_batch) with the GPU
timing replaced by a fake batch whose step time depends on the configured
pipeline depth and work-balance tile cost: the fastest pair wins, is cached
under the workload's signature and reused without timing, and settings the
library refuses are skipped."""
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

    def __init__(self, ms_per_stage, refuse=(), ns=(8, 16, 32), cost_factor=None, refuse_cost=()):
        self.solvers = [_FakeSolver(n) for n in ns]
        self.site_direction_updates_per_step = 187203584
        self.ms_per_stage = ms_per_stage
        self.cost_factor = cost_factor or {}
        self.refuse = set(refuse)
        self.refuse_cost = set(refuse_cost)
        self.stages = None
        self.tile_cost = 4
        self.steps = 0
        self.configured = []
        self.balanced = []

    def configure(self, st):
        if st in self.refuse:
            raise _lib.RtlbError(4, "stages must be 2, 4, 6 or 8 and fit in shared memory")
        self.stages = st
        self.configured.append(st)

    def balance(self, cost):
        if cost in self.refuse_cost:
            raise _lib.RtlbError(4, "tile_cost must be in [0, 64]")
        self.tile_cost = cost
        self.balanced.append(cost)

    def step(self, k):
        self.steps += k
        _Clock.now += k * self.ms_per_stage[self.stages] * self.cost_factor.get(self.tile_cost, 1.0)


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
    assert val["stages"] == 4 and val["tile_cost"] == 4 and val["ms_per_step"] == pytest.approx(1.0)

    # same signature: the cached depth is applied without timing anything
    b2 = _FakeBatch({2: 0.1, 4: 9.0, 6: 9.0, 8: 9.0})
    assert solver.autotune_batch(b2, cache_path=path) == 4
    assert b2.steps == 0 and b2.configured == [4] and b2.balanced == [4]

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


def test_tile_cost_dimension(tmp_path, fake_cuda):
    """The depth and the work-balance cost are searched together: the best
    pair (6 stages, cost 16) is applied and cached; refused costs are
    skipped."""
    path = str(tmp_path / "tune.json")
    b = _FakeBatch({2: 2.0, 4: 1.2, 6: 1.0, 8: 1.1}, cost_factor={0: 1.3, 4: 1.0, 8: 0.9, 16: 0.8},
                   refuse_cost=(8,))
    assert solver.autotune_batch(b, cache_path=path) == 6
    assert b.stages == 6 and b.tile_cost == 16
    assert 8 not in b.balanced
    (val,) = json.loads(open(path).read()).values()
    assert val == {"stages": 6, "tile_cost": 16, "ms_per_step": pytest.approx(0.8)}
    # a cached entry from before the cost was tuned applies the default cost
    key = next(iter(json.loads(open(path).read())))
    with open(path, "w") as f:
        json.dump({key: {"stages": 2, "ms_per_step": 1.0}}, f)
    b2 = _FakeBatch({2: 1.0, 4: 1.0, 6: 1.0, 8: 1.0})
    b2.tile_cost = 99
    assert solver.autotune_batch(b2, cache_path=path) == 2
    assert b2.balanced == [4] and b2.steps == 0

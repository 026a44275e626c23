"""Host-side helpers of bench.py (no GPU): sampled per-kernel profiling and
the replica seeds."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeProfiler:
    """Records the profiling switch at every step, like the library's hooks."""

    def __init__(self):
        self.on = False
        self.seen = []
        self.collected = 0
        self.resets = 0

    def profile_enable(self, on=True):
        self.on = bool(on)

    def profile_collect(self):
        self.collected += 1

    def profile_reset(self):
        self.resets += 1


def test_profiled_samples_every_nth_step():
    f = FakeProfiler()
    for i in range(40):
        bench.profiled(f, i, lambda: f.seen.append(f.on))
    assert f.seen == [i % bench.PROFILE_EVERY == 0 for i in range(40)]
    assert not f.on


def test_profiled_switches_off_after_an_exception():
    f = FakeProfiler()

    def boom():
        raise RuntimeError("x")
    try:
        bench.profiled(f, 0, boom)
    except RuntimeError:
        pass
    assert not f.on


def test_prewarm_profiles_enough_steps(monkeypatch):
    f = FakeProfiler()
    monkeypatch.setattr(bench.torch.cuda, "synchronize", lambda *a, **k: None)
    steps = []
    bench.profiler_prewarm(f, lambda: steps.append(f.on), 2000)
    # every sampled step of the timed region has its events made beforehand
    assert len(steps) >= 2000 // bench.PROFILE_EVERY and all(steps)
    assert f.collected == 1 and f.resets == 1 and not f.on


def test_replica_seeds_are_distinct():
    seeds = {bench.replica_seed(2, r) for r in range(8)}
    assert len(seeds) == 8 and bench.replica_seed(2, 0) == 2

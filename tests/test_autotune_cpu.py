"""Host logic of the batch autotuner: candidates in order (item sizes, then pack counts at the
best size, then the unfused schedule), more packs than simulations skipped, the fastest kept
and cached per bucket, a cached bucket reused without timing.  The timing of a candidate is
replaced by a table, so no GPU is needed."""
import types

import pytest


class FakeBatch:
    def __init__(self, n, capacity=10**6):
        self.sims = [types.SimpleNamespace(gs=types.SimpleNamespace(particle_capacity=capacity))
                     for _ in range(n)]
        self.cur = None
        self.calls = []

    def set_tuning(self, particles_per_item, packs):
        self.cur = (particles_per_item, packs)
        self.calls.append(self.cur)


@pytest.fixture
def tuner(tmp_path, monkeypatch):
    from paper_1912_04674_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    return autotune


def test_fastest_schedule_is_picked_and_cached(tuner, monkeypatch):
    cost = {(2048, 0): 5.0, (4096, 0): 4.0, (8192, 0): 4.5, (16384, 0): 6.0,
            (4096, 2): 3.9, (4096, 4): 3.8, (4096, -1): 3.5}
    monkeypatch.setattr(tuner, "_time_batch", lambda b, steps: cost[b.cur])
    b = FakeBatch(6)
    assert tuner.tune_batch(b, "fp32") == (4096, -1)
    assert b.cur == (4096, -1)
    assert b.calls[:4] == [(2048, 0), (4096, 0), (8192, 0), (16384, 0)]
    assert (4096, 8) not in b.calls and (4096, 16) not in b.calls   # more packs than sims
    assert [c for c, p, m in b.tuning_log] == [c for c, p in b.calls[:-1]]
    assert tuner.batch_tuning_for(6 * 10**6, 6, "fp32") == (4096, -1)
    # the bucket is cached: a second batch of the same shape is set without timing
    monkeypatch.setattr(tuner, "_time_batch", lambda b, steps: pytest.fail("timed again"))
    b2 = FakeBatch(6)
    assert tuner.tune_batch(b2, "fp32") == (4096, -1) and b2.cur == (4096, -1)


def test_fused_schedule_kept_when_faster(tuner, monkeypatch):
    cost = {(2048, 0): 1.0, (4096, 0): 2.0, (8192, 0): 2.0, (16384, 0): 3.0,
            (2048, 2): 1.1, (2048, 4): 0.9, (2048, 8): 1.2, (2048, 16): 1.3, (2048, -1): 1.5}
    monkeypatch.setattr(tuner, "_time_batch", lambda b, steps: cost[b.cur])
    b = FakeBatch(64, capacity=10**5)
    assert tuner.tune_batch(b, "fp32") == (2048, 4)
    assert tuner.batch_tuning_for(64 * 10**5, 64, "fp32") == (2048, 4)
    assert tuner.batch_tuning_for(64 * 10**5, 64, "fp64") == (tuner.TILE_DEFAULT, 0)   # untuned

"""The launch-shape autotuner's host logic on CPU (autotune.tune), with the CUDA events and the
library step faked by a cost model: it times every candidate of the space from the same
restored state, returns the fastest, clamps steps per launch to the steps asked for, and caches
the choice per (device, precision, field kinds, electron total to a power of two)."""
import contextlib
import types

import pytest

from paper_1612_07592_gb300 import autotune


class _FakeRun:
    def __init__(self, n, precision=1, geometry=0, polarisation=0):
        self.n = n
        self.params = types.SimpleNamespace(precision=precision, geometry=geometry, polarisation=polarisation)
        self.stream = object()
        self.handle = object()
        self.restores = 0
        self.state = "initial"

    def snapshot(self):
        return "initial"

    def restore(self, snap):
        self.restores += 1
        self.state = snap

    def rebind(self, tables):
        pass


@pytest.fixture
def fake_cuda(monkeypatch, tmp_path):
    import torch
    log = {"calls": [], "last_ms": 0.0}

    def cost(cfg):       # fastest at block 256, 8 CTAs per SM, the longest launch
        return 10.0 + abs(cfg["block"] - 256) / 64 + abs(cfg["ctas_per_sm"] - 8) + 100.0 / cfg["steps_per_launch"]

    def step_ex(handles, steps, **cfg):
        log["calls"].append(dict(cfg, steps=steps))
        log["last_ms"] = cost(cfg)

    class Event:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream=None):
            pass

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return log["last_ms"]

    monkeypatch.setattr(autotune, "pe_step_ex", step_ex)
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "Event", Event)
    return log


def test_tune_times_every_candidate_and_picks_the_fastest(fake_cuda):
    runs = [_FakeRun(1000), _FakeRun(3000)]
    space = dict(block=(128, 256), ctas_per_sm=(4, 8, 15), steps_per_launch=(256, 1024, 2048))
    best, results = autotune.tune(0, runs, 1500, space=space, use_cache=False, repeats=2)
    assert len(results) == 2 * 3 * 3
    assert best == dict(block=256, ctas_per_sm=8, steps_per_launch=1500)      # 2048 clamped to the 1500 steps
    assert min(ms for _, ms in results) == pytest.approx(10.0 + 100.0 / 1500)
    # every timing (repeats + a warm-up, per candidate) restarts the runs from the same state, and
    # the runs are left at it afterwards
    assert all(r.restores == 18 * 3 + 1 for r in runs)
    assert len(fake_cuda["calls"]) == 18 * 3 and all(c["steps"] == 1500 for c in fake_cuda["calls"])


def test_tune_caches_the_choice_per_key(fake_cuda):
    runs = [_FakeRun(5000)]
    space = dict(block=(128, 256), ctas_per_sm=(8,), steps_per_launch=(512,))
    first, res1 = autotune.tune(0, runs, 512, space=space)
    n_calls = len(fake_cuda["calls"])
    again, res2 = autotune.tune(0, runs, 512, space=space)
    assert again == first and res2 == [] and len(fake_cuda["calls"]) == n_calls      # served from the cache
    autotune.tune(0, [_FakeRun(5000, precision=0)], 512, space=space)              # another precision: tuned
    assert len(fake_cuda["calls"]) > n_calls


def test_key_buckets_electrons_and_separates_kinds():
    a = autotune._key("G", [_FakeRun(5000)])
    assert a == autotune._key("G", [_FakeRun(4096)]) == autotune._key("G", [_FakeRun(8191)])
    assert a != autotune._key("G", [_FakeRun(8192)])
    assert a != autotune._key("G", [_FakeRun(5000, geometry=1)])
    assert a != autotune._key("G", [_FakeRun(5000, polarisation=1)])
    assert a != autotune._key("H", [_FakeRun(5000)])

"""The continuous-batching server's host logic on CPU (serve.Server), with the library calls
replaced by fakes that count steps: admission by free slot and by device memory, mid-run
admission with each run's own launch boundaries, iterations of min(K, fewest steps left),
resident runs capped at one batched launch, retirement freeing every run.  The GPU tests check the
same server against the library (results alone equal results in the mix)."""
import pytest

import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import serve


class _Fakes:
    def __init__(self):
        self.runs = {}
        self.calls = []

    def run(self, tables, params, n, capacity=0, stream=None, events=False):
        fake = self

        class FakeRun:
            def __init__(self):
                self.n = n
                self.handle = object()
                self.done = 0
                self.closed = False
                fake.runs[self.handle] = self

            def tally_out(self):
                return ("steps", self.done)

            def state(self):
                return None

            def event_words(self):
                return None

            def close(self):
                self.closed = True

        return FakeRun()

    def step_ex(self, handles, steps, **cfg):
        self.calls.append((len(handles), steps, dict(cfg)))
        for h in handles:
            self.runs[h].done += steps


@pytest.fixture
def fakes(monkeypatch):
    f = _Fakes()
    monkeypatch.setattr(serve, "Run", f.run)
    monkeypatch.setattr(serve, "pe_step_ex", f.step_ex)
    monkeypatch.setattr(serve, "run_params", lambda **kw: kw)
    import torch
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    return f


def _server(K=500, slots=64, free=1 << 40, server_box=None):
    box = server_box if server_box is not None else {}

    def mem():
        s = box.get("server")
        used = s.resident_bytes if s is not None else 0
        return free - used, free

    s = serve.Server(tables=0, steps_per_iteration=K, max_slots=slots, memory_reserve_bytes=0, mem_get_info=mem,
                     stream=object())
    box["server"] = s
    return s


def _req(t, n, steps):
    return serve.Request(arrival_s=t, n=n, steps=steps, run={}, capacity=1 << 12)


def test_every_run_finishes_its_own_steps(fakes):
    reqs = [_req(0.0, 1000 * (k + 1), 300 + 250 * k) for k in range(5)]
    stats = _server(K=400).run_trace(reqs, virtual_step_s=1e-3)
    assert stats.latencies_s and len(stats.latencies_s) == 5
    for r in reqs:
        assert r.tally == ("steps", r.steps) and r.boundaries[-1] == r.steps
        # every iteration advances by at most K and ends when the first resident run is done
        assert all(0 < b - a <= 400 for a, b in zip([0] + r.boundaries[:-1], r.boundaries))
    assert stats.particle_steps == sum(r.n * r.steps for r in reqs)
    assert all(run.closed for run in fakes.runs.values())


def test_slots_bound_the_resident_runs(fakes):
    reqs = [_req(0.0, 100, 500) for _ in range(7)]
    stats = _server(K=500, slots=3).run_trace(reqs, virtual_step_s=1e-3)
    assert stats.max_resident == 3 and stats.iterations == 3
    assert max(c[0] for c in fakes.calls) == 3


def test_device_memory_bounds_the_resident_runs(fakes):
    reqs = [_req(0.0, 10000, 500) for _ in range(6)]
    need = serve.Server.bytes_needed(reqs[0])
    box = {}
    s = _server(K=500, free=2 * need + need // 2, server_box=box)
    stats = s.run_trace(reqs, virtual_step_s=1e-3)
    assert stats.max_resident == 2 and s.resident_bytes == 0
    assert len(stats.latencies_s) == 6


def test_a_request_is_admitted_while_others_run(fakes):
    """A request arriving mid-run joins at the next iteration: its launch boundaries fall at steps of
    its own that differ from the first run's, and it is retired when its steps are done."""
    first, second = _req(0.0, 1000, 1000), _req(0.25, 500, 300)
    stats = _server(K=200).run_trace([first, second], virtual_step_s=1e-3)
    # arrives during the second iteration (0.2 s each), joins after step 400 of the first run; the
    # iteration that follows is min(K, 600, 300) = 200 steps, the next ends the second run (100)
    assert second.admitted_iteration == 2 and second.resident_at_admission == 1
    assert first.boundaries == [200, 400, 600, 700, 900, 1000]
    assert second.boundaries == [200, 300]
    assert stats.max_resident == 2 and stats.iterations == 6


def test_resident_runs_capped_at_the_batch_limit(fakes):
    """More slots than one batched launch takes are clamped to it: never more than MAX_BATCH runs
    resident, so every launch holds at most MAX_BATCH runs."""
    n = pe.MAX_BATCH + 6
    reqs = [_req(0.0, 10, 100) for _ in range(n)]
    stats = _server(K=100, slots=4 * pe.MAX_BATCH).run_trace(reqs, virtual_step_s=1e-3)
    assert stats.max_resident == pe.MAX_BATCH
    assert max(c[0] for c in fakes.calls) == pe.MAX_BATCH and len(stats.latencies_s) == n


def test_requests_from_workload_scale_and_capacity():
    cfg = {"requests": [{"arrival_s": 0.1 * k, "n": 1000 * (k + 1), "steps": 100, "run": {"a0": 1.0}}
                        for k in range(4)]}
    rs = serve.requests_from_workload(cfg, limit=3, n_scale=0.5)
    assert [r.n for r in rs] == [500, 1000, 1500]
    assert all(r.capacity == max(1 << 12, min(4 * r.n, 1 << 24)) for r in rs)
    assert [r.arrival_s for r in rs] == [0.0, 0.1, 0.2]

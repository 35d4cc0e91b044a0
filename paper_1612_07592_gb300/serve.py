"""Continuous-batching request loop for emission runs.

Requests (one laser-target run each: parameters, electron count, step count)
arrive over time.  The server admits a waiting request as soon as a slot
(at most 64 runs per batched launch) and device memory for its buffers are
free, keeps every admitted run's state resident, and advances all resident runs
together in batched persistent launches (runs of different field kinds go to one
launch per kind).  An iteration advances every resident run by
min(K, the fewest steps any resident run still has to do), so a run is retired
the moment its steps are done: its tallies are read, its buffers freed, its
latency (arrival to results on the host) recorded, and its slot and memory go
to the next waiting request.  Runs admitted at different times therefore share
launches with changing company and see their launch boundaries at different
steps of their own.

Because positions and optical depths are kept as exact float pairs across
launch boundaries, a run's results do not depend on which other runs share its
launches or where its launch boundaries fall: a request gives the same result
alone and in the mix.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import MAX_BATCH, PE_F32, Run, pe_step_ex, run_params

STATE_BYTES_F32 = 8 + 8 + 3 * 4 + 8          # x pair, y pair, u, tau pair
STATE_BYTES_F64 = 8 + 8 + 3 * 8 + 8


@dataclass
class Request:
    arrival_s: float
    n: int
    steps: int
    run: dict
    capacity: int = 1 << 18
    precision: int = PE_F32
    # filled by the server
    admitted_s: float = -1.0
    done_s: float = -1.0
    tally: object = None
    state: np.ndarray | None = None
    events: np.ndarray | None = None
    admitted_iteration: int = -1       # server iteration at which the run was admitted
    resident_at_admission: int = 0     # runs already resident (mid-run) when it was admitted
    boundaries: list = field(default_factory=list)   # own step counts at the end of each launch set


@dataclass
class ServerStats:
    latencies_s: list = field(default_factory=list)
    queue_s: list = field(default_factory=list)
    particle_steps: float = 0.0
    makespan_s: float = 0.0
    iterations: int = 0
    max_resident: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies_s) if self.latencies_s else np.zeros(1)
        q = np.array(self.queue_s) if self.queue_s else np.zeros(1)
        return {"requests": len(self.latencies_s), "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "mean_queue_s": float(q.mean()),
                "particle_steps": self.particle_steps, "makespan_s": self.makespan_s,
                "particle_steps_per_s": self.particle_steps / max(self.makespan_s, 1e-12),
                "iterations": self.iterations, "max_resident": self.max_resident}


class Server:
    """Admit, batch and retire emission runs on one GPU."""

    def __init__(self, tables: int, steps_per_iteration: int = 500, max_slots: int = MAX_BATCH,
                 memory_reserve_bytes: int = 4 << 30, launch: dict | None = None, keep_results: bool = False,
                 mem_get_info=None, stream=None):
        import torch
        self.torch = torch
        self.tables = tables
        self.K = int(steps_per_iteration)
        self.max_slots = min(int(max_slots), MAX_BATCH)
        self.reserve = int(memory_reserve_bytes)
        self.launch = dict(launch or {})
        self.keep = keep_results
        self.mem_get_info = mem_get_info or torch.cuda.mem_get_info
        self.stream = stream or torch.cuda.Stream()
        self.resident_bytes = 0          # buffers of the admitted runs

    @staticmethod
    def bytes_needed(req: Request) -> int:
        per = STATE_BYTES_F32 if req.precision == PE_F32 else STATE_BYTES_F64
        return req.n * per + req.capacity * 32 + 16 * 1024

    def _admit(self, req: Request, now: float):
        run = Run(self.tables, run_params(precision=req.precision, **req.run), req.n, capacity=req.capacity,
                  stream=self.stream, events=self.keep)
        req.admitted_s = now
        return run

    def run_trace(self, requests: list[Request], realtime: bool = True,
                  virtual_step_s: float | None = None) -> ServerStats:
        """Serve the requests (sorted by arrival).

        realtime=True: arrivals follow the wall clock (the server sleeps while idle).
        realtime=False: idle time is skipped (the next arrival is taken as due when nothing
        is resident).  virtual_step_s: the clock is simulated instead -- it advances by
        virtual_step_s per step of each iteration -- so admissions happen at reproducible
        iterations (tests); latencies are then in simulated seconds."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival_s)
        active = []                     # [request, run, remaining steps]
        stats = ServerStats()
        t0 = time.perf_counter()
        vclock = [0.0]
        if virtual_step_s is not None:
            clock = lambda: vclock[0]
        else:
            clock = lambda: time.perf_counter() - t0
        i = 0
        while i < len(pending) or active:
            now = clock()
            if not active and i < len(pending) and pending[i].arrival_s > now:
                if virtual_step_s is not None:
                    vclock[0] = pending[i].arrival_s
                elif realtime:
                    time.sleep(min(pending[i].arrival_s - now, 0.05))
                    continue
                else:
                    t0 -= pending[i].arrival_s - now          # skip idle time
                now = clock()
            # admission: arrived, a slot free, memory available
            while i < len(pending) and pending[i].arrival_s <= now and len(active) < self.max_slots:
                free, _ = self.mem_get_info()
                if self.bytes_needed(pending[i]) > free - self.reserve:
                    break
                req = pending[i]
                req.admitted_iteration = stats.iterations
                req.resident_at_admission = len(active)
                active.append([req, self._admit(req, now), req.steps])
                self.resident_bytes += self.bytes_needed(req)
                stats.queue_s.append(now - req.arrival_s)
                i += 1
            if not active:
                continue
            stats.max_resident = max(stats.max_resident, len(active))
            # one iteration: every resident run advances by the same chunk, ending when the
            # first of them is done
            chunk = min(self.K, min(a[2] for a in active))
            cfg = dict(self.launch)
            cfg.setdefault("steps_per_launch", self.K)
            for j in range(0, len(active), MAX_BATCH):
                part = active[j:j + MAX_BATCH]
                pe_step_ex([a[1].handle for a in part], chunk, **cfg)
                for a in part:
                    a[2] -= chunk
                    a[0].boundaries.append(a[0].steps - a[2])
                    stats.particle_steps += chunk * a[1].n
            stats.iterations += 1
            if virtual_step_s is not None:
                vclock[0] += chunk * virtual_step_s
            # retire finished runs (reading the tallies synchronises the stream)
            still = []
            for a in active:
                req, run, rem = a
                if rem > 0:
                    still.append(a)
                    continue
                req.tally = run.tally_out()
                req.done_s = clock()
                if self.keep:
                    req.state = run.state()
                    req.events = run.event_words()
                stats.latencies_s.append(req.done_s - req.arrival_s)
                self.resident_bytes -= self.bytes_needed(req)
                run.close()
                del run
            active = still
        torch.cuda.synchronize()
        stats.makespan_s = clock()
        return stats


def requests_from_workload(cfg: dict, limit: int | None = None, n_scale: float = 1.0) -> list[Request]:
    out = []
    for q in cfg["requests"][:limit]:
        n = max(1, int(q["n"] * n_scale))
        out.append(Request(arrival_s=q["arrival_s"], n=n, steps=q["steps"], run=dict(q["run"]),
                           capacity=max(1 << 12, min(4 * n, 1 << 24))))
    return out

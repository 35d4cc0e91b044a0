"""Autotuner of the persistent kernel's launch shape.

Sweeps threads per CTA, CTAs per SM and steps per launch on the caller's own runs
(each candidate restarts the same runs from the same state on fresh handles, so
every candidate does identical work), times each with CUDA events on the runs'
stream, and caches the fastest per (device, precision, field kinds, total
electrons rounded to a power of two) in a JSON file next to the library.
"""
from __future__ import annotations

import json
import os

from . import HERE, pe_step_ex

CACHE = os.path.join(HERE, "_autotune_cache.json")
DEFAULT_SPACE = dict(block=(128, 256), ctas_per_sm=(4, 8, 15), steps_per_launch=(256, 1024, 2048))


def _key(device_name: str, runs) -> str:
    prec = runs[0].params.precision
    kinds = sorted({(r.params.geometry, r.params.polarisation) for r in runs})
    ntot = sum(r.n for r in runs)
    bucket = 1 << max(0, int(ntot).bit_length() - 1)
    return f"{device_name}|p{prec}|{kinds}|n{bucket}"


def load_cache() -> dict:
    if os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def tune(tables: int, runs, steps: int, space: dict | None = None, use_cache: bool = True, repeats: int = 1):
    """Return (best config dict, list of (config, ms)) for advancing `runs` by `steps`."""
    import torch
    space = space or DEFAULT_SPACE
    dev = torch.cuda.get_device_name()
    key = _key(dev, runs)
    cache = load_cache()
    if use_cache and key in cache:
        return cache[key], []
    stream = runs[0].stream
    snaps = [r.snapshot() for r in runs]
    results = []
    for block in space["block"]:
        for cps in space["ctas_per_sm"]:
            for spl in space["steps_per_launch"]:
                cfg = dict(block=block, ctas_per_sm=cps, steps_per_launch=min(spl, steps))
                best = None
                for _ in range(repeats + 1):             # first repeat warms up
                    with torch.cuda.stream(stream):
                        for r, sn in zip(runs, snaps):
                            r.restore(sn)
                    for r in runs:
                        r.rebind(tables)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    pe_step_ex([r.handle for r in runs], steps, **cfg)
                    e1.record(stream)
                    e1.synchronize()
                    ms = e0.elapsed_time(e1)
                    best = ms if best is None else min(best, ms)
                results.append((cfg, best))
    with torch.cuda.stream(stream):
        for r, sn in zip(runs, snaps):
            r.restore(sn)
    for r in runs:
        r.rebind(tables)
    cfg = min(results, key=lambda kv: kv[1])[0]
    cache[key] = cfg
    try:
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return cfg, results

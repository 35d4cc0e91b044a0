"""Sharding of one run's electrons over ranks, and exact merging of their tallies.

Electrons are independent under prescribed fields, so a run shards by
contiguous electron-id ranges with no exchange while stepping (each id keeps
its own Philox stream).  The only exchange is at the end: histograms and
counters add as integers, and the 128-bit fixed-point energy tallies add with
their carries, so the merged result equals the unsharded run bit for bit.
"""
from __future__ import annotations

import numpy as np

from . import HIST_WORDS, T, TALLY_WORDS

FIXED_PAIRS = [T[k] for k in ("E_NCS_STORED", "E_NCS_BELOW", "E_BR_STORED", "E_BR_BELOW", "E_RECOIL_NCS",
                              "E_RECOIL_BR")]


def shard_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [lo, hi) electron ids of `rank` out of `world` (sizes differ by at most one)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def merge_tallies(tallies) -> np.ndarray:
    """Exact sum of tally vectors (uint64): counters mod 2^64, energy pairs as 128-bit."""
    out = np.zeros(TALLY_WORDS, dtype=np.uint64)
    pair_lo = set(FIXED_PAIRS)
    pair_hi = {k + 1 for k in FIXED_PAIRS}
    for t in tallies:
        t = np.asarray(t).astype(np.uint64)
        for k in range(TALLY_WORDS):
            if k in pair_lo or k in pair_hi:
                continue
            out[k] = np.uint64((int(out[k]) + int(t[k])) & 0xFFFFFFFFFFFFFFFF)
        for k in FIXED_PAIRS:
            v = (int(out[k + 1]) << 64) + int(out[k]) + (int(t[k + 1]) << 64) + int(t[k])
            v &= (1 << 128) - 1
            out[k] = np.uint64(v & 0xFFFFFFFFFFFFFFFF)
            out[k + 1] = np.uint64(v >> 64)
    return out


def merge_hists(hists) -> np.ndarray:
    out = np.zeros(HIST_WORDS, dtype=np.uint64)
    for h in hists:
        out += np.asarray(h).astype(np.uint64)
    return out


def allgather_merge(tally, hist, group=None):
    """All ranks receive the exact merged tally and histogram (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.from_numpy(np.asarray(tally).astype(np.uint64).view(np.int64).copy())
    h = torch.from_numpy(np.asarray(hist).astype(np.uint64).view(np.int64).copy())
    ts = [torch.zeros_like(t) for _ in range(world)]
    hs = [torch.zeros_like(h) for _ in range(world)]
    dist.all_gather(ts, t, group=group)
    dist.all_gather(hs, h, group=group)
    return (merge_tallies([x.numpy().view(np.uint64) for x in ts]),
            merge_hists([x.numpy().view(np.uint64) for x in hs]))

"""Multi-rank logic on the CPU (gloo, world size 2): a run sharded over ranks by
electron id, advanced by the FP64 oracle on each shard, merged exactly, equals
the unsharded run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1612_07592_gb300.shard import merge_hists, merge_tallies, shard_range


def test_shard_ranges_cover():
    for n in (0, 1, 7, 1000, 1_000_003):
        for w in (1, 2, 3, 8):
            rs = [shard_range(n, w, r) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(h - l for l, h in rs) - min(h - l for l, h in rs) <= 1


def test_merge_carries_128bit():
    a = np.zeros(32, np.uint64)
    b = np.zeros(32, np.uint64)
    a[16] = np.uint64(2 ** 64 - 1)
    b[16] = np.uint64(5)
    a[17] = np.uint64(3)
    m = merge_tallies([a, b])
    assert int(m[16]) == 4 and int(m[17]) == 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_1612_07592_gb300.shard import allgather_merge
    t = O.Tables(O.table_params(n_eta=24, n_y=24, n_E=24, n_s=24), [79.0])
    r = O.run_params(a0=270.0, Z=79.0, charge_state=51.0, init_dist=1, seed=3)
    lo, hi = shard_range(600, world, rank)
    ids = np.arange(lo, hi)
    st = O.init(t, r, ids)
    _, _, hist, tally = O.run(t, r, ids, st, 0, 800, threads=1)
    mt, mh = allgather_merge(tally, hist)
    out[rank] = (mt.tolist(), mh.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_equals_single_run():
    import oracle as O
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, out)) for k in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    t = O.Tables(O.table_params(n_eta=24, n_y=24, n_E=24, n_s=24), [79.0])
    r = O.run_params(a0=270.0, Z=79.0, charge_state=51.0, init_dist=1, seed=3)
    ids = np.arange(600)
    st = O.init(t, r, ids)
    _, _, hist, tally = O.run(t, r, ids, st, 0, 800, threads=1)
    for k in range(2):
        mt, mh = out[k]
        assert mt == [int(v) for v in tally]
        assert mh == [int(v) for v in hist]
    assert int(tally[0] + tally[1]) > 0

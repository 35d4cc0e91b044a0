"""One run split over contiguous electron-id ranges (pe_run_params.id0) through the library.

Under prescribed fields the electrons are independent (the paper's test mode, Sec. 2.2) and
every random number an electron draws is keyed on its global id, so a run of N electrons
equals the union of runs over id ranges [id0, id0 + n): the same particles, event words and
photons for each id, and tallies and histograms that add up exactly.  Checked in one process
(two ranges, three kernels) and with two processes on GPU 0 that each step their range and
merge the tallies over gloo.
"""
import os
import socket

import numpy as np
import pytest

import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import workloads as W
from paper_1612_07592_gb300.shard import merge_hists, merge_tallies, shard_range

pytestmark = pytest.mark.gpu

TP = dict(W.tables_small(), n_eta=48, n_y=48, n_E=48, n_s=48)
RUN = W.base_run(a0=270.0, init_dist=1, T_mev=1.0, seed=21, run_id=5, **W.AU)
N, STEPS = 3001, 900


def _photon_keys(ph):
    return np.sort(ph["id_mech"].astype(np.uint64) << np.uint64(32) | ph["step"].astype(np.uint64))


def _whole_and_parts(tables, precision, launch, world):
    whole = pe.Run(tables, pe.run_params(precision=precision, **RUN), N, capacity=1 << 18, events=True)
    pe.pe_step_ex([whole.handle], STEPS, **launch)
    parts = []
    for rank in range(world):
        lo, hi = shard_range(N, world, rank)
        r = pe.Run(tables, pe.run_params(precision=precision, **dict(RUN, id0=lo)), hi - lo, capacity=1 << 18,
                   events=True)
        pe.pe_step_ex([r.handle], STEPS, **launch)
        parts.append((lo, hi, r))
    return whole, parts


@pytest.mark.parametrize("precision,launch", [(pe.PE_F32, {}), (pe.PE_F32, dict(steps_per_launch=1)),
                                              (pe.PE_F64, {})])
def test_id_ranges_equal_whole_run(precision, launch):
    tables = pe.pe_create_tables(TP, (13.0, 79.0))
    whole, parts = _whole_and_parts(tables, precision, launch, 3)
    st, ev = whole.state(), whole.event_words()
    tw = whole.tally_out()
    tallies, hists, keys = [], [], []
    for lo, hi, r in parts:
        np.testing.assert_array_equal(r.state(), st[lo:hi])
        np.testing.assert_array_equal(r.event_words(), ev[lo:hi])
        t = r.tally_out()
        tallies.append(np.frombuffer(bytes(t.tally), dtype=np.uint64))
        hists.append(np.frombuffer(bytes(t.hist), dtype=np.uint64))
        keys.append(_photon_keys(r.photon_records()))
        r.close()
    assert tw.tally[pe.T["N_PHOTONS"]] > 0
    np.testing.assert_array_equal(merge_tallies(tallies), np.frombuffer(bytes(tw.tally), dtype=np.uint64))
    np.testing.assert_array_equal(merge_hists(hists), np.frombuffer(bytes(tw.hist), dtype=np.uint64))
    np.testing.assert_array_equal(np.sort(np.concatenate(keys)), _photon_keys(whole.photon_records()))
    whole.close()
    pe.pe_destroy_tables(tables)


def test_id0_range_is_checked():
    tables = pe.pe_create_tables(TP, (13.0, 79.0))
    with pytest.raises(pe.PeError) as e:
        pe.Run(tables, pe.run_params(precision=pe.PE_F32, **dict(RUN, id0=0xFFFFFFFF)), 2)
    assert e.value.status == pe.PE_ERR_ARG
    pe.pe_destroy_tables(tables)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1612_07592_gb300.shard import allgather_merge
    torch.cuda.set_device(0)
    tables = pe.pe_create_tables(TP, (13.0, 79.0))
    lo, hi = shard_range(N, world, rank)
    r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **dict(RUN, id0=lo)), hi - lo, capacity=1 << 18)
    pe.pe_step([r.handle], STEPS)
    t = r.tally_out()
    mt, mh = allgather_merge(np.frombuffer(bytes(t.tally), dtype=np.uint64),
                             np.frombuffer(bytes(t.hist), dtype=np.uint64))
    out[rank] = (lo, hi, r.state(), mt, mh)
    r.close()
    pe.pe_destroy_tables(tables)
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_merge_equals_whole_run():
    """Two processes on GPU 0 (their kernels are independent: nothing waits on the other rank)
    each advance their id range through the library; the exact gloo merge of their tallies and
    histograms equals the unsplit run's, and their particles are its slices."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, out)) for k in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
    assert all(p.exitcode == 0 for p in procs)
    tables = pe.pe_create_tables(TP, (13.0, 79.0))
    whole = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **RUN), N, capacity=1 << 18)
    pe.pe_step([whole.handle], STEPS)
    st = whole.state()
    tw = whole.tally_out()
    for k in range(2):
        lo, hi, s, mt, mh = out[k]
        np.testing.assert_array_equal(s, st[lo:hi])
        np.testing.assert_array_equal(mt, np.frombuffer(bytes(tw.tally), dtype=np.uint64))
        np.testing.assert_array_equal(mh, np.frombuffer(bytes(tw.hist), dtype=np.uint64))
    whole.close()
    pe.pe_destroy_tables(tables)

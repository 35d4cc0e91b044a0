"""pe_pic_step_noalloc: PIC steps for callers that cannot allocate device memory.

Such callers (a host framework or a fixed pool owns the device memory, or the
memory budget forbids allocations once a simulation is set up) step their PIC
state with this entry point, which sums the currents in a fixed array compiled
into the library instead of memory that pe_init_particles allocates.  The test
steps one PIC state with pe_step and an identical copy with the new entry point,
two calls each in a row, and requires the same particles, grid, tallies, histograms
and photons bit for bit.  It sets up everything itself, so it runs alone in a fresh process as
well as after the other tests.
"""
import numpy as np
import pytest

import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _params(precision, n_cells=600, **kw):
    run = W.base_run(**dict(W.AU, ne_over_nc=50.0, a0=270.0, geometry=pe.PE_PIC_1D, n_cells=n_cells,
                            init_dist=1, T_mev=1.0, seed=11, **kw))
    return pe.run_params(precision=precision, **run)


def _photons_sorted(run, count):
    ph = run.photon_records(count)
    return ph[np.lexsort((ph["step"], ph["id_mech"]))]


# LP with direct brems in both precisions; CP, and null-collision brems (its wait words are
# part of the state), in FP32
CASES = [(pe.PE_F64, {}), (pe.PE_F32, {}), (pe.PE_F32, dict(polarisation=pe.PE_CP)),
         (pe.PE_F32, dict(brems_method=pe.PE_BREMS_NULL))]


@pytest.mark.parametrize("precision,kw", CASES)
def test_noalloc_pic_steps_match_pe_step(precision, kw):
    import torch
    tp, Z = pe.table_params(n_eta=48, n_y=48, n_E=48, n_s=48, Z=(13.0, 79.0))
    tables = pe.pe_create_tables(tp, Z)
    n = 1500
    a = pe.Run(tables, _params(precision, **kw), n, capacity=1 << 18, events=True)
    b = pe.Run(tables, _params(precision, **kw), n, capacity=1 << 18, events=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.state(), b.state())
    np.testing.assert_array_equal(a.grid.cpu().numpy(), b.grid.cpu().numpy())
    steps = (250, 150)                                   # two calls in a row, the pulse arrives in the second
    done = 0
    for k in steps:
        pe.pe_step([a.handle], k)
        pe.pe_pic_step_noalloc(tables, b.params, n, b._buffers(), done, k, b.stream.cuda_stream)
        done += k
        torch.cuda.synchronize()
        # the same kernels on the same state, currents summed in exact fixed point: equal bit for bit
        np.testing.assert_array_equal(b.state(), a.state())
        np.testing.assert_array_equal(b.grid.cpu().numpy(), a.grid.cpu().numpy())
        np.testing.assert_array_equal(b.event_words(), a.event_words())
        if a.wait is not None:
            np.testing.assert_array_equal(b.wait_words(), a.wait_words())
        ta = np.frombuffer(bytes(a.tally_out().tally), dtype=np.uint64)
        tb = b.tally.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(tb, ta)
        np.testing.assert_array_equal(b.hist.cpu().numpy(), a.hist.cpu().numpy())
    assert ta[pe.T["N_NCS_STORED"]] + ta[pe.T["N_NCS_BELOW"]] > 0
    cnt = int(min(ta[pe.T["N_PHOTONS"]], 1 << 18))
    np.testing.assert_array_equal(_photons_sorted(b, cnt), _photons_sorted(a, cnt))
    a.close()
    b.close()
    pe.pe_destroy_tables(tables)


def test_noalloc_rejects_grids_beyond_its_array():
    tp, Z = pe.table_params(n_eta=16, n_y=16, n_E=16, n_s=16, Z=(13.0, 79.0))
    tables = pe.pe_create_tables(tp, Z)
    p = _params(pe.PE_F32, n_cells=pe.PE_PIC_MAX_CELLS + 1)
    with pytest.raises(pe.PeError, match="PE_PIC_MAX_CELLS"):
        pe.pe_pic_step_noalloc(tables, p, 10, pe.Buffers(), 0, 1, None)
    pe.pe_destroy_tables(tables)

"""pe_pic_step_noalloc: PIC steps for callers that cannot allocate device memory.

Such callers (a host framework or a fixed pool owns the device memory, or the
memory budget forbids allocations once a simulation is set up) step their PIC
state with this entry point, which sums the currents in a fixed array compiled
into the library instead of memory that pe_init_particles allocates.  The test
steps one PIC state with pe_step and an identical copy with the new entry point,
two calls each in a row, and requires the same particles, grid, tallies and
photons.  It sets up everything itself, so it runs alone in a fresh process as
well as after the other tests.
"""
import numpy as np
import pytest

import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _params(precision, n_cells=600):
    run = W.base_run(**dict(W.AU, ne_over_nc=50.0, a0=270.0, geometry=pe.PE_PIC_1D, n_cells=n_cells,
                            init_dist=1, T_mev=1.0, seed=11))
    return pe.run_params(precision=precision, **run)


@pytest.mark.parametrize("precision", [pe.PE_F64, pe.PE_F32])
def test_noalloc_pic_steps_match_pe_step(precision):
    import torch
    tp, Z = pe.table_params(n_eta=48, n_y=48, n_E=48, n_s=48, Z=(13.0, 79.0))
    tables = pe.pe_create_tables(tp, Z)
    n = 1500
    a = pe.Run(tables, _params(precision), n, capacity=1 << 18, events=True)
    b = pe.Run(tables, _params(precision), n, capacity=1 << 18, events=True)
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
        rtol = 1e-9 if precision == pe.PE_F64 else 1e-5    # the parity tolerances of the PIC tests
        np.testing.assert_allclose(b.state(), a.state(), rtol=rtol, atol=rtol)
        np.testing.assert_allclose(b.grid.double().cpu().numpy(), a.grid.double().cpu().numpy(), rtol=rtol,
                                   atol=rtol * max(1.0, float(a.grid.abs().max())))
        np.testing.assert_array_equal(b.event_words(), a.event_words())
        ta = np.frombuffer(bytes(a.tally_out().tally), dtype=np.uint64)
        tb = np.frombuffer(b.tally.cpu().numpy().tobytes(), dtype=np.uint64)
        for key in ("N_NCS_STORED", "N_NCS_BELOW", "N_BR_STORED", "N_PHOTONS", "N_KILLED"):
            assert ta[pe.T[key]] == tb[pe.T[key]], key
    assert ta[pe.T["N_NCS_STORED"]] + ta[pe.T["N_NCS_BELOW"]] > 0
    ka = np.sort(a.photon_records(int(ta[pe.T["N_PHOTONS"]]))[["id_mech", "step"]], order=["id_mech", "step"])
    kb = np.sort(b.photon_records(int(tb[pe.T["N_PHOTONS"]]))[["id_mech", "step"]], order=["id_mech", "step"])
    np.testing.assert_array_equal(ka, kb)
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

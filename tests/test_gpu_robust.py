"""Failure handling that needs no GPU fault: particles whose momenta are not finite.

The caller's buffers (or arithmetic that overflowed) can hold a NaN or infinite momentum.
Every step kernel checks the state it loads at a launch boundary: such a particle is removed
(x = NaN, momenta zeroed), counted once in N_NONFINITE and N_KILLED with the steps it was
alive, and takes no further part; the other particles are untouched.  The bad values are
planted on the host, in the caller's buffers.
"""
import numpy as np
import pytest

import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TP = dict(W.tables_small(), n_eta=48, n_y=48, n_E=48, n_s=48)
BAD = {5: ("ux", float("nan")), 17: ("uz", float("inf")), 300: ("uy", float("-inf")), 301: ("ux", float("nan"))}


@pytest.mark.parametrize("precision,launch", [(pe.PE_F32, {}), (pe.PE_F32, dict(steps_per_launch=1)),
                                              (pe.PE_F32, dict(steps_per_launch=50, block=128)),
                                              (pe.PE_F64, {}), (pe.PE_F64, dict(steps_per_launch=40))])
def test_nonfinite_momenta_removed_and_counted(precision, launch):
    import torch
    run = W.base_run(a0=270.0, init_dist=1, T_mev=1.0, seed=31, **W.AU)
    tables = pe.pe_create_tables(TP, (13.0, 79.0))
    n, steps = 1001, 120
    clean = pe.Run(tables, pe.run_params(precision=precision, **run), n, events=True)
    bad = pe.Run(tables, pe.run_params(precision=precision, **run), n, events=True)
    torch.cuda.synchronize()
    for i, (name, v) in BAD.items():
        getattr(bad, name)[i] = v
    pe.pe_step_ex([clean.handle], steps, **launch)
    pe.pe_step_ex([bad.handle], steps, **launch)
    sc, sb = clean.state(), bad.state()
    tb = bad.tally_out()
    tc = clean.tally_out()
    ids = np.array(sorted(BAD))
    keep = np.setdiff1d(np.arange(n), ids)
    np.testing.assert_array_equal(sb[keep], sc[keep])
    np.testing.assert_array_equal(bad.event_words()[keep], clean.event_words()[keep])
    assert np.isnan(sb[ids, 0]).all() and (sb[ids, 2:5] == 0).all()
    assert tb.tally[pe.T["N_NONFINITE"]] == len(BAD)
    assert tb.tally[pe.T["N_KILLED"]] == len(BAD) + tc.tally[pe.T["N_KILLED"]]
    assert tb.tally[pe.T["KILLED_STEPS"]] == tc.tally[pe.T["KILLED_STEPS"]]   # removed before step 0
    assert tb.live_particle_steps == tc.live_particle_steps - len(BAD) * steps
    # counted once: stepping on finds them removed
    pe.pe_step_ex([bad.handle], 10, **launch)
    assert bad.tally_out().tally[pe.T["N_NONFINITE"]] == len(BAD)
    clean.close()
    bad.close()
    pe.pe_destroy_tables(tables)

"""Checkpoint and resume (pe_resume_particles): a run saved after some steps, written to a
file, read back into fresh buffers and continued gives the uninterrupted run's results bit
for bit -- state, event words, null-collision waits, PIC grid, tallies, histograms and
photons.  The draws are keyed on (seed, id, step, purpose), so nothing but the buffers and
the step index has to be kept."""
import numpy as np
import pytest

import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import workloads as W
from test_gpu_parity import _tp, tables

pytestmark = pytest.mark.gpu
Z = (13.0, 79.0)


def _params(kind):
    d = dict(W.AU, a0=270.0, init_dist=1, T_mev=1.0, seed=41, run_id=2)
    prec = pe.PE_F64 if kind == "f64" else pe.PE_F32
    if kind == "f32-null":
        d.update(brems_method=pe.PE_BREMS_NULL, slab_thick_m=20e-6, ne_over_nc=2e4)
    if kind == "pic":
        d.update(geometry=pe.PE_PIC_1D, n_cells=600, ne_over_nc=50.0)
    return pe.run_params(precision=prec, **W.base_run(**d))


def _sorted_photons(r):
    ph = r.photon_records()
    key = ph["id_mech"].astype(np.uint64) << np.uint64(32) | ph["step"].astype(np.uint64)
    return ph[np.argsort(key, kind="stable")]


@pytest.mark.parametrize("kind", ["f32", "f64", "f32-null", "pic"])
def test_resume_equals_uninterrupted(kind, tmp_path):
    lt, _ = tables(_tp(48), Z)
    n, first, second = 3000, 250, 350
    a = pe.Run(lt, _params(kind), n, capacity=1 << 20, events=True)
    pe.pe_step([a.handle], first + second)
    b = pe.Run(lt, _params(kind), n, capacity=1 << 20, events=True)
    pe.pe_step([b.handle], first)
    path = str(tmp_path / "ckpt.npz")
    b.save(path)
    b.close()
    c = pe.Run.load(lt, _params(kind), path)
    assert c.tally_out().steps_done == first
    pe.pe_step([c.handle], second)
    ta, tc = a.tally_out(), c.tally_out()
    assert ta.steps_done == tc.steps_done == first + second
    np.testing.assert_array_equal(c.state(), a.state())
    np.testing.assert_array_equal(c.event_words(), a.event_words())
    assert bytes(tc.tally) == bytes(ta.tally) and bytes(tc.hist) == bytes(ta.hist)
    assert ta.tally[pe.T["N_NCS_STORED"]] > 0
    np.testing.assert_array_equal(_sorted_photons(c), _sorted_photons(a))
    if kind == "f32-null":
        np.testing.assert_array_equal(c.wait_words(), a.wait_words())
    if kind == "pic":
        np.testing.assert_array_equal(c.grid.cpu().numpy(), a.grid.cpu().numpy())
    a.close()
    c.close()


def test_resume_argument_checks():
    lt, _ = tables(_tp(33), Z)
    r = pe.Run(lt, _params("f32"), 10)
    with pytest.raises(pe.PeError):
        pe.pe_resume_particles(lt, _params("f32"), 10, r._buffers(), -1, r.stream.cuda_stream)
    with pytest.raises(pe.PeError):
        pe.pe_resume_particles(lt, _params("f32"), 10, r._buffers(), 1 << 32, r.stream.cuda_stream)
    r.close()

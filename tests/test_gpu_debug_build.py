"""The debug build (PE_DEBUG) on the workloads of the test suite: no table row or column, guide
entry or histogram bin out of range, and results equal to the release build's.

In the debug library every table index a kernel is about to use is checked against its array
and an index out of range is counted and clamped (pe_debug_count), the substitute for a memory
checker.  Each library is loaded in a child process of its own (the binding loads one library
per process); the child runs the paired FP32 step (resident and one-step forms), the FP64 plain
and persistent steps, the 2D focus, the reflected wave, null-collision brems, the 1D PIC, the
Bethe-Heitler and Breit-Wheeler transports of the photons, and writes its results.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _workloads(out_path):
    sys.path.insert(0, ROOT)
    import torch
    import paper_1612_07592_gb300 as pe
    from paper_1612_07592_gb300 import workloads as W
    tp = dict(W.tables_small(), n_eta=48, n_y=48, n_E=48, n_s=48)
    tables = pe.pe_create_tables(tp, (13.0, 79.0))
    bw = pe.pe_bw_tables_create(64, 1e-2, 1e3, 128)
    res = {"debug_build": np.array([pe.pe_debug_build()])}
    cases = {
        "f32_resident": (W.base_run(a0=270.0, init_dist=1, seed=2, **W.AU), pe.PE_F32, 1500, 600, {}),
        "f32_stream": (W.base_run(a0=270.0, init_dist=1, seed=3, **W.AU), pe.PE_F32, 1501, 300,
                       dict(steps_per_launch=1)),
        "f64_plain": (W.base_run(a0=270.0, init_dist=1, seed=4, **W.AU), pe.PE_F64, 700, 400, {}),
        "f64_persistent": (W.base_run(a0=270.0, init_dist=1, seed=4, **W.AU), pe.PE_F64, 700, 400,
                           dict(steps_per_launch=50)),
        "f32_2d_cp": (W.base_run(a0=855.0, polarisation=1, geometry=1, slab_thick_m=2e-6, seed=5, **W.AU), pe.PE_F32,
                      800, 500, {}),
        "f32_reflected": (W.base_run(a0=270.0, init_dist=1, reflect_r=1.0, mirror_x_m=3e-6, seed=6, **W.AU),
                          pe.PE_F32, 1000, 900, {}),
        "f32_null_dense": (W.base_run(a0=270.0, init_dist=1, seed=7, brems_method=1, slab_thick_m=20e-6,
                                      **dict(W.AU, ne_over_nc=2e4)), pe.PE_F32, 1000, 600, {}),
        "f32_pic": (W.base_run(a0=270.0, init_dist=1, geometry=pe.PE_PIC_1D, n_cells=600, seed=8, **W.AU), pe.PE_F32,
                    1000, 300, {}),
        "f64_bunch": (dict(W.bunch(1000.0, "Au")["run"]), pe.PE_F64, 400, 2000, {}),
    }
    for name, (run, prec, n, steps, launch) in cases.items():
        r = pe.Run(tables, pe.run_params(precision=prec, **run), n, capacity=1 << 18, events=True)
        pe.pe_step_ex([r.handle], steps, **launch)
        t = r.tally_out()
        res[name + "_state"] = r.state()
        res[name + "_events"] = r.event_words()
        res[name + "_tally"] = np.frombuffer(bytes(t.tally), dtype=np.uint64).copy()
        res[name + "_hist"] = np.frombuffer(bytes(t.hist), dtype=np.uint64).copy()
        if name in ("f64_bunch", "f32_reflected"):
            ph = r.photon_records()
            ph = ph[np.lexsort((ph["step"], ph["id_mech"]))]
            if name == "f64_bunch":
                pairs, n_pairs, ptal = r.pair_transport(photons=ph)
            else:
                pairs, n_pairs, ptal = r.bw_transport(bw, photons=ph)
            res[name + "_pairs"] = np.sort(pairs["photon"].astype(np.int64) << 32 | pairs["step"].astype(np.int64))
            res[name + "_ptally"] = ptal.copy()
        r.close()
    torch.cuda.synchronize()
    res["violations"] = np.array([pe.pe_debug_count(tables, bw)])
    np.savez(out_path, **res)


def _run_child(lib, out):
    env = dict(os.environ, PE_LIB_PATH=lib)
    subprocess.run([sys.executable, os.path.abspath(__file__), str(out)], env=env, check=True, timeout=900)
    return dict(np.load(out))


@pytest.mark.gpu
def test_debug_build_finds_nothing_out_of_range(tmp_path):
    from paper_1612_07592_gb300 import build
    rel = _run_child(build.build(), tmp_path / "release.npz")
    dbg = _run_child(build.build_debug(), tmp_path / "debug.npz")
    assert rel["debug_build"][0] == 0 and dbg["debug_build"][0] == 1
    assert rel["violations"][0] == 0
    assert dbg["violations"][0] == 0, "table indices out of range in the debug build"
    for k in rel:
        if k in ("debug_build", "violations"):
            continue
        np.testing.assert_array_equal(dbg[k], rel[k], err_msg=k)


if __name__ == "__main__":
    _workloads(sys.argv[1])

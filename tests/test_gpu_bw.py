"""Breit-Wheeler pair production of photons in the laser field on the device (pe_bw_transport)
against the oracle's or_bw_transport (Sec. 1 names the process; the rate is the locally constant
crossed field one of the NCS module, Sec. 2.2).

FP64: the same pair list as the oracle -- photon, conversion step, position, energies -- and the
same tallies, in a constant crossed field (constant chi) and in the a0 = 270 pulse reflected by
a mirror (photons meeting the incident or the reflected pulse head on).  The two sides build
their tables independently (64 x 128 nodes agree to ~1e-13), so the optical depths agree to
rounding.  FP32: the same draws, so conversions coincide with the FP64 oracle's except where
the optical depth crosses zero within FP32 rounding; the positron spectrum is checked by
chi-square.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import workloads as W

pytestmark = pytest.mark.gpu
Z = (13.0, 79.0)
TP = dict(W.tables_small(), n_eta=16, n_y=16, n_E=16, n_s=16)

_T = {}


def tables():
    if not _T:
        _T["lib"] = pe.pe_create_tables(TP, Z)
        _T["bw"] = pe.pe_bw_tables_create(64, 1e-2, 1e3, 128)
        _T["o"] = O.Tables(O.table_params(**{("photon_min" if k == "photon_min_mc2" else k): v
                                             for k, v in TP.items()}), list(Z))
        _T["obw"] = O.BWTables(n_chi=64, chi_min=1e-2, chi_max=1e3, n_x=128)
    return _T


def _orun(run):
    d = dict(run)
    d["iz"] = list(Z).index(d["Z"])
    return O.run_params(**d)


def _lib_run(run, steps, precision):
    r = pe.Run(tables()["lib"], pe.run_params(precision=precision, **run), 0, capacity=1)
    pe.pe_step([r.handle], steps)
    return r


def _photons_crossed(n):
    ph = np.zeros(n, dtype=pe.PHOTON_DTYPE)
    rng = np.random.default_rng(7)
    ph["energy"] = np.exp(rng.uniform(math.log(300.0), math.log(3000.0), n))
    ph["kx"] = -1.0
    ph["x"] = rng.uniform(-5.0, 5.0, n)
    ph["step"] = rng.integers(0, 20, n)
    ph["id_mech"] = np.arange(n, dtype=np.uint32) | (rng.integers(0, 2, n).astype(np.uint32) << np.uint32(31))
    ph["energy"][:7] = 1.5                                   # below the pair threshold: skipped
    return ph


def _photons_reflected(n):
    # emitted in and around a 1 um Au slab at 2-3 um (12.6-18.8 c/omega), both directions
    ph = W.synthetic_photons(n, 11, x_range=(10.0, 22.0), k_range=(30.0, 1e4), step_range=(0, 600),
                             theta_max=0.4)
    back = np.random.default_rng(12).uniform(0, 1, n) < 0.45
    ph["kx"] = np.where(back, -np.abs(ph["kx"]), np.abs(ph["kx"]))
    return ph


def _sorted_pairs(p):
    return p[np.argsort(p["photon"], kind="stable")]


def _compare_f64(r, run, ph, step_end):
    t = tables()
    pairs, npairs, tal = r.bw_transport(t["bw"], photons=ph, step_end=step_end)
    po, npo, talo = O.bw_transport(t["obw"], t["o"], _orun(run), ph, step_end=step_end)
    print(f"pairs {npairs} (oracle {npo}) of {len(ph)} photons, photon-steps {int(tal[3])}")
    assert npairs == npo > 0
    for k in ("N_ENTERED", "N_K_ABOVE", "N_TESTS"):
        assert tal[pe.PT[k]] == talo[O.PT[k]], k
    assert tal[pe.PT["E_PAIRS"]] == talo[O.PT["E_PAIRS"]] and tal[pe.PT["E_PAIRS"] + 1] == talo[O.PT["E_PAIRS"] + 1]
    ep = pe.fixed_to_float(tal, pe.PT["E_POSITRONS"])
    assert abs(ep / O.fixed_to_float(talo, O.PT["E_POSITRONS"]) - 1) < 1e-12
    a, b = _sorted_pairs(pairs), _sorted_pairs(po)
    for f in ("photon", "step", "id_mech", "kx", "ky", "kz"):
        np.testing.assert_array_equal(a[f], b[f])
    for f in ("x", "y", "e_minus", "e_plus"):
        np.testing.assert_allclose(a[f], b[f], rtol=1e-6, atol=1e-6)
    return pairs, tal


def test_f64_constant_crossed_field_equals_oracle():
    run = W.base_run(geometry=pe.PE_CONST, E_const=(0.0, 300.0, 0.0), B_const=(0.0, 0.0, 300.0), seed=77,
                     run_id=3)
    steps = 90
    r = _lib_run(run, steps, pe.PE_F64)
    pairs, tal = _compare_f64(r, run, _photons_crossed(30_000), steps)
    assert tal[pe.PT["N_ENTERED"]] == 30_000 - 7
    r.close()


@pytest.mark.parametrize("pol", [pe.PE_LP_Y, pe.PE_CP])
def test_f64_reflected_wave_equals_oracle(pol):
    run = W.base_run(a0=270.0, polarisation=pol, reflect_r=1.0, mirror_x_m=3e-6, seed=5, run_id=9, **W.AU)
    steps = 1400
    r = _lib_run(run, steps, pe.PE_F64)
    _compare_f64(r, run, _photons_reflected(20_000), steps)
    r.close()


def test_f32_conversions_follow_the_f64_oracle():
    """FP32 transport of the reflected-wave photons: the draws are the oracle's, so a photon
    converts at the same step unless its optical depth crosses zero within FP32 rounding of the
    fields and the rate (a small fraction); the positron-share spectrum agrees (chi-square)."""
    from scipy.stats import chi2 as chi2d
    t = tables()
    run = W.base_run(a0=270.0, reflect_r=1.0, mirror_x_m=3e-6, seed=5, run_id=9, **W.AU)
    steps = 1400
    ph = _photons_reflected(60_000)
    r = _lib_run(run, steps, pe.PE_F32)
    pairs, npairs, tal = r.bw_transport(t["bw"], photons=ph, step_end=steps)
    po, npo, talo = O.bw_transport(t["obw"], t["o"], _orun(run), ph, step_end=steps)
    conv = np.full(len(ph), -1, np.int64)
    conv[pairs["photon"]] = pairs["step"]
    conv_o = np.full(len(ph), -1, np.int64)
    conv_o[po["photon"]] = po["step"]
    same = np.mean(conv == conv_o)
    print(f"FP32 pairs {npairs}, oracle {npo}; same conversion step for {same:.5f} of the photons")
    assert npo > 2000
    assert same > 0.995
    assert abs(npairs - npo) <= np.sum(conv != conv_o)
    assert tal[pe.PT["N_ENTERED"]] == talo[O.PT["N_ENTERED"]]
    h1 = np.histogram(pairs["e_plus"] / (pairs["e_plus"] + pairs["e_minus"]), 20, (0, 1))[0].astype(float)
    h2 = np.histogram(po["e_plus"] / (po["e_plus"] + po["e_minus"]), 20, (0, 1))[0].astype(float)
    stat = np.sum((h1 - h2) ** 2 / np.maximum(h1 + h2, 1))
    assert chi2d.sf(stat, 19) > 1e-3
    r.close()


def test_bw_edge_cases():
    import torch
    t = tables()
    run = W.base_run(geometry=pe.PE_CONST, E_const=(0.0, 300.0, 0.0), B_const=(0.0, 0.0, 300.0), seed=77)
    r = _lib_run(run, 60, pe.PE_F64)
    ph = _photons_crossed(5000)
    full, n_full, tal_full = r.bw_transport(t["bw"], photons=ph, step_end=60)
    # capacity overflow: exact counts, nothing past the capacity
    small, n_small, tal_small = r.bw_transport(t["bw"], photons=ph, step_end=60, capacity=3)
    assert n_small == n_full > 3 and len(small) == 3
    np.testing.assert_array_equal(tal_small, tal_full)
    # no steps after emission: nothing happens
    _, n0, tal0 = r.bw_transport(t["bw"], photons=ph, step_end=0)
    assert n0 == 0 and tal0[pe.PT["N_TESTS"]] == 0
    # argument errors
    with pytest.raises(pe.PeError) as e:
        r.bw_transport(t["bw"], photons=ph, step_end=61)
    assert e.value.status == pe.PE_ERR_ARG
    pic = pe.Run(t["lib"], pe.run_params(precision=pe.PE_F64, **W.base_run(geometry=pe.PE_PIC_1D, n_cells=600)), 10)
    dev = torch.zeros(8 * 4, dtype=torch.int32, device="cuda")
    out = torch.zeros(10, dtype=torch.int32, device="cuda")
    tl = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(pe.PeError) as e:
        pe.pe_bw_transport(pic.handle, t["bw"], dev.data_ptr(), 4, 0, out.data_ptr(), 1, tl.data_ptr())
    assert e.value.status == pe.PE_ERR_STATE
    with pytest.raises(pe.PeError) as e:
        pe.pe_bw_tables_create(1, 1e-2, 1e3, 128)
    assert e.value.status == pe.PE_ERR_ARG
    pic.close()
    r.close()

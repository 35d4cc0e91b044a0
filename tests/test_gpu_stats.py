"""FP32 statistics against the FP64 oracle: photon spectra and angles (the paper's Figs. 6-7),
the bremsstrahlung / NCS yield ratio, and the photon (x, energy) map (Fig. 4, in 1D).

The FP32 path and the oracle run the same workload with independent seeds, so only
distributions can agree.  One electron's successive photons are correlated (its energy and
direction change slowly), so the spectra and angle distributions are compared on one photon
per electron -- its first stored photon, the same rule on both sides -- which makes the
entries independent.  Two-sample chi-square over the bins (sparse bins merged until each
merged bin holds >= 20 entries of the two samples together), p > 1e-3.  The yield ratio is
compared within 3 sigma, sigma from the per-electron event counts (the variance of a ratio
estimator; it reduces to the Poisson one when the electrons are alike).  The device histogram
words themselves are checked against the histogram of the device's photon records.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import workloads as W
from test_gpu_parity import _tp, orun, run_oracle, sort_photons, tables

pytestmark = pytest.mark.gpu
Z = (13.0, 79.0)
P_MIN = 1e-3
LASER = W.base_run(a0=270.0, init_dist=1, T_mev=1.0, **W.AU)
# a 20 um Au slab at 2e4 n_c under the same pulse: NCS and brems both abundant
DENSE = W.base_run(a0=270.0, init_dist=1, T_mev=1.0, slab_thick_m=20e-6, **dict(W.AU, ne_over_nc=2e4))
E_EDGES = np.linspace(math.log(0.51099895), math.log(1e4), 513)       # histogram bins of the library (MeV)
T_EDGES = np.linspace(-math.pi, math.pi, 181)


def chi2_two_sample(h1, h2, min_count=20):
    """Two-sample chi-square of histograms with different totals; returns (stat, dof, p)."""
    from scipy.stats import chi2
    m1, m2, a, b = [], [], 0.0, 0.0
    for x, y in zip(np.asarray(h1, float), np.asarray(h2, float)):
        a += x
        b += y
        if a + b >= min_count:
            m1.append(a)
            m2.append(b)
            a = b = 0.0
    if a + b > 0 and m1:
        m1[-1] += a
        m2[-1] += b
    m1, m2 = np.array(m1), np.array(m2)
    k1, k2 = math.sqrt(m2.sum() / m1.sum()), math.sqrt(m1.sum() / m2.sum())
    stat = float(np.sum((k1 * m1 - k2 * m2) ** 2 / (m1 + m2)))
    dof = len(m1) - 1
    return stat, dof, float(chi2.sf(stat, dof))


def first_photons(ph, mech):
    """The first stored photon of each electron for one mechanism (0 NCS, 1 brems)."""
    sel = ph[(ph["id_mech"] >> 31) == mech]
    sel = sel[np.lexsort((sel["step"], sel["id_mech"]))]
    _, first = np.unique(sel["id_mech"], return_index=True)
    return sel[first]


def energy_theta(ph):
    e = np.log(ph["energy"].astype(np.float64) * 0.51099895)
    th = np.arctan2(ph["ky"].astype(np.float64), ph["kx"].astype(np.float64))
    return np.histogram(e, E_EDGES)[0], np.histogram(th, T_EDGES)[0]


def _gpu(lt, run, n, steps, seed):
    r = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **dict(run, seed=seed)), n, capacity=1 << 23, events=True)
    pe.pe_step([r.handle], steps)
    out = r.tally_out()
    assert out.status == pe.PE_OK
    return r, out


def _oracle(ot, run, n, steps, seed):
    st, ph, nph, hist, tal, ev = run_oracle(ot, dict(run, seed=seed), Z, np.arange(n), steps)
    assert nph == len(ph)
    return ph, hist, tal, ev


def _assert_device_hist_is_records(out, ph):
    """The histogram words equal the histogram of the stored records (a few bin-edge ties)."""
    hist = np.frombuffer(bytes(out.hist), dtype=np.uint64).astype(np.int64)
    for mech in (0, 1):
        sel = ph[(ph["id_mech"] >> 31) == mech]
        he, ht = energy_theta(sel)
        assert np.abs(hist[512 * mech:512 * mech + 512] - he).sum() <= max(4, len(sel) // 20000)
        assert np.abs(hist[1024 + 180 * mech:1024 + 180 * mech + 180] - ht).sum() <= max(4, len(sel) // 20000)


def _check(name, h1, h2):
    stat, dof, p = chi2_two_sample(h1, h2)
    print(f"{name}: chi2 {stat:.1f} dof {dof} p {p:.3g} (entries {int(np.sum(h1))} / {int(np.sum(h2))})")
    assert np.sum(h1) > 1000 and np.sum(h2) > 1000
    assert p > P_MIN, name


def test_ncs_spectrum_and_angles_chi2():
    lt, ot = tables(_tp(48), Z)
    r, out = _gpu(lt, LASER, 100_000, 1200, seed=202)
    ph = r.photon_records()
    _assert_device_hist_is_records(out, ph)
    ph_o, _, _, _ = _oracle(ot, LASER, 40_000, 1200, seed=101)
    e1, t1 = energy_theta(first_photons(ph, 0))
    e2, t2 = energy_theta(first_photons(ph_o, 0))
    _check("NCS energy", e1, e2)
    _check("NCS angle", t1, t2)
    r.close()


def _ratio_sigma(ev):
    """Brems / NCS ratio of one sample and its standard error from the per-electron counts."""
    ev = ev.astype(np.uint64)
    n_c = (ev & np.uint64(0xFFFF)).astype(float)
    b_c = ((ev >> np.uint64(16)) & np.uint64(0xFFFF)).astype(float)
    R = b_c.sum() / n_c.sum()
    m = len(ev)
    var = np.var(b_c - R * n_c, ddof=1) * m / n_c.sum() ** 2
    return R, math.sqrt(var)


def test_brems_spectrum_angles_and_yield_ratio():
    lt, ot = tables(_tp(48), Z)
    r, out = _gpu(lt, DENSE, 100_000, 1200, seed=204)
    ph = r.photon_records()
    _assert_device_hist_is_records(out, ph)
    ph_o, _, tal_o, ev_o = _oracle(ot, DENSE, 40_000, 1200, seed=103)
    e1, t1 = energy_theta(first_photons(ph, 1))
    e2, t2 = energy_theta(first_photons(ph_o, 1))
    _check("brems energy", e1, e2)
    _check("brems angle", t1, t2)
    ev = r.event_words()
    R1, s1 = _ratio_sigma(ev)
    R2, s2 = _ratio_sigma(ev_o)
    print(f"brems/NCS: FP32 {R1:.5f} +- {s1:.5f}, oracle {R2:.5f} +- {s2:.5f}")
    tal = np.frombuffer(bytes(out.tally), dtype=np.uint64)
    assert tal[pe.T["N_BR_STORED"]] + tal[pe.T["N_BR_BELOW"]] > 5000
    assert abs(R1 - R2) <= 3 * math.hypot(s1, s2)
    r.close()


def test_bunch_brems_spectrum_chi2():
    """The paper's own benchmark (Sec. 2.2: 1 GeV electrons into 5 mm Au, fields off): the first
    brems photon of each electron samples the Eq. 1 spectrum at the beam energy."""
    c = W.bunch(1000.0, "Au", n=20_000)
    lt, ot = tables(c["tables"], c["Z"])
    r, out = _gpu(lt, c["run"], 60_000, c["steps"], seed=301)
    ph = r.photon_records()
    ph_o, _, _, _ = _oracle(ot, c["run"], 20_000, c["steps"], seed=302)
    e1, _ = energy_theta(first_photons(ph, 1))
    e2, _ = energy_theta(first_photons(ph_o, 1))
    _check("bunch brems energy", e1, e2)
    # and all photons of the bunch: the energy-loss spectrum
    _check("bunch brems energy, all photons / 10", energy_theta(ph[::10])[0], energy_theta(ph_o[::3])[0])
    r.close()


def _map_of(ph, nx, x0, x1, ne, e0, e1, kl):
    xb = np.floor((ph["x"].astype(np.float64) - x0 * kl) * (nx / ((x1 - x0) * kl)))
    eb = np.floor((np.log(ph["energy"].astype(np.float64) * 0.51099895) - math.log(e0)) *
                  (ne / (math.log(e1) - math.log(e0))))
    ok = (xb >= 0) & (xb < nx) & (eb >= 0) & (eb < ne)
    m = np.zeros((nx, ne), dtype=np.int64)
    np.add.at(m, (xb[ok].astype(int), eb[ok].astype(int)), 1)
    return m


@pytest.mark.parametrize("case", ["prescribed", "pic"])
def test_photon_map_matches_oracle(case):
    """pe_photon_map of an FP64 run against the same map binned from the oracle's photon records
    (identical event lists, so the records agree to rounding: only bin-edge ties may differ)."""
    lt, ot = tables(_tp(48), Z)
    kl = 2 * math.pi / 1e-6
    if case == "prescribed":
        run = dict(LASER, seed=2)
        n, steps = 1000, 1500
        r = pe.Run(lt, pe.run_params(precision=pe.PE_F64, **run), n, capacity=1 << 20, events=True)
        pe.pe_step([r.handle], steps)
        _, ph_o, nph_o, _, _, ev_o = run_oracle(ot, run, Z, np.arange(n), steps)
        x0, x1 = 0.0, 40e-6
    else:
        from test_gpu_pic import NC, _oracle as pic_oracle, _run as pic_run
        run = pic_run()
        n, steps = 2000, 400
        r = pe.Run(lt, pe.run_params(precision=pe.PE_F64, **run), n, capacity=1 << 20, events=True)
        pe.pe_step([r.handle], steps)
        _, _, ev_o, ph_o, nph_o, _, _ = pic_oracle(ot, run, n, steps)
        x0, x1 = 0.0, NC * 0.01e-6
    np.testing.assert_array_equal(r.event_words(), ev_o)
    assert r.tally_out().photons_stored == nph_o > 50
    m = r.photon_map(48, x0, x1, 40, 0.511, 1e4)
    want = _map_of(ph_o, 48, x0, x1, 40, 0.511, 1e4, kl)
    print(f"{case}: {int(m.sum())} photons in the map, {int(np.abs(m.astype(np.int64) - want).sum())} differ")
    assert m.sum() > 50
    assert np.abs(m.astype(np.int64) - want).sum() <= 2
    r.close()

"""GPU parity of the Bethe-Heitler pair production of photons in the target
(pe_pair_transport) with the oracle, and its conversion law at the size of the
bunch workload."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import workloads as W
from test_gpu_parity import _tp, tables

pytestmark = pytest.mark.gpu
Z = (13.0, 79.0)
KL = 2 * math.pi / 1e-6


@pytest.mark.parametrize("n", [33, 128])
def test_bh_tables_match_oracle(n):
    lt, ot = tables(_tp(n), Z)
    for iz in (0, 1):
        np.testing.assert_allclose(pe.pe_tables_export(lt, 5, iz), ot.export(5, iz), rtol=1e-9, atol=1e-300)
        np.testing.assert_allclose(pe.pe_tables_export(lt, 6, iz), ot.export(6, iz).ravel(), rtol=1e-9, atol=1e-13)


def _run(lt, steps, precision=pe.PE_F64, **kw):
    """A run with no electrons advanced `steps` steps: its target, seed and step count are
    what the transport of external photon records uses."""
    d = dict(a0=0.0, geometry=2, Z=79.0, charge_state=79.0, ne_over_nc=4177.0, slab_x0_m=0.0,
             slab_thick_m=2e-3, dt_over_T=1.0, enable_ncs=0, seed=31, run_id=4)
    d.update(kw)
    r = pe.Run(lt, pe.run_params(precision=precision, **W.base_run(**d)), 0)
    pe.pe_step([r.handle], steps)
    return r, d


def _oracle_pairs(ot, d, photons, step_end, method=O.PAIR_DIRECT):
    od = dict(W.base_run(**d))
    od.pop("precision", None)
    od["iz"] = list(Z).index(od["Z"])
    return O.pair_transport(ot, O.run_params(**od), photons, step_end, capacity=len(photons) + 1, method=method)


METHODS = [(pe.PE_PAIR_DIRECT, O.PAIR_DIRECT), (pe.PE_PAIR_FREE_PATH, O.PAIR_FREE_PATH)]


def _compare(dev, dev_n, dev_t, orc, orc_n, orc_t):
    assert dev_n == orc_n
    for k in ("N_PAIRS", "N_ENTERED", "N_K_ABOVE", "N_TESTS"):
        assert int(dev_t[pe.PT[k]]) == int(orc_t[O.PT[k]]), k
    for k in ("E_PAIRS", "E_POSITRONS"):
        a, b = pe.fixed_to_float(dev_t, pe.PT[k]), O.fixed_to_float(orc_t, O.PT[k])
        assert abs(a - b) <= 1e-9 * max(b, 1.0), k
    d = np.sort(dev, order="photon")
    o = np.sort(orc, order="photon")
    for f in ("photon", "step", "id_mech", "x", "y", "kx", "ky", "kz"):
        np.testing.assert_array_equal(d[f], o[f], err_msg=f)
    for f in ("e_minus", "e_plus"):
        np.testing.assert_allclose(d[f], o[f], rtol=2e-7, err_msg=f)


@pytest.mark.parametrize("method", METHODS, ids=["direct", "free_path"])
@pytest.mark.parametrize("precision", [pe.PE_F64, pe.PE_F32])
def test_pair_transport_parity_1d(precision, method):
    """Synthetic photons (emission points through and before a 2 mm solid-Au target, 1 mc^2 to
    1e5 mc^2, cones about +x with 10 % reversed, emission steps up to 2500): the device converts
    the same photons at the same steps with the same positron energies as the oracle, by either
    method."""
    lt, ot = tables(_tp(48), Z)
    steps = 3000
    r, d = _run(lt, steps, precision)
    ph = W.synthetic_photons(30000, 9, (-50.0, 2e-3 * KL), (1.0, 1e5), (0, 2500))
    dev, dev_n, dev_t = r.pair_transport(ph, method=method[0])
    orc, orc_n, orc_t = _oracle_pairs(ot, d, ph, steps, method[1])
    assert orc_n > 2000 and orc_t[O.PT["N_K_ABOVE"]] == 0
    if method[0] == pe.PE_PAIR_FREE_PATH:
        # one draw per photon in the target with P > 0 (sigma_BH is clamped to 0 just above k = 2)
        assert 0 < orc_t[O.PT["N_TESTS"]] <= orc_t[O.PT["N_ENTERED"]]
    _compare(dev, dev_n, dev_t, orc, orc_n, orc_t)
    r.close()


@pytest.mark.parametrize("method", METHODS, ids=["direct", "free_path"])
def test_pair_transport_parity_2d_and_al(method):
    """2D target strip |y| <= 3 um (photons leave it sideways) on Al, and a transport window that
    ends before the run's last step."""
    lt, ot = tables(_tp(48), Z)
    steps = 4000
    r, d = _run(lt, steps, geometry=1, Z=13.0, charge_state=13.0, ne_over_nc=711.0, slab_thick_m=3e-3,
                y_half_m=3e-6)
    ph = W.synthetic_photons(30000, 10, (0.0, 3e-3 * KL), (3.0, 2e6), (0, 3000), theta_max=0.003,
                             y_half=3e-6 * KL)
    dev, dev_n, dev_t = r.pair_transport(ph, step_end=3500, method=method[0])
    orc, orc_n, orc_t = _oracle_pairs(ot, d, ph, 3500, method[1])
    assert orc_n > 100 and orc_t[O.PT["N_K_ABOVE"]] > 0
    _compare(dev, dev_n, dev_t, orc, orc_n, orc_t)
    r.close()


def test_pair_transport_edges_and_capacity():
    lt, ot = tables(_tp(33), Z)
    r, d = _run(lt, 100, slab_thick_m=1e-3)
    x1 = 1e-3 * KL
    ph = np.zeros(6, dtype=W.PHOTON_RECORD)
    ph["energy"] = [1e4, 2.0, 1e4, 1e4, 1e4, 1e4]
    ph["x"] = [-1.0, 10.0, -1.0, x1 + 1.0, 10.0, 10.0]
    ph["kx"] = [1.0, 1.0, -1.0, 1.0, 1.0, 1.0]
    ph["step"] = [0, 0, 0, 0, 98, 99]
    ph["id_mech"] = np.arange(6)
    dev, dev_n, dev_t = r.pair_transport(ph)
    orc, orc_n, orc_t = _oracle_pairs(ot, d, ph, 100)
    _compare(dev, dev_n, dev_t, orc, orc_n, orc_t)
    assert int(dev_t[pe.PT["N_ENTERED"]]) == 2
    # no photons; capacity below the pair count (the true count is reported, capacity records written)
    e, n0, t0 = r.pair_transport(ph[:0], n_photons=0)
    assert n0 == 0 and len(e) == 0
    many = W.synthetic_photons(5000, 3, (0.0, x1), (1e3, 1e5), (0, 10))
    full, nf, tf = r.pair_transport(many)
    part, npart, tp = r.pair_transport(many, capacity=7)
    assert npart == nf > 7 and len(part) == 7
    assert set(part["photon"].tolist()) <= set(full["photon"].tolist())
    with pytest.raises(pe.PeError):
        r.pair_transport(many, step_end=101)
    with pytest.raises(pe.PeError):
        r.pair_transport(many, method=2)
    # the free path on the edge photons (entering at the last step, reversed, beyond the target)
    dev, dev_n, dev_t = r.pair_transport(ph, method=pe.PE_PAIR_FREE_PATH)
    orc, orc_n, orc_t = _oracle_pairs(ot, d, ph, 100, O.PAIR_FREE_PATH)
    _compare(dev, dev_n, dev_t, orc, orc_n, orc_t)
    r.close()


def test_pair_conversion_of_the_bunch_photons():
    """The paper's bunch (1 GeV electrons into 5 mm of solid Au, fields off): the brems photons the
    device stored convert in the rest of the target.  Expected count: the sum over photons of
    1 - (1 - P(k))^N, N the steps each spends inside the target before the run ends and P from the
    exported sigma_BH table; the device count agrees within 5 sigma."""
    b = W.bunch(1000.0, "Au", n=20000)
    lt, _ = tables(_tp(48), Z)
    run = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **b["run"]), b["n"], capacity=1 << 22)
    pe.pe_step([run.handle], b["steps"])
    ph = run.photon_records()
    assert len(ph) > 100000
    pairs, n_pairs, t = run.pair_transport()
    fpairs, n_free, tf = run.pair_transport(method=pe.PE_PAIR_FREE_PATH)
    steps = b["steps"]
    dt = 2 * math.pi
    x1 = 5e-3 * KL
    k = ph["energy"].astype(np.float64)
    kx = ph["kx"].astype(np.float64)
    xe = ph["x"].astype(np.float64)
    ne = ph["step"].astype(np.int64)
    # steps inside [0, x1] at positions xe + kx (m - ne) dt for ne < m < steps (kx > 0 here)
    assert np.all(kx > 0)
    m_lo = np.maximum(ne + 1, ne + np.ceil((0.0 - xe) / (kx * dt)).astype(np.int64))
    m_hi = np.minimum(steps - 1, ne + np.floor((x1 - xe) / (kx * dt)).astype(np.int64))
    N = np.clip(m_hi - m_lo + 1, 0, None)
    ks = np.exp(np.linspace(np.log(2.0), np.log(1e6), 48))
    sig = np.interp(np.log(np.maximum(k, 2.0)), np.log(ks), pe.pe_tables_export(lt, 5, 1))
    sig[k <= 2.0] = 0.0
    n_i = 4177.0 * math.pi / (2.8179403262e-15 * 1e-12) / 79.0
    P = -np.expm1(-n_i * 7.2973525693e-3 * 2.8179403262e-15 ** 2 * sig * 1e-6)
    pc = 1.0 - (1.0 - P) ** N
    mean, var = pc.sum(), (pc * (1 - pc)).sum()
    assert n_pairs > 1000
    assert abs(n_pairs - mean) < 5 * math.sqrt(var), (n_pairs, mean)
    assert abs(n_free - mean) < 5 * math.sqrt(var), (n_free, mean)
    assert 0 < int(tf[pe.PT["N_TESTS"]]) <= int(tf[pe.PT["N_ENTERED"]]) == int(t[pe.PT["N_ENTERED"]])
    for p in (pairs, fpairs):
        np.testing.assert_allclose(p["e_minus"].astype(np.float64) + p["e_plus"], k[p["photon"]], rtol=1e-6)
    run.close()

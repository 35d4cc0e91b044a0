"""Pins of the oracle's Breit-Wheeler pair production (photon in the laser field, locally
constant crossed-field rate): the special function, the spectrum's structure against the
pinned emission spectrum, both asymptotic limits of the total rate, the tables, the sampler,
the photon quantum parameter, and the conversion law of the transport in a constant crossed
field.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O

ALPHA = 7.2973525693e-3


def _int_kv(nu, x):
    si = pytest.importorskip("scipy.integrate")
    sp = pytest.importorskip("scipy.special")
    return si.quad(lambda t: sp.kv(nu, t), x, np.inf, limit=400, epsabs=0, epsrel=1e-12)[0]


@pytest.fixture(scope="module")
def bw():
    return O.BWTables(n_chi=24, chi_min=1e-2, chi_max=1e3, n_x=64)


def test_int_k13_matches_scipy():
    for x in (0.05, 0.5, 1.0, 4.0, 20.0):
        assert O.int_k13(x) == pytest.approx(_int_kv(1.0 / 3.0, x), rel=1e-9)


def test_spectrum_structure_against_the_emission_spectrum():
    """The pair spectrum is the crossed form of the quantum-synchrotron one: with the photon
    fraction delta and y = 2 delta / (3 eta (1 - delta)) the pinned emissivity satisfies
    F(eta, chi)/delta = (2/(3 eta)) [(1/(1-delta) + (1-delta)) K_{2/3}(y) - int_y K_{1/3}],
    the bracket whose sign of the integral term flips for the pair process."""
    for eta in (0.1, 1.0, 10.0):
        for d in (0.1, 0.5, 0.9):
            y = 2 * d / (3 * eta * (1 - d))
            lhs = O.ncs_F(eta, d * eta / 2) / d
            rhs = 2 / (3 * eta) * ((1 / (1 - d) + (1 - d)) * O.bessel_k(2 / 3, y) - O.int_k13(y))
            assert lhs == pytest.approx(rhs, rel=1e-9), (eta, d)


def test_G_symmetric_and_vanishing_at_the_ends():
    for chi in (0.1, 1.0, 50.0):
        for x in (0.01, 0.2, 0.45):
            assert O.bw_G(chi, x) == pytest.approx(O.bw_G(chi, 1 - x), rel=1e-12)
        assert O.bw_G(chi, 0.0) == 0.0 and O.bw_G(chi, 1.0) == 0.0
    # both terms positive: the integrand of the rate is never negative
    assert all(O.bw_G(c, x) > 0 for c in (0.05, 1, 1e3) for x in np.linspace(0.05, 0.95, 7))


def test_small_chi_limit():
    """chi << 1: T = (3/16) sqrt(3/2) chi exp(-8/(3 chi)) (1 + O(chi)), the saddle point at x = 1/2."""
    r = []
    for chi in (0.01, 0.02, 0.04):
        a = 3 / 16 * math.sqrt(1.5) * chi * math.exp(-8 / (3 * chi))
        r.append(O.bw_T_direct(chi) / a - 1)
    assert all(abs(v) < 0.5 * c for v, c in zip(r, (0.01, 0.02, 0.04)))
    # the correction is first order in chi: halving chi halves it (within 15 %)
    assert r[1] / r[0] == pytest.approx(2.0, rel=0.15) and r[2] / r[1] == pytest.approx(2.0, rel=0.15)


def test_large_chi_limit():
    """chi >> 1: T -> C chi^(2/3), C = 15 3^(2/3) Gamma(2/3)^3 / (14 sqrt(3) pi Gamma(1/3)) = 0.3796
    (the K_{2/3} term at small argument integrated with Beta functions); the remainder falls
    as chi^(-2/3)."""
    C = 15 * 3 ** (2 / 3) * math.gamma(2 / 3) ** 3 / (14 * math.sqrt(3) * math.pi * math.gamma(1 / 3))
    assert C == pytest.approx(0.37961, abs=2e-5)
    d4 = O.bw_T_direct(1e4) / (C * 1e4 ** (2 / 3)) - 1
    d6 = O.bw_T_direct(1e6) / (C * 1e6 ** (2 / 3)) - 1
    assert abs(d6) < 1e-3 and abs(d4) < 1e-2
    assert d4 / d6 == pytest.approx(100 ** (2 / 3), rel=0.1)


def test_tables_equal_direct_quadrature(bw):
    T = bw.export(0)
    chis = np.exp(np.linspace(math.log(1e-2), math.log(1e3), 24))
    for i in (0, 5, 12, 23):
        assert T[i] == pytest.approx(O.bw_T_direct(chis[i]), rel=1e-8)
        v, fl = bw.T_interp(chis[i] * (1 + 1e-12))
        assert fl == (1 if i == 23 else 0) and v == pytest.approx(T[i], rel=1e-6)
    # between nodes ln(T e^{8/(3 chi)}) is linear in ln chi; below the table 0, above it the last node
    assert bw.T_interp(5e-3) == (0.0, -1)
    assert bw.T_interp(1e4) == (T[-1], 1)
    for i in (0, 4, 10, 20):
        mid = math.sqrt(chis[i] * chis[i + 1])
        la, lb = math.log(T[i]) + 8 / (3 * chis[i]), math.log(T[i + 1]) + 8 / (3 * chis[i + 1])
        assert bw.T_interp(mid)[0] == pytest.approx(math.exp(0.5 * (la + lb) - 8 / (3 * mid)), rel=1e-9)
        assert bw.T_interp(mid)[0] == pytest.approx(O.bw_T_direct(mid), rel=5e-3)
    # CDF rows: nodes x_j = (1 - cos(pi j/63))/2, cumulative G by scipy quadrature
    si = pytest.importorskip("scipy.integrate")
    cdf = bw.export(1)
    for i in (6, 14):
        chi = chis[i]
        xs = 0.5 * (1 - np.cos(np.pi * np.arange(64) / 63))
        tot = si.quad(lambda x: O.bw_G(chi, x), 0, 1, points=[0.5], limit=200, epsrel=1e-10)[0]
        for j in (8, 20, 32, 50):
            part = si.quad(lambda x: O.bw_G(chi, x), 0, xs[j], limit=200, epsrel=1e-10)[0]
            assert cdf[i, j] == pytest.approx(part / tot, abs=1e-8)
        assert cdf[i, 0] == 0.0 and cdf[i, -1] == pytest.approx(1.0, abs=1e-14)
        assert np.all(np.diff(cdf[i]) >= 0)


def test_sampler_follows_the_spectrum(bw):
    """x sampled at a node chi = chis[14] (~11) follows G(chi, x) (chi-square over 20 bins) and is
    symmetric about 1/2."""
    chis = np.exp(np.linspace(math.log(1e-2), math.log(1e3), 24))
    chi = chis[14]
    rng = np.random.default_rng(3)
    R = rng.random(40000)
    xs = np.array([bw.sample_x(chi, r) for r in R])
    assert xs.min() > 0 and xs.max() < 1
    si = pytest.importorskip("scipy.integrate")
    ss = pytest.importorskip("scipy.stats")
    edges = np.linspace(0, 1, 21)
    tot = si.quad(lambda x: O.bw_G(chi, x), 0, 1, points=[0.5], limit=400)[0]
    p = np.array([si.quad(lambda x: O.bw_G(chi, x), a, b, limit=200)[0] for a, b in zip(edges[:-1], edges[1:])]) / tot
    obs = np.histogram(xs, edges)[0]
    exp = p * len(xs)
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert ss.chi2.sf(chi2, 19) > 1e-4, chi2
    assert abs(xs.mean() - 0.5) < 5 * xs.std() / math.sqrt(len(xs))


def test_photon_chi_special_cases():
    E_S = O.schwinger_field(1e-6)
    k = 2000.0
    # k perpendicular to a pure magnetic field: chi = k B / E_S; to a pure electric field: k E / E_S
    assert O.chi_photon([k, 0, 0], [0, 0, 0], [0, 0, 30.0], E_S) == pytest.approx(k * 30 / E_S, rel=1e-14)
    assert O.chi_photon([0, k, 0], [0, 0, 7.0], [0, 0, 0], E_S) == pytest.approx(k * 7 / E_S, rel=1e-14)
    # along E or B: no transverse force, chi = 0
    assert O.chi_photon([0, 0, k], [0, 0, 7.0], [0, 0, 3.0], E_S) == 0.0
    # plane wave E = a y^, B = a z^: co-propagating photon chi = 0 exactly, counter-propagating 2 k a / E_S
    a = 270.0
    assert O.chi_photon([k, 0, 0], [0, a, 0], [0, 0, a], E_S) == 0.0
    assert O.chi_photon([-k, 0, 0], [0, a, 0], [0, 0, a], E_S) == pytest.approx(2 * k * a / E_S, rel=1e-14)
    # generic vectors: sqrt((k E + kvec x B)^2 - (kvec . E)^2) / E_S in exact rational arithmetic
    from fractions import Fraction as Fr
    rng = np.random.default_rng(1)
    for _ in range(20):
        kv, E, B = rng.normal(size=3) * 100, rng.normal(size=3) * 50, rng.normal(size=3) * 50
        kf, Ef, Bf = [Fr(float(v)) for v in kv], [Fr(float(v)) for v in E], [Fr(float(v)) for v in B]
        kk = math.sqrt(float(sum(v * v for v in kf)))
        kn = Fr(kk)
        cr = [kf[1] * Bf[2] - kf[2] * Bf[1], kf[2] * Bf[0] - kf[0] * Bf[2], kf[0] * Bf[1] - kf[1] * Bf[0]]
        V = [kn * Ef[i] + cr[i] for i in range(3)]
        q = sum(v * v for v in V) - sum(kf[i] * Ef[i] for i in range(3)) ** 2
        assert O.chi_photon(kv, E, B, E_S) == pytest.approx(math.sqrt(float(q)) / E_S, rel=1e-11)


def _const_run(E0, **kw):
    d = dict(geometry=2, E_const=(0.0, E0, 0.0), B_const=(0.0, 0.0, E0), dt_over_T=0.01, seed=77, run_id=3)
    d.update(kw)
    return O.run_params(**d)


def test_transport_conversion_law_in_a_constant_crossed_field(bw):
    """Photons counter-propagating through a constant crossed field E = B = E0 have a constant
    chi = 2 k E0 / E_S; the optical depth method converts at step m (counted from emission) with
    probability e^{-lam (m-1)} - e^{-lam m}, lam = alpha E_S T(chi) dt / k; photons along the
    field's propagation direction never convert."""
    tables = O.Tables(O.table_params(n_eta=8, n_y=8, n_E=8, n_s=8), [13.0])
    E_S = O.schwinger_field(1e-6)
    k, E0 = 1000.0, 300.0
    chi = 2 * k * E0 / E_S
    run = _const_run(E0)
    n, steps = 20000, 60
    ph = np.zeros(n, dtype=O.PHOTON_DTYPE)
    ph["energy"] = k
    ph["kx"] = -1.0
    ph["id_mech"] = np.arange(n, dtype=np.uint32)
    pairs, npairs, tally = O.bw_transport(bw, tables, run, ph, step_end=steps)
    T, fl = bw.T_interp(chi)
    assert fl == 0
    lam = ALPHA * E_S * T * (2 * math.pi * 0.01) / k
    assert 0.005 < lam < 0.2
    m = pairs["step"].astype(np.int64)
    assert m.min() >= 1 and m.max() <= steps - 1
    mm = np.arange(1, steps)
    p = np.exp(-lam * (mm - 1)) - np.exp(-lam * mm)
    obs = np.append(np.bincount(m, minlength=steps)[1:], n - npairs).astype(float)
    exp = n * np.append(p, np.exp(-lam * (steps - 1)))
    ss = pytest.importorskip("scipy.stats")
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert ss.chi2.sf(chi2, len(obs) - 1) > 1e-4, chi2
    assert tally[O.PT["N_ENTERED"]] == n and tally[O.PT["N_K_ABOVE"]] == 0
    assert tally[O.PT["N_TESTS"]] == int(m.sum()) + (n - npairs) * (steps - 1)
    np.testing.assert_allclose(pairs["e_minus"].astype(np.float64) + pairs["e_plus"], k, rtol=1e-6)
    # the pairs keep the photon's direction and position; x follows the spectrum at chi (mean 1/2)
    assert np.all(pairs["kx"] == -1.0)
    np.testing.assert_allclose(pairs["x"], -(m * 2 * math.pi * 0.01), rtol=1e-6)
    xr = pairs["e_plus"] / k
    assert abs(xr.mean() - 0.5) < 5 * xr.std() / math.sqrt(len(xr))
    # co-propagating photons, and photons at or below threshold: no pairs
    ph2 = ph.copy()
    ph2["kx"] = 1.0
    _, n2, t2 = O.bw_transport(bw, tables, run, ph2, step_end=steps)
    assert n2 == 0 and t2[O.PT["N_TESTS"]] == n * (steps - 1)
    ph3 = ph[:10].copy()
    ph3["energy"] = 2.0
    _, n3, t3 = O.bw_transport(bw, tables, run, ph3, step_end=steps)
    assert n3 == 0 and t3[O.PT["N_ENTERED"]] == 0


def test_transport_in_the_plane_wave(bw):
    """The 1D a0 = 270 pulse: photons moving with it never convert; photons meeting it head on
    convert with probability 1 - exp(-sum_m W(chi_m) dt), chi_m from the fields along the path
    (summed here in numpy from the oracle's fields and chi), within 5 sigma."""
    tables = O.Tables(O.table_params(n_eta=8, n_y=8, n_E=8, n_s=8), [79.0])
    run = O.run_params(a0=270.0, Z=79.0, charge_state=51.0, dt_over_T=0.02, seed=5)
    E_S = O.schwinger_field(1e-6)
    dt = 2 * math.pi * 0.02
    n, steps, k = 4000, 900, 800.0
    ph = np.zeros(n, dtype=O.PHOTON_DTYPE)
    ph["energy"] = k
    ph["x"] = 60.0
    ph["kx"] = -1.0
    ph["id_mech"] = np.arange(n, dtype=np.uint32)
    _, npairs, _ = O.bw_transport(bw, tables, run, ph, step_end=steps)
    lam = 0.0
    for m in range(1, steps):
        E, B = O.fields(run, 60.0 - m * dt, 0.0, m * dt)
        T, _ = bw.T_interp(O.chi_photon([-k, 0, 0], E, B, E_S))
        lam += ALPHA * E_S * T * dt / k
    p = -math.expm1(-lam)
    assert 0.05 < p < 0.95
    assert abs(npairs - n * p) < 5 * math.sqrt(n * p * (1 - p)), (npairs, n * p)
    ph["kx"] = 1.0
    ph["x"] = -60.0
    assert O.bw_transport(bw, tables, run, ph, step_end=steps)[1] == 0

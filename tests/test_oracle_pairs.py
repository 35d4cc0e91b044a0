"""Pins of the oracle's Bethe-Heitler pair production (Sec. 2.2: implemented like the
bremsstrahlung, Eq. 4 with the pair cross section).

Pinned against: the complete-screening closed form of the pair cross section,
sigma -> 4 alpha r_e^2 {(7/9) [Z^2 (L_rad - f) + Z L'_rad] - (Z^2 + Z)/54} (the 7/9
of the radiation-length cross section) and its x-shape; the unscreened high-energy
Bethe-Heitler DCS where the screening variables are large; the x <-> 1 - x symmetry of
the DCS; the threshold k = 2 m c^2; the tables against direct quadrature; the
conversion law of a photon beam crossing a slab step by step (1 - (1 - P)^N, the
geometric depth distribution) with P from the target density and units written out
here; energy bookkeeping; the geometric edge cases.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1612_07592_gb300 import workloads as W

ALPHA = 7.2973525693e-3
R_E = 2.8179403262e-15


def _closed_form(Z):
    """A = Z^2 (L_rad - f) + Z L'_rad, B = Z^2 + Z with Tsai's L_rad = ln(184.15 Z^-1/3),
    L'_rad = ln(1194 Z^-2/3)."""
    f = O.coulomb_f(Z)
    A = Z * Z * (math.log(184.15 * Z ** (-1 / 3)) - f) + Z * math.log(1194.0 * Z ** (-2 / 3))
    return A, Z * Z + Z


@pytest.mark.parametrize("Z", [13.0, 79.0])
def test_bh_complete_screening_limit(Z):
    A, B = _closed_form(Z)
    sigma_inf = 4.0 * ((7.0 / 9.0) * A - B / 54.0)
    assert abs(O.bh_sigma_direct(Z, 1e7) / sigma_inf - 1.0) < 1e-4
    # screening weakens the cross section at lower energy, monotonically
    s = [O.bh_sigma_direct(Z, k) for k in (1e2, 1e3, 1e4, 1e5, 1e7)]
    assert all(a < b for a, b in zip(s, s[1:]))
    # the DCS in complete screening: 4 {[1 - 4/3 x(1-x)] A - x(1-x) B / 9}
    for x in (0.01, 0.2, 0.5, 0.77, 0.99):
        want = 4.0 * ((1.0 - 4.0 / 3.0 * x * (1 - x)) * A - x * (1 - x) * B / 9.0)
        assert abs(O.bh_dcs_raw(Z, 1e3, x, 1) / want - 1.0) < 1e-4


@pytest.mark.parametrize("Z", [13.0, 79.0])
def test_bh_no_screening_limit(Z):
    """Where the screening variables 100 / (k x (1-x) Z^{1/3}) are large the DCS is the
    unscreened high-energy Bethe-Heitler form 4 [1 - 4/3 x(1-x)] [(Z^2 + Z)(ln(2 k x(1-x)) - 1/2)
    - Z^2 f], to the screening corrections (~2/(0.31 g^2) in the bracket, below 5e-3 of the
    coefficient 4 [1 - 4/3 x(1-x)] (Z^2 + Z) of the logarithm here)."""
    f = O.coulomb_f(Z)
    for k, x in ((3.0, 0.5), (4.0, 0.3), (3.5, 0.7), (2.5, 0.4)):
        g = 100.0 / (k * x * (1 - x) * Z ** (1 / 3))
        assert g > 25.0
        xx = x * (1 - x)
        scale = 4.0 * (1 - 4 / 3 * xx) * (Z * Z + Z)
        want = scale * (math.log(2 * k * xx) - 0.5) - 4.0 * (1 - 4 / 3 * xx) * Z * Z * f
        assert abs(O.bh_dcs_raw(Z, k, x, 0) - want) < 5e-3 * scale, (k, x)


def test_bh_dcs_symmetric_and_threshold():
    rng = np.random.default_rng(3)
    for Z in (13.0, 79.0):
        for k, x in zip(np.exp(rng.uniform(np.log(3.0), np.log(1e6), 50)), rng.uniform(0.0, 1.0, 50)):
            x = min(max(x, 1.0 / k), 1.0 - 1.0 / k)
            a, b = O.bh_dcs_raw(Z, k, x, 0), O.bh_dcs_raw(Z, k, 1.0 - x, 0)
            assert abs(a - b) <= 1e-9 * max(abs(a), 1.0)
        assert O.bh_sigma_direct(Z, 2.0) == 0.0 and O.bh_sigma_direct(Z, 1.5) == 0.0
        assert O.bh_sigma_direct(Z, 20.0) > 0.0


def test_bh_tables_match_direct_quadrature():
    t = O.Tables(O.table_params(n_eta=16, n_y=16, n_E=33, n_s=33, gamma_max=1e6), [13.0, 79.0])
    ks = np.exp(np.linspace(np.log(2.0), np.log(1e6), 33))
    for iz, Z in enumerate((13.0, 79.0)):
        sig = t.export(5, iz)
        assert sig[0] == 0.0
        for i in (3, 10, 20, 32):
            assert abs(sig[i] - O.bh_sigma_direct(Z, ks[i])) <= 1e-10 * sig[i]
        cdf = t.export(6, iz)
        assert np.all(np.diff(cdf, axis=1) >= 0.0) and np.all(cdf[:, 0] == 0.0) and np.all(cdf[:, -1] == 1.0)
        # the interpolant at a grid point is the grid value; k <= 2 has no pairs
        v, above = t.bh_sigma_interp(iz, float(ks[20]))
        assert abs(v / sig[20] - 1.0) < 1e-12 and above == 0
        assert t.bh_sigma_interp(iz, 2.0)[0] == 0.0 and t.bh_sigma_interp(iz, 2e6)[1] == 1


def test_bh_x_distribution_complete_screening():
    """Inverse-CDF samples at k = 1e5 on a quantile grid follow the complete-screening
    x-distribution (closed-form CDF) to the table resolution, and E+ / k is symmetric."""
    Z = 79.0
    t = O.Tables(O.table_params(n_eta=16, n_y=16, n_E=65, n_s=129, gamma_max=1e6), [Z])
    A, B = _closed_form(Z)
    F = lambda x: A * (x - 2 / 3 * x ** 2 + 4 / 9 * x ** 3) - B / 9 * (x ** 2 / 2 - x ** 3 / 3)
    N = 4000
    R = (np.arange(N) + 0.5) / N
    xs = np.array([t.sample_bh_x(0, 1e5, r) for r in R])
    assert np.all(np.diff(xs) >= 0.0) and xs[0] >= 1e-5 and xs[-1] <= 1 - 1e-5
    got = F(xs) / F(1.0)
    assert np.abs(got - R).max() < 3e-3
    assert abs(xs.mean() - 0.5) < 1e-3


def _beam_run(**kw):
    d = dict(a0=0.0, geometry=2, Z=79.0, charge_state=79.0, ne_over_nc=4177.0, slab_x0_m=0.0,
             slab_thick_m=200e-6, dt_over_T=1.0, enable_ncs=0, seed=21, iz=0)
    d.update(kw)
    return O.run_params(**d)


def test_pair_conversion_law_of_a_beam():
    """A 5 GeV photon beam normally incident on 200 um of solid Au: each step inside is a
    Bernoulli trial with P = 1 - exp(-n_i sigma c dt), n_i = n_e / Z* with n_c = pi / (r_e
    lambda^2), sigma in alpha r_e^2; the converted fraction is 1 - (1 - P)^N_in and the
    conversion depth geometric."""
    t = O.Tables(O.table_params(n_eta=16, n_y=16, n_E=65, n_s=65, gamma_max=1e6), [79.0])
    r = _beam_run()
    k = 1e4
    n = 40000
    ph = np.zeros(n, dtype=W.PHOTON_RECORD)
    kl = 2 * math.pi / 1e-6
    ph["x"] = -0.5
    ph["energy"] = k
    ph["kx"] = 1.0
    ph["step"] = 0
    ph["id_mech"] = np.arange(n, dtype=np.uint32)
    pairs, npairs, tally = O.pair_transport(t, r, ph, step_end=1000)
    dt = 2 * math.pi
    x1 = 200e-6 * kl
    m = np.arange(1, 1000)
    inside = (np.float64(-0.5) + m * dt >= 0.0) & (np.float64(-0.5) + m * dt <= x1)
    n_in = int(inside.sum())
    assert n_in == 200
    n_i = 4177.0 * math.pi / (R_E * 1e-12) / 79.0
    sigma = t.bh_sigma_interp(0, k)[0]
    assert abs(sigma / O.bh_sigma_direct(79.0, k) - 1) < 1e-3
    P = -math.expm1(-n_i * ALPHA * R_E ** 2 * sigma * 1e-6)
    p_conv = 1.0 - (1.0 - P) ** n_in
    assert tally[O.PT["N_ENTERED"]] == n
    sd = math.sqrt(n * p_conv * (1 - p_conv))
    assert abs(npairs - n * p_conv) < 5 * sd, (npairs, n * p_conv)
    # depth: first step inside is m0; conversion at m0 + j with probability (1 - P)^j P
    m0 = int(m[inside][0])
    j = pairs["step"].astype(np.int64) - m0
    assert j.min() >= 0 and j.max() < n_in
    jj = np.arange(n_in)
    pj = (1 - P) ** jj * P / p_conv
    mean = float((jj * pj).sum())
    var = float(((jj - mean) ** 2 * pj).sum())
    assert abs(j.mean() - mean) < 5 * math.sqrt(var / len(j))
    # positions: the photon's position at the conversion step
    np.testing.assert_allclose(pairs["x"], (-0.5 + pairs["step"] * dt).astype(np.float32), rtol=1e-6)


def test_pair_bookkeeping_and_streams():
    t = O.Tables(O.table_params(n_eta=16, n_y=16, n_E=33, n_s=33, gamma_max=1e6), [79.0])
    r = _beam_run(slab_thick_m=2e-3)
    kl = 2 * math.pi / 1e-6
    ph = W.synthetic_photons(20000, 5, (0.0, 2e-3 * kl), (1.0, 1e5), (0, 500))
    pairs, npairs, tally = O.pair_transport(t, r, ph, step_end=3000)
    assert npairs > 1000
    src = ph[pairs["photon"]]
    np.testing.assert_array_equal(pairs["id_mech"], src["id_mech"])
    assert np.all(src["energy"] > 2.0)
    np.testing.assert_allclose(pairs["e_minus"].astype(np.float64) + pairs["e_plus"], src["energy"], rtol=1e-6)
    assert np.all(pairs["e_plus"] >= 1.0 - 1e-4) and np.all(pairs["e_minus"] >= 1.0 - 1e-4)
    assert np.all(pairs["step"] > src["step"]) and np.all(pairs["step"] < 3000)
    assert abs(O.fixed_to_float(tally, O.PT["E_PAIRS"]) / src["energy"].astype(np.float64).sum() - 1) < 1e-6
    # each photon converts at most once, inside the slab
    assert len(np.unique(pairs["photon"])) == npairs
    assert np.all(pairs["x"] >= 0.0) and np.all(pairs["x"] <= 2e-3 * kl * (1 + 1e-6))
    # independent streams: the same photon emitted at another step, or by the other mechanism,
    # converts at an independent depth
    base = np.zeros(4000, dtype=W.PHOTON_RECORD)
    base["x"] = 1.0
    base["energy"] = 1e4
    base["kx"] = 1.0
    base["id_mech"] = 7
    a = base.copy()
    a["step"] = np.arange(4000)
    b = a.copy()
    b["id_mech"] = 7 | (1 << 31)
    pa, na, _ = O.pair_transport(t, r, a, step_end=10000)
    pb, nb, _ = O.pair_transport(t, r, b, step_end=10000)
    da = pa["step"] - a["step"][pa["photon"]]
    assert len(np.unique(da)) > 100
    common = np.intersect1d(pa["photon"], pb["photon"])
    same = (pa["step"][np.searchsorted(pa["photon"], common)] == pb["step"][np.searchsorted(pb["photon"], common)])
    assert same.mean() < 0.05


def test_pair_transport_edges():
    t = O.Tables(O.table_params(n_eta=16, n_y=16, n_E=33, n_s=33, gamma_max=1e6), [79.0])
    kl = 2 * math.pi / 1e-6
    r = _beam_run(slab_thick_m=1e-3)
    x1 = 1e-3 * kl
    ph = np.zeros(6, dtype=W.PHOTON_RECORD)
    ph["energy"] = [1e4, 2.0, 1e4, 1e4, 1e4, 1e4]
    ph["x"] = [-1.0, 10.0, -1.0, x1 + 1.0, 10.0, 10.0]
    ph["kx"] = [1.0, 1.0, -1.0, 1.0, 1.0, 1.0]
    ph["step"] = [0, 0, 0, 0, 98, 99]
    ph["id_mech"] = np.arange(6)
    pairs, n, tally = O.pair_transport(t, r, ph, step_end=100)
    # photon 1: k = 2 (threshold); 2: outside moving away; 3: beyond the rear face;
    # 5: emitted at the last step (never tested); 4: one test
    assert set(pairs["photon"].tolist()) <= {0, 4}
    assert tally[O.PT["N_ENTERED"]] == 2
    # 2D: a photon leaving the strip |y| <= y_half sideways stops being tested
    r2 = _beam_run(slab_thick_m=1e-2, geometry=1, y_half_m=3e-6, a0=0.0)
    yh = 3e-6 * kl
    q = np.zeros(3000, dtype=W.PHOTON_RECORD)
    q["x"] = 1.0
    q["y"] = 0.0
    q["energy"] = 1e5
    q["kx"] = math.cos(0.01)
    q["ky"] = math.sin(0.01)
    q["id_mech"] = np.arange(3000)
    p2, n2, t2 = O.pair_transport(t, r2, q, step_end=100000)
    dt = 2 * math.pi
    last = int(np.floor(yh / (math.sin(0.01) * dt) + 1e-9))       # last step with |y| <= y_half
    assert n2 > 0 and p2["step"].max() <= last and np.all(np.abs(p2["y"]) <= yh * (1 + 1e-6))


def test_pair_free_path_conversion_law():
    """The free-path method (one geometric draw per crossing) gives the beam the same law: the
    converted fraction 1 - (1 - P)^N and geometric depths, with one draw per photon."""
    t = O.Tables(O.table_params(n_eta=16, n_y=16, n_E=65, n_s=65, gamma_max=1e6), [79.0])
    r = _beam_run()
    k, n = 1e4, 40000
    ph = np.zeros(n, dtype=W.PHOTON_RECORD)
    ph["x"] = -0.5
    ph["energy"] = k
    ph["kx"] = 1.0
    ph["id_mech"] = np.arange(n, dtype=np.uint32)
    pairs, npairs, tally = O.pair_transport(t, r, ph, step_end=1000, method=O.PAIR_FREE_PATH)
    n_i = 4177.0 * math.pi / (R_E * 1e-12) / 79.0
    P = -math.expm1(-n_i * ALPHA * R_E ** 2 * t.bh_sigma_interp(0, k)[0] * 1e-6)
    n_in = 200
    p_conv = 1.0 - (1.0 - P) ** n_in
    assert tally[O.PT["N_TESTS"]] == n == tally[O.PT["N_ENTERED"]]
    assert abs(npairs - n * p_conv) < 5 * math.sqrt(n * p_conv * (1 - p_conv))
    m0 = 1                                              # first step inside: -0.5 + dt >= 0
    j = pairs["step"].astype(np.int64) - m0
    assert j.min() >= 0 and j.max() < n_in
    jj = np.arange(n_in)
    pj = (1 - P) ** jj * P / p_conv
    mean = float((jj * pj).sum())
    var = float(((jj - mean) ** 2 * pj).sum())
    assert abs(j.mean() - mean) < 5 * math.sqrt(var / len(j))


def test_pair_free_path_equals_direct_in_law():
    """On synthetic photons through 2 mm of Au both methods convert the same number of photons,
    at the same mean depth after entry and with the same positron-energy fractions, within the
    statistics (the realisations differ: other draws)."""
    t = O.Tables(O.table_params(n_eta=16, n_y=16, n_E=33, n_s=33, gamma_max=1e6), [79.0])
    r = _beam_run(slab_thick_m=2e-3)
    kl = 2 * math.pi / 1e-6
    ph = W.synthetic_photons(40000, 6, (0.0, 2e-3 * kl), (3.0, 1e5), (0, 500))
    res = {}
    for m in (O.PAIR_DIRECT, O.PAIR_FREE_PATH):
        pairs, n, tally = O.pair_transport(t, r, ph, step_end=3000, method=m)
        depth = pairs["step"].astype(np.int64) - ph["step"][pairs["photon"]].astype(np.int64)
        res[m] = (n, depth, pairs["e_plus"] / (pairs["e_plus"] + pairs["e_minus"]), tally)
    (n1, d1, x1, t1), (n2, d2, x2, t2) = res[O.PAIR_DIRECT], res[O.PAIR_FREE_PATH]
    assert n1 > 3000 and abs(n1 - n2) < 5 * math.sqrt(n1 + n2)
    assert abs(d1.mean() - d2.mean()) < 5 * math.sqrt(d1.var() / len(d1) + d2.var() / len(d2))
    assert abs(x1.mean() - x2.mean()) < 5 * math.sqrt(x1.var() / len(x1) + x2.var() / len(x2))
    assert t1[O.PT["N_ENTERED"]] == t2[O.PT["N_ENTERED"]]
    assert t2[O.PT["N_TESTS"]] <= t2[O.PT["N_ENTERED"]] < t1[O.PT["N_TESTS"]]


@pytest.mark.parametrize("method", [O.PAIR_DIRECT, O.PAIR_FREE_PATH])
def test_pair_depth_histogram_is_geometric(method):
    """With P ~ 0.1 per step (Au at 50x solid density, 10 um steps) the number of steps inside
    before the conversion follows P (1 - P)^j for j < N_in and the rest pass through: a
    chi-square over the N_in + 1 outcomes, by either method (a free path that rounded the
    geometric count up or down by one step would fail it)."""
    scipy_stats = pytest.importorskip("scipy.stats")
    t = O.Tables(O.table_params(n_eta=16, n_y=16, n_E=65, n_s=65, gamma_max=1e6), [79.0])
    r = _beam_run(ne_over_nc=4177.0 * 50, dt_over_T=10.0, seed=33)
    k, n = 1e4, 40000
    ph = np.zeros(n, dtype=W.PHOTON_RECORD)
    ph["x"] = -0.5
    ph["energy"] = k
    ph["kx"] = 1.0
    ph["id_mech"] = np.arange(n, dtype=np.uint32)
    pairs, npairs, tally = O.pair_transport(t, r, ph, step_end=1000, method=method)
    n_i = 50 * 4177.0 * math.pi / (R_E * 1e-12) / 79.0
    P = -math.expm1(-n_i * ALPHA * R_E ** 2 * t.bh_sigma_interp(0, k)[0] * 10e-6)
    assert 0.05 < P < 0.2
    n_in = 20                                           # steps 1..20 at x = -0.5 + 10 * 2 pi m < 200 um
    j = pairs["step"].astype(np.int64) - 1
    assert j.min() >= 0 and j.max() < n_in
    obs = np.append(np.bincount(j, minlength=n_in), n - npairs).astype(float)
    exp = n * np.append(P * (1 - P) ** np.arange(n_in), (1 - P) ** n_in)
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert scipy_stats.chi2.sf(chi2, n_in) > 1e-4, chi2

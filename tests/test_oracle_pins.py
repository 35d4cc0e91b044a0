"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, library routines (scipy.special), closed forms, exact
rational arithmetic, brute-force quadrature, or numbers printed in the paper.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp
import scipy.stats as st_
from scipy.optimize import brentq

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA = 7.2973525693e-3
RE = 2.8179403262e-15
NA = 6.02214076e23


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- Philox ----
def test_philox_known_answers():
    for r in _golden("philox_kat.txt"):
        v = [int(t, 16) for t in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


# ----------------------------------------------------------------- units ----
def test_units_and_paper_densities():
    E_S = O.schwinger_field(1e-6)
    assert abs(E_S / 4.12148e5 - 1) < 2e-6          # m c^2 / (hbar omega) at 1 um
    n_c = O.critical_density(1e-6)
    assert abs(n_c / 1.11485e27 - 1) < 1e-5
    g = {r[0]: float(r[1]) for r in _golden("paper_numbers.txt")}
    # Sec. 3: fully ionised Al (2.70 g/cc) and Au (19.3 g/cc) give ~711 and ~4177 n_c
    for Z, A, rho, key in ((13, 26.98, 2.70, "ne_over_nc_Al_full_ionisation"),
                           (79, 196.97, 19.3, "ne_over_nc_Au_full_ionisation")):
        ne = Z * rho * 1e3 / (A * 1e-3) * NA           # m^-3
        assert abs(ne / n_c / g[key] - 1) < 0.02


# --------------------------------------------------------------- Bessel ----
@pytest.mark.parametrize("x", [1e-6, 1e-3, 0.05, 0.7, 3.0, 20.0, 90.0])
def test_bessel_vs_scipy(x):
    for nu in (1.0 / 3.0, 2.0 / 3.0, 5.0 / 3.0):
        assert abs(O.bessel_k(nu, x) / sp.kv(nu, x) - 1) < 1e-12
    # int_x^inf K_{5/3} = 2 K_{2/3}(x) - int_x^inf K_{1/3}  (Bessel recurrence)
    ik13 = si.quad(lambda t: sp.kv(1.0 / 3.0, t), x, np.inf, epsabs=0, epsrel=1e-13, limit=400)[0]
    ref = 2.0 * sp.kv(2.0 / 3.0, x) - ik13
    assert abs(O.int_k53(x) / ref - 1) < 1e-10


# ------------------------------------------------ NCS: classical limits ----
def test_classical_spectrum_integrals():
    # int_0^inf (int_y^inf K53) dy = int_0^inf t K53(t) dt = 5 pi / 3  (h at eta -> 0)
    t = O.Tables(O.table_params(n_eta=2, n_y=16, n_E=2, n_s=2), [13.0])
    assert abs(t.classical_total() / (5 * math.pi / 3) - 1) < 1e-11
    assert abs(O.ncs_h_direct(1e-7) / (5 * math.pi / 3) - 1) < 1e-5


def test_larmor_limit():
    # radiated power int (hbar omega) dN -> (2/3) alpha m c^2 (c / lambdabar_C) eta^2:
    # with the rate prefactor sqrt(3) alpha/(2 pi) this is g = 3 sqrt3/(2 pi) int F dchi / eta^2 -> 1
    for eta in (1e-6, 1e-4):
        g = 3 * math.sqrt(3) / (2 * math.pi) * O.ncs_power_integral(eta) / eta ** 2
        assert abs(g - 1) < 1e-3
        # small-eta series of the quantum power ratio: 1 - (55 sqrt3 / 16) eta + 48 eta^2 + O(eta^3)
        assert abs(g - (1 - 55 * math.sqrt(3) / 16 * eta + 48 * eta * eta)) < 1e3 * eta ** 3 + 1e-10


@pytest.mark.parametrize("eta", [0.01, 0.1, 1.0, 10.0])
def test_power_vs_published_fit(eta):
    # g(eta) ~ [1 + 4.8 (1+eta) ln(1+1.7 eta) + 2.44 eta^2]^(-2/3) (Baier-Katkov fit), a few %
    g = 3 * math.sqrt(3) / (2 * math.pi) * O.ncs_power_integral(eta) / eta ** 2
    fit = (1 + 4.8 * (1 + eta) * math.log(1 + 1.7 * eta) + 2.44 * eta * eta) ** (-2.0 / 3.0)
    assert abs(g / fit - 1) < 0.02


def test_ncs_F_vs_scipy_pointwise():
    for eta in (1e-3, 0.5, 20.0):
        for frac in (1e-4, 0.1, 0.3, 0.49):
            chi = frac * eta
            y = 4 * chi / (3 * eta * (eta - 2 * chi))
            if y > 60:          # F ~ exp(-y): nothing left to compare
                continue
            d = 2 * chi / eta
            ik53 = 2 * sp.kv(2 / 3, y) - si.quad(lambda s: sp.kv(1 / 3, s), y, np.inf,
                                                 epsabs=0, epsrel=1e-13, limit=400)[0]
            ref = d * d * y * sp.kv(2 / 3, y) + (1 - d) * y * ik53
            assert abs(O.ncs_F(eta, chi) / ref - 1) < 1e-10


# ----------------------------------------- NCS table: brute-force quadrature --
def _cum_simpson_segments(lny_nodes_per_seg, f):
    """Cumulative Simpson over concatenated uniform segments; returns values at segment ends."""
    out = [0.0]
    for seg in lny_nodes_per_seg:
        v = f(seg)
        out.append(out[-1] + si.simpson(v, x=seg))
    return np.array(out[1:])


def _ik53_on(y):
    """int_y^inf K_{5/3} via 2 K_{2/3}(y) - int_y^inf K_{1/3}, the latter by cumulative Simpson."""
    top = 250.0
    lt = np.linspace(math.log(float(y.min())), math.log(top), 400001)
    tt = np.exp(lt)
    integ = tt * sp.kv(1 / 3, tt)
    cum = si.cumulative_simpson(integ[::-1], x=-lt[::-1], initial=0.0)[::-1]   # int_t^top
    ik13 = np.interp(np.log(y), lt, cum)
    return 2 * sp.kv(2 / 3, y) - ik13


def test_ncs_table_vs_brute_force():
    p = O.table_params(n_eta=3, n_y=8, eta_min=1e-3, eta_max=30.0, y_min=1e-6, y_max=1e2, n_E=2, n_s=2)
    t = O.Tables(p, [13.0])
    cdf = t.export(1)
    h = t.export(0)
    ygrid = np.exp(np.linspace(math.log(p.y_min), math.log(p.y_max), p.n_y))
    ylo = p.y_min * 1e-8
    for i, eta in enumerate(np.exp(np.linspace(math.log(p.eta_min), math.log(p.eta_max), p.n_eta))):
        def f(lny):
            y = np.exp(lny)
            d = 3 * eta * y / (2 + 3 * eta * y)
            F = d * d * y * sp.kv(2 / 3, y) + (1 - d) * y * _ik53_on(y)
            return F * 2 / (2 + 3 * eta * y)
        segs = [np.linspace(math.log(ylo), math.log(p.y_min), 4001)]
        for j in range(1, p.n_y):
            segs.append(np.linspace(math.log(ygrid[j - 1]), math.log(ygrid[j]), 2001))
        cum = _cum_simpson_segments(segs, f)
        cum = cum + 3.0 * f(np.array([math.log(ylo)]))[0]     # y^(1/3) tail below ylo
        assert abs(h[i] / cum[-1] - 1) < 1e-9
        np.testing.assert_allclose(cdf[i], cum / cum[-1], rtol=1e-9, atol=1e-12)


# --------------------------------------------------------- bremsstrahlung ----
def _closed_complete(Z, y):
    # complete screening: phi1(0) = 20.863 (= 4 ln 184.15 to 5 digits), psi1(0) = 28.340
    # (= 4 ln 1194), phi1 - phi2 = psi1 - psi2 = 2/3
    assert abs(4 * math.log(184.15) / 20.863 - 1) < 1e-5 and abs(4 * math.log(1194) / 28.340 - 1) < 1e-5
    Lrad = 20.863 / 4 - math.log(Z) / 3
    Lp = 28.340 / 4 - 2 * math.log(Z) / 3
    f = O.coulomb_f(Z)
    return 4 / y * ((4 / 3 - 4 / 3 * y + y * y) * (Z * Z * (Lrad - f) + Z * Lp) + (1 - y) * (Z * Z + Z) / 9)


def test_coulomb_correction_values():
    assert abs(O.coulomb_f(13.0) - 0.010735) < 2e-6
    assert abs(O.coulomb_f(79.0) - 0.31280) < 2e-5


@pytest.mark.parametrize("Z", [13.0, 79.0])
def test_brems_complete_screening_closed_form(Z):
    for y in (1e-4, 0.01, 0.3, 0.77, 0.999):
        v = O.brems_dcs_raw(Z, 1e3, y, 1)
        assert abs(v / _closed_complete(Z, y) - 1) < 1e-12


@pytest.mark.parametrize("Z", [13.0, 79.0])
def test_brems_sigma_high_energy_limit(Z):
    g = 1e6
    ycut = 1.0 / g
    Lrad = math.log(184.15 * Z ** (-1 / 3))
    Lp = math.log(1194 * Z ** (-2 / 3))
    f = O.coulomb_f(Z)
    A1 = 4 / 3 * math.log(1 / ycut) - 4 / 3 * (1 - ycut) + (1 - ycut ** 2) / 2
    A2 = math.log(1 / ycut) - (1 - ycut)
    closed = 4 * (A1 * (Z * Z * (Lrad - f) + Z * Lp) + A2 * (Z * Z + Z) / 9)
    s = O.brems_sigma_direct(Z, g, 1.0)
    assert abs(s / closed - 1) < 1e-3


def test_brems_Z_scaling_paper():
    # Sec. 2.1: sigma_b ~ Z^2 alpha r_e^2 (6241 = 79^2 for Au; the "139" printed for Al reads 169 = 13^2)
    g = {r[0]: float(r[1]) for r in _golden("paper_numbers.txt")}
    assert g["sigma_b_Au_over_alpha_re2"] == 79 ** 2
    # the Z^2 bracket dominates: sigma(Au)/sigma(Al) lies between (79/13)^2 * 0.5 and (79/13)^2
    r = O.brems_sigma_direct(79.0, 1e3, 1.0) / O.brems_sigma_direct(13.0, 1e3, 1.0)
    assert 0.5 * (79 / 13) ** 2 < r < (79 / 13) ** 2


def test_radiation_length_pdg():
    for Z, A, X0 in _golden("radiation_length.txt"):
        Z, A, X0 = float(Z), float(A), float(X0)
        # int_0^1 y dsigma/dy dy under complete screening, without the small (Z^2+Z)/18 term (PDG form)
        ys = np.linspace(1e-9, 1 - 1e-9, 200001)
        v = np.array([O.brems_dcs_raw(Z, 1e12, float(y), 1) for y in ys[::50]])
        integ = si.simpson(ys[::50] * v, x=ys[::50])
        integ -= 4 * (Z * Z + Z) / 18
        inv_x0 = ALPHA * RE ** 2 * integ * NA / A * 1e-4     # cm^2/g  (r_e in m -> cm^2)
        inv_x0 = ALPHA * (RE * 100) ** 2 * integ * NA / A
        assert abs(1 / inv_x0 / X0 - 1) < 0.01


@pytest.mark.parametrize("Z", [13.0, 79.0])
def test_brems_table_vs_brute_force(Z):
    p = O.table_params(n_eta=2, n_y=2, n_E=3, n_s=8, gamma_min=3.0, gamma_max=1e5)
    t = O.Tables(p, [Z])
    sig = t.export(3)
    cdf = t.export(4)
    dcs = np.vectorize(lambda g, y: O.brems_dcs_raw(Z, g, y, 0))
    for i, g in enumerate(np.exp(np.linspace(math.log(p.gamma_min), math.log(p.gamma_max), p.n_E))):
        ycut, ymax = 1.0 / g, 1 - 1.0 / g
        L = math.log(ymax / ycut)
        yof = lambda s: ycut * np.exp(s * L)
        raw = lambda s: dcs(g, yof(s))
        cum = [0.0]
        for j in range(1, p.n_s):
            a, b = (j - 1) / (p.n_s - 1), j / (p.n_s - 1)
            edges = [a, b]
            if raw(np.array(a)) * raw(np.array(b)) < 0:           # clamp kink (dcs < 0 near the tip)
                edges = [a, brentq(lambda s: float(raw(np.array(s))), a, b, xtol=1e-15), b]
            tot = 0.0
            for lo, hi in zip(edges[:-1], edges[1:]):
                # the integrand falls steeply at the kinematic tip: adaptive QUADPACK per piece
                fs = lambda s: max(float(raw(np.array(s))), 0.0) * float(yof(s)) * L
                tot += si.quad(fs, lo, hi, epsabs=0, epsrel=1e-13, limit=500)[0]
            cum.append(cum[-1] + tot)
        cum = np.array(cum)
        assert abs(sig[i] / cum[-1] - 1) < 1e-9
        np.testing.assert_allclose(cdf[i], cum / cum[-1], rtol=1e-9, atol=1e-12)


# --------------------------------------------------------- eta invariant ----
def _eta2_exact(u, E, B):
    u = [Fraction(v) for v in u]
    E = [Fraction(v) for v in E]
    B = [Fraction(v) for v in B]
    g2 = 1 + sum(v * v for v in u)
    # gamma is irrational: use (gamma E + u x B)^2 - (u.E)^2 expanded so that gamma appears linearly
    uxB = [u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2], u[0] * B[1] - u[1] * B[0]]
    E2 = sum(v * v for v in E)
    cross = sum(a * b for a, b in zip(E, uxB))
    uxB2 = sum(v * v for v in uxB)
    uE = sum(a * b for a, b in zip(u, E))
    return g2 * E2 + uxB2 - uE * uE, 2 * cross     # value = first + gamma * second


def test_eta_identity_exact():
    rng = np.random.default_rng(1)
    E_S = 4.12148e5
    cases = []
    for _ in range(40):
        cases.append((rng.normal(size=3) * 10 ** rng.uniform(-2, 4), rng.normal(size=3) * 100, rng.normal(size=3) * 100))
    # electrons riding a plane wave along x: gamma E + u x B nearly cancels
    for a, ux in ((270.0, 3.6e4), (855.0, 3.6e5), (27.0, 364.0)):
        uy = math.sqrt(2 * ux)
        E = np.array([0.0, a, 0.0])
        B = np.array([0.0, 0.0, a])
        cases.append((np.array([ux, uy, 0.3]), E, B))
        cases.append((np.array([ux, uy, 0.0]), E * 1.01, B))
    for u, E, B in cases:
        A, Bc = _eta2_exact(u, E, B)
        g = math.sqrt(float(1 + sum(Fraction(v) ** 2 for v in u)))
        # gamma to ~35 digits: refine the float with one Newton step in rationals
        g2 = 1 + sum(Fraction(v) ** 2 for v in u)
        gq = Fraction(g)
        gq = (gq + g2 / gq) / 2
        gq = (gq + g2 / gq) / 2
        ref2 = A + gq * Bc
        ref = math.sqrt(max(float(ref2), 0.0)) / E_S
        got = O.eta(u, E, B, E_S)
        assert abs(got - ref) <= 1e-13 * max(ref, 1e-300) + 1e-300, (u, E, B, got, ref)


# -------------------------------------------------------------- pusher ----
def test_boris_constant_B_rotation():
    B = np.array([0.0, 0.0, 3.0])
    u = np.array([5.0, 0.0, 0.7])
    dt = 0.05
    g = math.sqrt(1 + u @ u)
    ang = 2 * math.atan(3.0 * dt / (2 * g))        # exact Boris rotation angle per step
    v = u.copy()
    n = 1000
    for _ in range(n):
        v = O.boris(v, np.zeros(3), B, dt)
    # charge -e in B along +z rotates u counter-clockwise: du/dt = -u x B / gamma
    phi = n * ang
    ref = np.array([5 * math.cos(phi), 5 * math.sin(phi), 0.7])
    np.testing.assert_allclose(v, ref, atol=1e-10)


def test_boris_constant_E_exact():
    E = np.array([0.4, -1.0, 2.0])
    u0 = np.array([1.0, 2.0, -3.0])
    v = u0.copy()
    for _ in range(500):
        v = O.boris(v, E, np.zeros(3), 0.01)
    np.testing.assert_allclose(v, u0 - 500 * 0.01 * E, rtol=0, atol=1e-11)


def _plane_wave_errors(a0, dto):
    """Max errors of u_y - A_y(phi) and (gamma - u_x) - 1 after 9 periods from rest."""
    r = O.run_params(a0=a0, enable_ncs=0, enable_brems=0, flat_s=3 * 3.33564095e-15, ramp_periods=1.0,
                     dt_over_T=dto)
    t = O.Tables(O.table_params(n_eta=2, n_y=4, n_E=2, n_s=2), [13.0])
    ids = np.arange(8)
    st = O.init(t, r, ids)
    x0 = st[:, 0].copy()
    n = int(round(9 / dto))
    dt = 2 * math.pi * dto
    O.run(t, r, ids, st, 0, n, capacity=16)
    e_perp = e_lf = 0.0
    pr, pf = 2 * math.pi, 2 * math.pi * 3 * 3.33564095e-15 * 299792458.0 / 1e-6
    for k in range(len(ids)):
        x, ux, uy, uz = st[k, 0], st[k, 2], st[k, 3], st[k, 4]
        g = math.sqrt(1 + ux * ux + uy * uy + uz * uz)
        phi = (n - 0.5) * dt - (x - 0.5 * dt * ux / g)      # u lives at the half step
        if phi < pr:
            env = math.sin(0.5 * math.pi * phi / pr) ** 2
        elif phi <= pr + pf:
            env = 1.0
        else:
            env = math.cos(0.5 * math.pi * (phi - pr - pf) / pr) ** 2
        # the vector potential of the LP pulse: A_y = a0 g(phi) sin(phi)
        e_perp = max(e_perp, abs(uy - a0 * env * math.sin(phi)))
        e_lf = max(e_lf, abs((g - ux) - 1.0))
        assert x > x0[k]
    return e_perp, e_lf


def test_plane_wave_orbit_from_rest():
    # canonical momentum: an electron starting at rest has u_perp = A_perp(phi) and gamma - u_x = 1;
    # the Boris/leapfrog scheme reproduces both with second-order error in dt
    a0 = 5.0
    p1, l1 = _plane_wave_errors(a0, 0.01)
    p2, l2 = _plane_wave_errors(a0, 0.005)
    assert p1 < 2e-3 * a0 and l1 < 5e-3
    assert 3.5 < l1 / l2 < 4.5
    assert p2 < 0.5 * p1


# ---------------------------------------------------------- sampling ----
def test_ncs_sampler_inverts_table():
    p = O.table_params(n_eta=16, n_y=64)
    t = O.Tables(p, [13.0])
    cdf = t.export(1)
    ygrid = np.exp(np.linspace(math.log(p.y_min), math.log(p.y_max), p.n_y))
    eta_i = math.exp(math.log(p.eta_min) + 5 * (math.log(p.eta_max) - math.log(p.eta_min)) / (p.n_eta - 1))
    for j in (3, 20, 40):
        d, below = t.sample_ncs_delta(eta_i * (1 + 1e-14), float(cdf[5, j]) * (1 + 1e-15))
        y = 2 * d / (3 * eta_i * (1 - d))
        assert abs(y / ygrid[j] - 1) < 1e-9
    # tail: CDF ~ y^(1/3) below the first node
    R = cdf[5, 0] / 8.0
    d, _ = t.sample_ncs_delta(eta_i * (1 + 1e-14), float(R))
    y = 2 * d / (3 * eta_i * (1 - d))
    assert abs(y / (p.y_min / 512.0) - 1) < 1e-6
    # classical row below eta_min
    d, below = t.sample_ncs_delta(1e-6, 0.5)
    assert below == 1 and 0 < d < 1e-4


def test_ncs_sampled_spectrum_matches_quadrature():
    # sampled photon-energy fractions follow the direct-quadrature CDF of F/chi
    p = O.table_params(n_eta=64, n_y=128)
    t = O.Tables(p, [13.0])
    eta = 0.37
    rng = np.random.default_rng(7)
    R = rng.random(20000)
    ds = np.array([t.sample_ncs_delta(eta, float(r))[0] for r in R])
    h = O.ncs_h_direct(eta)
    for dq in (1e-3, 1e-2, 0.1, 0.3, 0.6):
        yq = 2 * dq / (3 * eta * (1 - dq))
        # CDF at yq by direct quadrature in ln y
        f = lambda ly: O.ncs_F(eta, 0.5 * eta * (3 * eta * math.exp(ly) / (2 + 3 * eta * math.exp(ly)))) \
            * 2 / (2 + 3 * eta * math.exp(ly))
        c = si.quad(f, math.log(1e-14), math.log(yq), epsrel=1e-10, limit=400)[0] / h
        emp = np.mean(ds <= dq)
        assert abs(emp - c) < 4 * math.sqrt(c * (1 - c) / len(R)) + 2e-3


def test_brems_sampler_range_and_inversion():
    p = O.table_params(n_eta=2, n_y=2, n_E=32, n_s=64)
    t = O.Tables(p, [79.0])
    for g in (2.5, 40.0, 3e3):
        lo = t.sample_brems_y(0, g, 1e-12)
        hi = t.sample_brems_y(0, g, 1 - 1e-12)
        assert abs(lo * g - 1.0) < 1e-6                   # photon energy >= m c^2 (Sec. 3 cut)
        assert hi <= 1 - 1 / g + 1e-12 and hi > 0.5 * (1 - 1 / g)
        ys = [t.sample_brems_y(0, g, r) for r in np.linspace(0.01, 0.99, 50)]
        assert np.all(np.diff(ys) > 0)


# --------------------------------------------------------------- runs ----
def test_tau_initial_is_exponential():
    t = O.Tables(O.table_params(n_eta=2, n_y=4, n_E=2, n_s=2), [13.0])
    st = O.init(t, O.run_params(seed=11), np.arange(20000))
    tau = st[:, 5]
    from scipy.stats import kstest
    assert kstest(tau, "expon").pvalue > 1e-3


def test_maxwell_juttner_mean_energy():
    t = O.Tables(O.table_params(n_eta=2, n_y=4, n_E=2, n_s=2), [79.0])
    theta = 1.0 / 0.51099895
    st = O.init(t, O.run_params(init_dist=1, T_mev=1.0, seed=3), np.arange(40000))
    g = np.sqrt(1 + (st[:, 2:5] ** 2).sum(1))
    mean = sp.kv(1, 1 / theta) / sp.kv(2, 1 / theta) + 3 * theta
    assert abs(g.mean() - mean) < 4 * g.std() / math.sqrt(len(g))
    # isotropy
    assert abs(st[:, 2].mean()) < 4 * st[:, 2].std() / math.sqrt(len(g))


def test_brems_first_event_is_geometric():
    # no field, thick slab: each step is an independent trial with P = 1 - exp(-n sigma v dt)
    p = O.table_params(n_eta=2, n_y=4, n_E=64, n_s=32)
    t = O.Tables(p, [79.0])
    r = O.run_params(geometry=2, Z=79.0, charge_state=51.0, ne_over_nc=2e6, slab_x0_m=-1.0, slab_thick_m=2.0,
                     init_dist=2, beam_gamma=2e3, enable_ncs=0, seed=5)
    ids = np.arange(3000)
    st = O.init(t, r, ids)
    ph, n, hist, tally = O.run(t, r, ids, st, 0, 400, capacity=1 << 16)
    first = {}
    for rec in ph:
        pid = int(rec["id_mech"]) & 0x7FFFFFFF
        first.setdefault(pid, int(rec["step"]))
    sig, _ = t.sigma_interp(0, 2e3)
    E_S = O.schwinger_field(1e-6)
    n_i = 2e6 * O.critical_density(1e-6) / 51.0
    dt = 2 * math.pi * 0.01
    xb = n_i * ALPHA * RE * RE * dt * 1e-6 / (2 * math.pi) * sig * math.sqrt(1 - 1 / 2e3 ** 2)
    P = -math.expm1(-xb)
    waits = np.array([first.get(i, 400) for i in ids])
    # P(first event at step k) = (1-P)^k P; censored at 400
    assert 0.003 < P < 0.05
    frac_none = np.mean(waits == 400)
    assert abs(frac_none - (1 - P) ** 400) < 4 * math.sqrt((1 - P) ** 400 / len(ids)) + 0.01
    k = waits[waits < 400]
    mean_trunc = sum(kk * (1 - P) ** kk * P for kk in range(400)) / (1 - (1 - P) ** 400)
    assert abs(k.mean() / mean_trunc - 1) < 0.05


def test_brems_probability_carries_beta():
    """Eq. 4's x_b = n_i sigma_Z(gamma) beta c dt: at gamma = 2.5 (beta = 0.917) the first-event
    law of the direct test separates beta from its omission.  One event takes gamma below
    1 + photon_min, so each electron's first event is its only one; fields off, thick slab."""
    t = O.Tables(O.table_params(n_eta=2, n_y=4, n_E=64, n_s=32), [79.0])
    g = 2.5
    r = O.run_params(geometry=2, Z=79.0, charge_state=51.0, ne_over_nc=1e8, slab_x0_m=-1.0, slab_thick_m=2.0,
                     init_dist=2, beam_gamma=g, enable_ncs=0, seed=19)
    n, S = 20000, 300
    ids = np.arange(n)
    st = O.init(t, r, ids)
    ph, _, _, _ = O.run(t, r, ids, st, 0, S, capacity=1 << 16)
    first = np.full(n, S)
    pid = ph["id_mech"].astype(np.int64) & 0x7FFFFFFF
    np.minimum.at(first, pid, ph["step"].astype(np.int64))
    sig, _ = t.sigma_interp(0, g)
    n_i = 1e8 * O.critical_density(1e-6) / 51.0
    dt = 2 * math.pi * 0.01
    beta = math.sqrt(1 - 1 / g ** 2)
    xb = n_i * ALPHA * RE * RE * dt * 1e-6 / (2 * math.pi) * sig * beta
    edges = list(range(0, S, 20)) + [S]
    obs = np.array([np.sum((first >= a) & (first < b)) for a, b in zip(edges[:-1], edges[1:])] + [np.sum(first == S)])

    def chi2(x):
        q = math.exp(-x)                                     # 1 - P per step
        e = np.array([n * (q ** a - q ** b) for a, b in zip(edges[:-1], edges[1:])] + [n * q ** S])
        return float(((obs - e) ** 2 / e).sum())

    dof = len(obs) - 1
    assert st_.chi2.sf(chi2(xb), dof) > 1e-3, chi2(xb)
    assert st_.chi2.sf(chi2(xb / beta), dof) < 1e-5            # beta left out


def test_ncs_first_emission_follows_the_rate():
    """The step's NCS optical depth falls at the paper's rate (Sec. 2.2): in a constant magnetic
    field across the electron's velocity, gamma and eta stay fixed until it emits, so tau drops
    by the same dtau = (sqrt3 alpha / 2 pi) (m c^2 / hbar omega) (eta / gamma) h(eta) omega dt each
    step and the first emission comes at step ceil(tau_0 / dtau) - 1, P(n_1 >= k) = e^{-k dtau}.
    m c^2 / hbar omega is lambda / (2 pi lambdabar_C) from CODATA, not the oracle's own E_S; h is
    the table, pinned to brute-force quadrature above.  A rate without the 1/gamma, with another
    prefactor or a decrement off by a step fails the chi^2.  The first photons point along the
    analytically rotated velocity, which fixes the emission direction and the push's sense."""
    t = O.Tables(O.table_params(n_eta=64, n_y=32, n_E=2, n_s=2), [13.0])
    lam, lbar_c = 1e-6, 3.8615926796e-13                     # m; CODATA reduced Compton wavelength
    E_S = lam / (2 * math.pi * lbar_c)                       # m c^2 / (hbar omega) = E_S / (m c omega / e)
    gamma, eta = 100.0, 0.05
    u = math.sqrt(gamma * gamma - 1.0)
    Bz = eta * E_S / u                                       # |u x B| / E_S = eta for u along x, B along z
    r = O.run_params(geometry=2, B_const=(0.0, 0.0, Bz), init_dist=2, beam_gamma=gamma, enable_brems=0, seed=13)
    dt = 2 * math.pi * 0.01
    h, _ = t.h_interp(eta)
    dtau = math.sqrt(3) * ALPHA / (2 * math.pi) * E_S * (eta / gamma) * h * dt
    n, S = 20000, 60
    ids = np.arange(n)
    st = O.init(t, r, ids)
    ev = np.zeros(n, dtype=np.uint64)
    first = np.full(n, S)
    photons = []
    for k in range(S):
        ph, _, _, _ = O.run(t, r, ids, st, k, 1, capacity=1 << 16, events=ev)
        emitted = (ev & np.uint64(0xFFFF)) > 0
        first[(first == S) & emitted] = k
        photons.append(ph)
    assert 0.05 < dtau < 0.2
    # each electron's first photon leaves along its velocity (collinear emission, Sec. 2.2): after
    # n + 1 pushes of a pure rotation by 2 atan(B dt / 2 gamma), toward +y for an electron from +x
    ph = np.concatenate(photons)
    pid = ph["id_mech"].astype(np.int64) & 0x7FFFFFFF
    at_first = (ph["id_mech"] >> 31 == 0) & (ph["step"].astype(np.int64) == first[pid])
    assert at_first.sum() > n // 4
    theta = 2.0 * math.atan(0.5 * dt * Bz / gamma)
    phi = (ph["step"][at_first].astype(np.float64) + 1.0) * theta
    assert np.abs(ph["kx"][at_first] - np.cos(phi)).max() < 1e-6
    assert np.abs(ph["ky"][at_first] - np.sin(phi)).max() < 1e-6
    assert np.abs(ph["kz"][at_first]).max() < 1e-6
    edges = list(range(0, S, 4)) + [S]
    obs = np.array([np.sum((first >= a) & (first < b)) for a, b in zip(edges[:-1], edges[1:])] + [np.sum(first == S)])

    def expected(d, lag=0):
        # P(n_1 >= k) = e^{-(k + lag) d}; lag = 1: the crossing tested before the step's decrement
        def surv(k):
            return math.exp(-max(k + lag, 0) * d)
        return np.array([n * (surv(a) - surv(b)) for a, b in zip(edges[:-1], edges[1:])] + [n * surv(S)])

    keep = expected(dtau) > 5                               # the bins of the stated rate, for every model

    def chi2(d, lag=0):
        e = np.maximum(expected(d, lag)[keep], 1e-3)
        return float(((obs[keep] - e) ** 2 / e).sum())

    dof = int(keep.sum()) - 1
    c = chi2(dtau)
    assert st_.chi2.sf(c, dof) > 1e-3, c
    # the statistic separates the rate from its plausible misreadings
    for wrong, lag in ((dtau * 1.05, 0), (dtau / 1.05, 0), (dtau * 2 * math.pi, 0), (dtau * gamma, 0), (dtau, 1)):
        assert st_.chi2.sf(chi2(wrong, lag), dof) < 1e-5, (wrong, lag)


def test_histograms_bin_the_photon_records():
    """The energy and angle histograms are the photon records binned by the stated rule: 512 bins
    of ln(E / m c^2) up to 10 GeV and 180 bins of atan2(k_y, k_x) over [-pi, pi), NCS and brems
    apart.  Only a record within 1e-5 of a bin edge may land one bin over (the record holds the
    energy and direction in float)."""
    p = O.table_params(n_eta=32, n_y=32, n_E=32, n_s=32)
    t = O.Tables(p, [79.0])
    r = O.run_params(a0=270.0, Z=79.0, charge_state=51.0, ne_over_nc=2e5, init_dist=1, T_mev=1.0, seed=4)
    ids = np.arange(2000)
    st = O.init(t, r, ids)
    ph, n, hist, tally = O.run(t, r, ids, st, 0, 1500, capacity=1 << 18)
    assert n == len(ph) and len(ph) > 500
    mech = (ph["id_mech"] >> 31).astype(np.int64)
    assert 0 < mech.sum() < len(ph)                           # both mechanisms present
    fe = 512 * np.log(ph["energy"].astype(np.float64)) / math.log(10000.0 / 0.51099895)
    ft = (np.arctan2(ph["ky"].astype(np.float64), ph["kx"].astype(np.float64)) + math.pi) / (2 * math.pi) * 180
    near = (np.abs(fe - np.round(fe)) < 1e-5) | (np.abs(ft - np.round(ft)) < 1e-5)
    eb = np.clip(np.floor(fe).astype(np.int64), 0, 511)
    tb = np.clip(np.floor(ft).astype(np.int64), 0, 179)
    want = np.zeros_like(hist)
    np.add.at(want, mech * 512 + eb, 1)
    np.add.at(want, 1024 + mech * 180 + tb, 1)
    assert int(np.abs(hist.astype(np.int64) - want.astype(np.int64)).sum()) <= 2 * int(near.sum())


def test_initial_positions_uniform_in_the_slab():
    """Electrons start uniform over the slab (x in [x0, x1], and in 2D y in [-y_h, y_h]; KS), a
    beam at its front face."""
    from scipy.stats import kstest
    t = O.Tables(O.table_params(n_eta=2, n_y=4, n_E=2, n_s=2), [13.0])
    k = 2 * math.pi / 1e-6
    r = O.run_params(geometry=1, slab_x0_m=2e-6, slab_thick_m=1e-6, y_half_m=3e-6, seed=23)
    st = O.init(t, r, np.arange(20000))
    x0, x1, yh = 2e-6 * k, 3e-6 * k, 3e-6 * k
    assert st[:, 0].min() >= x0 and st[:, 0].max() <= x1 and np.abs(st[:, 1]).max() <= yh
    assert kstest((st[:, 0] - x0) / (x1 - x0), "uniform").pvalue > 1e-3
    assert kstest((st[:, 1] + yh) / (2 * yh), "uniform").pvalue > 1e-3
    rb = O.run_params(slab_x0_m=2e-6, init_dist=2, beam_gamma=10.0, seed=23)
    assert np.all(O.init(t, rb, np.arange(100))[:, 0] == x0)


def test_free_streaming_and_the_absorbing_box():
    """Fields and emissions off, 2D geometry: each electron streams, x^n = x^0 + n dt u_x / gamma
    and y^n = y^0 + n dt u_y / gamma, and the absorbing box removes it at the first step whose
    position lies outside [box0, box1] through either face; the kill tallies count those steps."""
    t = O.Tables(O.table_params(n_eta=2, n_y=4, n_E=2, n_s=2), [13.0])
    k = 2 * math.pi / 1e-6
    r = O.run_params(a0=0.0, geometry=1, init_dist=1, T_mev=1.0, enable_ncs=0, enable_brems=0, box_enable=1,
                     box_x_m=(2.2e-6, 2.8e-6), slab_x0_m=2e-6, slab_thick_m=1e-6, y_half_m=3e-6, seed=29)
    n, S = 5000, 50
    ids = np.arange(n)
    st = O.init(t, r, ids)
    x0, y0, u = st[:, 0].copy(), st[:, 1].copy(), st[:, 2:5].copy()
    _, _, _, tally = O.run(t, r, ids, st, 0, S, capacity=1 << 10)
    dt = 2 * math.pi * 0.01
    v = u / np.sqrt(1 + (u ** 2).sum(1))[:, None]
    steps = np.arange(1, S + 1)[None, :]
    xs = x0[:, None] + steps * dt * v[:, :1]
    out = (xs < 2.2e-6 * k) | (xs > 2.8e-6 * k)
    killed = out.any(1)
    first = np.where(killed, out.argmax(1) + 1, 0)
    assert 0.2 < killed.mean() < 0.9 and np.any(v[killed, 0] < 0) and np.any(v[killed, 0] > 0)
    assert np.array_equal(np.isnan(st[:, 0]), killed)
    assert int(tally[O.T["N_KILLED"]]) == int(killed.sum())
    assert int(tally[O.T["KILLED_STEPS"]]) == int(first.sum())
    live = ~killed
    assert np.allclose(st[live, 0], x0[live] + S * dt * v[live, 0], rtol=0, atol=1e-11)
    assert np.allclose(st[live, 1], y0[live] + S * dt * v[live, 1], rtol=0, atol=1e-11)
    assert np.array_equal(st[:, 2:5], u)                     # no field, no emission: momenta unchanged


def _constant_B_run(gamma, eta, n, seed):
    """Electrons along +x at gamma in a constant B_z with |u x B| / E_S = eta, NCS only."""
    t = O.Tables(O.table_params(n_eta=64, n_y=32, n_E=2, n_s=2), [13.0])
    E_S = 1e-6 / (2 * math.pi * 3.8615926796e-13)
    Bz = eta * E_S / math.sqrt(gamma * gamma - 1.0)
    r = O.run_params(geometry=2, B_const=(0.0, 0.0, Bz), init_dist=2, beam_gamma=gamma, enable_brems=0, seed=seed)
    ids = np.arange(n)
    return t, r, ids, O.init(t, r, ids)


def test_ncs_optical_depth_resets_after_emission():
    """After the step of an NCS emission the optical depth is a fresh -ln U (Sec. 2.2): over the
    electrons that emitted in a step, tau is exponential with unit mean (KS)."""
    from scipy.stats import kstest
    t, r, ids, st = _constant_B_run(100.0, 0.05, 20000, 31)
    ev = np.zeros(len(ids), dtype=np.uint64)
    taus = []
    for k in range(30):
        before = ev & np.uint64(0xFFFF)
        O.run(t, r, ids, st, k, 1, capacity=1 << 16, events=ev)
        taus.append(st[(ev & np.uint64(0xFFFF)) > before, 5])
    taus = np.concatenate(taus)
    assert len(taus) > 5000 and taus.min() > 0.0
    assert kstest(taus, "expon").pvalue > 1e-3


def test_photon_energy_clamp_conserves_energy():
    """At gamma = 3 and eta = 5 the sampled fraction often exceeds 1 - 1/gamma; the photon then takes
    gamma - 1 (counted) and leaves the electron at rest, and recoil still equals the emitted energy."""
    t, r, ids, st = _constant_B_run(3.0, 5.0, 4000, 37)
    ev = np.zeros(len(ids), dtype=np.uint64)
    ph, n, hist, tally = O.run(t, r, ids, st, 0, 40, capacity=1 << 18, events=ev)
    assert int(tally[O.T["N_CLAMP"]]) > 100
    emitted = sum(O.fixed_to_float(tally, O.T[k]) for k in ("E_NCS_STORED", "E_NCS_BELOW"))
    assert abs(O.fixed_to_float(tally, O.T["E_RECOIL_NCS"]) / emitted - 1) < 1e-12
    # a clamped emission leaves the electron at rest for good (u = 0: eta = 0 in a pure B field)
    assert int(np.all(st[:, 2:5] == 0.0, axis=1).sum()) == int(tally[O.T["N_CLAMP"]])


def test_brems_only_inside_the_target():
    """Eq. 4 acts in the target only: with fields off in 2D, electrons drifting out of the slab in x
    and in y, every brems photon starts inside [x0, x1] x [-y_h, y_h]."""
    t = O.Tables(O.table_params(n_eta=2, n_y=4, n_E=32, n_s=16), [79.0])
    k = 2 * math.pi / 1e-6
    r = O.run_params(a0=0.0, geometry=1, Z=79.0, charge_state=51.0, ne_over_nc=2e7, init_dist=1, T_mev=1.0,
                     enable_ncs=0, slab_x0_m=2e-6, slab_thick_m=0.3e-6, y_half_m=0.3e-6, seed=41)
    ids = np.arange(5000)
    st = O.init(t, r, ids)
    ph, n, _, _ = O.run(t, r, ids, st, 0, 60, capacity=1 << 18)
    assert n > 500
    x0, x1, yh = 2e-6 * k, 2.3e-6 * k, 0.3e-6 * k
    assert np.mean((st[:, 0] < x0) | (st[:, 0] > x1) | (np.abs(st[:, 1]) > yh)) > 0.5   # most drifted out
    tol = 1e-5
    assert np.all((ph["x"] >= x0 - tol) & (ph["x"] <= x1 + tol) & (np.abs(ph["y"]) <= yh + tol))


def test_energy_bookkeeping():
    p = O.table_params(n_eta=32, n_y=32, n_E=32, n_s=32)
    t = O.Tables(p, [79.0])
    r = O.run_params(a0=270.0, Z=79.0, charge_state=51.0, init_dist=1, T_mev=1.0, seed=2)
    ids = np.arange(200)
    st = O.init(t, r, ids)
    ph, n, hist, tally = O.run(t, r, ids, st, 0, 1500, capacity=1 << 18)
    emitted = sum(O.fixed_to_float(tally, O.T[k]) for k in ("E_NCS_STORED", "E_NCS_BELOW", "E_BR_STORED", "E_BR_BELOW"))
    recoil = O.fixed_to_float(tally, O.T["E_RECOIL_NCS"]) + O.fixed_to_float(tally, O.T["E_RECOIL_BR"])
    assert tally[O.T["N_NCS_STORED"]] + tally[O.T["N_NCS_BELOW"]] > 100
    assert abs(recoil / emitted - 1) < 1e-12
    assert n == int(tally[O.T["N_PHOTONS"]])
    assert int(hist[:512].sum()) == int(tally[O.T["N_NCS_STORED"]])
    assert int(hist[512:1024].sum()) == int(tally[O.T["N_BR_STORED"]])
    assert np.all(ph["energy"] >= 1.0)


# ---------------------------------------------------------- field model ----
def _envelope_definition(phi, pr, pf):
    """Sec. 3's pulse envelope: sin^2 rise over pr, flat top pf, cos^2 fall."""
    if phi <= 0.0 or phi >= 2.0 * pr + pf:
        return 0.0
    if phi < pr:
        return math.sin(0.5 * math.pi * phi / pr) ** 2
    if phi <= pr + pf:
        return 1.0
    return math.cos(0.5 * math.pi * (phi - pr - pf) / pr) ** 2


def test_plane_wave_fields_from_the_vector_potential():
    """The 1D pulse is defined through its vector potential, A_y = a0 g(phi) sin phi (and for CP
    A_z = -a0 g(phi) cos phi), phi = t - x: E = -dA/dt and B = x^ x E at 997 phases across the
    five parts of the pulse, by central differences of the test's own A (measured 2.3e-8 at
    a0 = 10).  Maxwell's equations cannot catch a wrong envelope derivative -- any f(t - x) is a
    vacuum wave -- so the fields are checked against the definition."""
    worst = 0.0
    for pol in (0, 1):
        r = O.run_params(a0=10.0, polarisation=pol, geometry=0)
        pr = 2 * math.pi * r.ramp_periods
        pf = 2 * math.pi * r.flat_s * 299792458.0 / r.lambda_m

        def A(p):
            g = _envelope_definition(p, pr, pf)
            return 10.0 * g * math.sin(p), (-10.0 * g * math.cos(p) if pol else 0.0)

        h = 1e-4
        for p in np.linspace(-3.0, 2 * pr + pf + 3.0, 997):
            E, B = O.fields(r, 0.0, 0.0, p)
            ap, am = A(p + h), A(p - h)
            ey, ez = -(ap[0] - am[0]) / (2 * h), -(ap[1] - am[1]) / (2 * h)
            worst = max(worst, abs(E[1] - ey), abs(E[2] - ez), abs(B[2] - E[1]), abs(B[1] + E[2]))
    assert worst < 1e-6


def test_gaussian_focus_satisfies_the_paraxial_equation():
    """The 2D focus on the flat top is Re[u e^{i(t - x)}] with u the exact Gaussian-beam solution of
    the paraxial equation 2i du/dx = d^2u/dy^2 (the wave equation without d^2u/dx^2): u is read off
    two samples of E_y a quarter period apart and the equation checked by finite differences from
    -150 to +170 about the focus, on and off axis (residual measured 4.2e-5 of |u|/z_R + |u_yy|).
    A Gouy phase of the wrong sign against the wavefront curvature leaves a residual of order 1."""
    r = O.run_params(a0=1.0, polarisation=0, geometry=1, w0_m=3e-6, focus_x_m=2e-6)
    k = 2 * math.pi / 1e-6
    xf, w0 = 2e-6 * k, 3e-6 * k
    zr = 0.5 * w0 * w0

    def u(x, y, t):
        c = -O.fields(r, x, y, t)[0][1]
        d = -O.fields(r, x, y, t + 0.5 * math.pi)[0][1]
        return (c - 1j * d) * np.exp(-1j * (t - x))

    hx, hy, worst = 0.5, 0.2, 0.0
    for xi in (-150.0, -40.0, 0.0, 60.0, 170.0):
        for y in (0.0, 5.0, 12.0, 20.0):
            x = xf + xi
            t = x + 30.0                                   # phase 30: on the flat top
            ux = (u(x + hx, y, t) - u(x - hx, y, t)) / (2 * hx)
            uyy = (u(x, y + hy, t) - 2 * u(x, y, t) + u(x, y - hy, t)) / (hy * hy)
            worst = max(worst, abs(2j * ux - uyy) / (abs(u(x, y, t)) / zr + abs(uyy)))
    assert worst < 1e-3


def test_fields_gaussian_reduces_to_plane_wave():
    for pol in (0, 1):
        r1 = O.run_params(a0=10.0, polarisation=pol, geometry=0)
        r2 = O.run_params(a0=10.0, polarisation=pol, geometry=1, w0_m=1e3, focus_x_m=2e-6)
        for (x, y, t) in ((13.0, 0.5, 20.0), (15.0, -2.0, 40.0), (14.1, 3.0, 70.3)):
            E1, B1 = O.fields(r1, x, y, t)
            E2, B2 = O.fields(r2, x, y, t)
            np.testing.assert_allclose(E2, E1, atol=1e-6 * 10)
            np.testing.assert_allclose(B2, B1, atol=1e-6 * 10)


def test_fields_cp_constant_amplitude_and_plane_wave_relation():
    r = O.run_params(a0=7.0, polarisation=1)
    for t in np.linspace(15.0, 60.0, 17):
        E, B = O.fields(r, 1.0, 0.0, t)              # inside the flat top (phi in [2 pi, 2 pi + 56.5])
        assert abs(math.sqrt(E @ E) - 7.0) < 1e-12
        np.testing.assert_allclose(B, np.cross([1.0, 0.0, 0.0], E), atol=1e-12)


def test_fields_gaussian_divergence_free_to_first_order():
    # div E = dEx/dx + dEy/dy vanishes up to terms of order (1/(k w0))^2 relative to |E|/w0
    r = O.run_params(a0=1.0, polarisation=1, geometry=1, w0_m=3e-6, focus_x_m=2e-6)
    w0 = 3e-6 * 2 * math.pi / 1e-6
    h = 1e-4
    for (x, y, t) in ((12.0, 3.0, 30.0), (20.0, -5.0, 45.0), (30.0, 8.0, 60.0)):
        dEx = (O.fields(r, x + h, y, t)[0][0] - O.fields(r, x - h, y, t)[0][0]) / (2 * h)
        dEy = (O.fields(r, x, y + h, t)[0][1] - O.fields(r, x, y - h, t)[0][1]) / (2 * h)
        dBx = (O.fields(r, x + h, y, t)[1][0] - O.fields(r, x - h, y, t)[1][0]) / (2 * h)
        dBy = (O.fields(r, x, y + h, t)[1][1] - O.fields(r, x, y - h, t)[1][1]) / (2 * h)
        assert abs(dEx + dEy) < 0.1 / w0
        assert abs(dBx + dBy) < 0.1 / w0
        # the leading transverse derivative alone is O(1/w0): the cancellation is real
        assert abs(dEy) > 0.3 * abs(y) / w0 ** 2 or abs(dEy) < 1e-3


def test_config2_time_step_is_ill_conditioned():
    """The 1D Au a0 = 270 workload at dt = T/100: passages through the nodes of the
    vector potential at low gamma are not resolved, so the discrete map is
    ill-conditioned there.  The FP64 oracle's own response to a 2^-24 relative
    perturbation of the initial momenta exceeds 1e-5 of the momentum scale for some
    particles, and a smaller time step shrinks it: no arithmetic can promise 1e-5 per
    particle on this workload, which is why its FP32 parity bound is distributional."""
    p = O.table_params(n_eta=32, n_y=32, n_E=32, n_s=32)
    t = O.Tables(p, [79.0])
    worst = []
    for dto, steps in ((0.01, 1500), (0.0025, 6000)):
        r = O.run_params(a0=270.0, Z=79.0, charge_state=51.0, init_dist=1, T_mev=1.0, seed=2, dt_over_T=dto,
                         enable_ncs=0, enable_brems=0)
        ids = np.arange(400)
        a = O.init(t, r, ids)
        b = a.copy()
        sgn = np.where((ids[:, None] + np.arange(3)[None, :]) % 2 == 0, 1.0, -1.0)
        b[:, 2:5] *= 1 + sgn * 2.0 ** -24
        O.run(t, r, ids, a, 0, steps, capacity=16)
        O.run(t, r, ids, b, 0, steps, capacity=16)
        scale = np.maximum(np.abs(a[:, 2:5]).max(1), 270.0)
        worst.append((np.abs(a[:, 2:5] - b[:, 2:5]).max(1) / scale).max())
    assert worst[0] > 1e-5
    assert worst[1] < worst[0] / 4


@pytest.mark.parametrize("E0,target", [(1000.0, "Au"), (1000.0, "Al"), (100.0, "Au")])
def test_bunch_energy_loss_radiation_length(E0, target):
    """Sec. 2.2 benchmark (fields off, pusher + brems only): a 1 GeV bunch through 5 mm of target
    loses energy by bremsstrahlung at the radiation-length rate, <E>/E0 ~ exp(-L/X0) (Tsai complete
    screening, PDG X0), to a few per cent.  A 100 MeV bunch slows into the regime of incomplete
    screening and of a hard-photon cut that is no longer negligible, so it loses less than that law."""
    from paper_1612_07592_gb300 import workloads as W
    c = W.bunch(E0, target, n=2000)
    X0_gcm2, rho = (6.46, 19.3) if target == "Au" else (24.01, 2.70)
    L_over_X0 = 0.5 / (X0_gcm2 / rho)
    p = O.table_params(n_eta=2, n_y=4, n_E=96, n_s=64, gamma_min=2.0, gamma_max=1e5)
    t = O.Tables(p, [13.0, 79.0])
    run = dict(c["run"]); run["iz"] = 1 if target == "Au" else 0
    r = O.run_params(**run)
    ids = np.arange(c["n"])
    st = O.init(t, r, ids)
    assert np.all(st[:, 0] == 0.0)
    ph, n, hist, tally = O.run(t, r, ids, st, 0, c["steps"], capacity=1 << 20)
    g0 = E0 / 0.51099895 + 1.0
    g = np.sqrt(1 + (st[:, 2:5] ** 2).sum(1))
    ratio = (g - 1).mean() / (g0 - 1)
    law = math.exp(-L_over_X0)
    if E0 >= 1000.0:
        assert abs(ratio / law - 1) < 0.06, (ratio, law)
    else:
        assert law < ratio < 1.3 * law, (ratio, law)
    # energy bookkeeping: electron loss = photon energy (stored, above the cut)
    emitted = O.fixed_to_float(tally, O.T["E_BR_STORED"])
    lost = (g0 - g).sum()
    assert abs(emitted / lost - 1) < 1e-9


def test_fp32_error_model_file_is_the_oracles():
    """tests/golden/fp32_error_model.txt (the bound of the FP32 parity tests on the 1D Au a0 = 270
    workload) is what its script computes from the oracle: the small case is recomputed here and
    must match the stored line.  The model itself: a one-ulp per-step momentum perturbation moves
    more electrons past 1e-5 than a single 2^-24 kick of the initial momenta does (the FP32 path
    rounds at every step, so the per-step model is the one that applies), and it never moves the
    positions, which the FP32 path keeps as compensated pairs, as far as the momenta."""
    import importlib.util
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_fp32_error_model.py")
    spec = importlib.util.spec_from_file_location("make_fp32_error_model", path)
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    tp, Z, run, ids, steps = mk.cases()["small"]
    m, eu, ex, et = mk.model(tp, Z, run, ids, steps)
    stored = {}
    for ln in open(mk.OUT):
        p = ln.split()
        if p and p[0] == "small":
            stored[p[1]] = [float(v) for v in p[2:]]
    for q, e in (("u", eu), ("x", ex), ("tau", et)):
        got = [float(m.sum()), float(m.mean())] + [float(np.mean(e < t)) for t in mk.THRESHOLDS]
        np.testing.assert_allclose(got, stored[q], rtol=0, atol=2e-6)
    # a single initial kick of 2^-24 leaves more electrons within 1e-5 than the per-step model
    ot = O.Tables(O.table_params(**{("photon_min" if k == "photon_min_mc2" else k): v for k, v in tp.items()}),
                  list(Z))
    d = dict(run)
    d["iz"] = list(Z).index(d["Z"])
    rp = O.run_params(**d)
    a = O.init(ot, rp, ids)
    b = a.copy()
    b[:, 2:5] *= 1 + np.where((ids[:, None] + np.arange(3)[None, :]) % 2 == 0, 1.0, -1.0) * 2.0 ** -24
    O.run(ot, rp, ids, a, 0, steps, capacity=1 << 16)
    O.run(ot, rp, ids, b, 0, steps, capacity=1 << 16)
    eu1, _, _ = mk.errors(a, b, run["a0"])
    assert np.mean(eu1 < 1e-5) > np.mean(eu < 1e-5) + 0.05
    assert np.mean(ex < 1e-5) > np.mean(eu < 1e-5)

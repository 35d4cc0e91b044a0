"""Pins of the oracle's two variants beyond the paper's direct step.

* Null-collision bremsstrahlung (the speed-up the paper names for its MC
  collision, Sec. 4): a majorant candidate process thinned by P/P_hat.  Pinned
  against the law of Eq. 4 itself (geometric first-event steps with the direct
  probability), the geometric law of the candidate waits, the radiation-length
  energy loss of the Sec. 2.2 bunch, and a two-sample comparison with the
  direct method.
* Reflected laser wave (the hole-boring front of Sec. 3 as a fixed mirror):
  pinned against Maxwell's equations in vacuum, the mirror condition, the
  light-front form of eta for a wave moving along -x, and the plane wave at r = 0.
"""
import math

import numpy as np
import pytest
import scipy.stats as st_

import oracle as O

ALPHA = 7.2973525693e-3
RE = 2.8179403262e-15


# ------------------------------------------------------- null collisions ----
def _frozen_run(method, n_e=2e6, gamma=2e3, seed=5):
    p = O.table_params(n_eta=2, n_y=4, n_E=64, n_s=32)
    t = O.Tables(p, [79.0])
    r = O.run_params(geometry=2, Z=79.0, charge_state=51.0, ne_over_nc=n_e, slab_x0_m=-1.0, slab_thick_m=2.0,
                     init_dist=2, beam_gamma=gamma, enable_ncs=0, seed=seed, brems_method=method)
    return t, r


def _direct_P(t, n_e, gamma):
    sig, _ = t.sigma_interp(0, gamma)
    n_i = n_e * O.critical_density(1e-6) / 51.0
    dt = 2 * math.pi * 0.01
    xb = n_i * ALPHA * RE * RE * dt * 1e-6 / (2 * math.pi) * sig * math.sqrt(1 - 1 / gamma ** 2)
    return -math.expm1(-xb)


def test_null_collision_first_event_has_direct_probability():
    """Fields off, electron at fixed gamma inside a thick slab: with null collisions the first
    brems event is still geometric with the Eq. 4 probability P(gamma) per step, although
    candidates come at the larger rate P_hat.  A candidate accepted without the P/P_hat thinning,
    or thinned with the wrong ratio, fails."""
    t, r = _frozen_run(1)
    n, S = 20000, 400
    ids = np.arange(n)
    wait = np.zeros(n, dtype=np.uint32)
    st = O.init(t, r, ids, wait=wait)
    ph, nph, hist, tally = O.run(t, r, ids, st, 0, S, capacity=1 << 18, wait=wait)
    first = {}
    for rec in ph:
        first.setdefault(int(rec["id_mech"]) & 0x7FFFFFFF, int(rec["step"]))
    P = _direct_P(t, 2e6, 2e3)
    x_hat = O.null_x_hat(t, r)
    P_hat = -math.expm1(-x_hat)
    assert P < 0.8 * P_hat                       # thinning matters at this energy
    waits = np.array([first.get(i, S) for i in ids])
    # chi^2 of the first-event step in 20 bins of 20 steps plus the censored bin
    edges = np.arange(0, S + 1, 20)
    obs = np.array([np.sum((waits >= a) & (waits < b)) for a, b in zip(edges[:-1], edges[1:])] +
                   [np.sum(waits == S)])
    q = 1 - P
    exp_ = np.array([n * (q ** a - q ** b) for a, b in zip(edges[:-1], edges[1:])] + [n * q ** S])
    chi2 = float(((obs - exp_) ** 2 / exp_).sum())
    assert st_.chi2.sf(chi2, len(obs) - 1) > 1e-3, chi2
    # the same statistic with the majorant probability is far off
    exp_hat = np.array([n * ((1 - P_hat) ** a - (1 - P_hat) ** b) for a, b in zip(edges[:-1], edges[1:])] +
                       [n * (1 - P_hat) ** S])
    assert float(((obs - exp_hat) ** 2 / exp_hat).sum()) > 10 * chi2 + 100


def test_null_collision_waits_are_geometric():
    """Initial waits: P(w >= k) = (1 - P_hat)^k with x_hat = n_i c dt max sigma_Z."""
    t, r = _frozen_run(1, n_e=2e5)
    n = 50000
    wait = np.zeros(n, dtype=np.uint32)
    O.init(t, r, np.arange(n), wait=wait)
    # the majorant: n_i c dt times the largest tabulated sigma_Z (in alpha r_e^2)
    n_i = 2e5 * O.critical_density(1e-6) / 51.0
    x_hat = n_i * ALPHA * RE * RE * (0.01 * 1e-6) * t.export(3, 0).max()
    assert abs(O.null_x_hat(t, r) / x_hat - 1) < 1e-12
    P_hat = -math.expm1(-x_hat)
    w = wait.astype(np.float64)
    mean = (1 - P_hat) / P_hat
    assert abs(w.mean() / mean - 1) < 5 / math.sqrt(n)
    # Kolmogorov distance to the geometric CDF at its support points
    ks = np.sort(w)
    emp = np.arange(1, n + 1) / n
    cdf = 1 - (1 - P_hat) ** (ks + 1)
    assert np.max(np.abs(emp - cdf)) < 1.63 / math.sqrt(n)      # 1 % KS level


def test_null_collision_no_target_never_collides():
    t, r = _frozen_run(1, n_e=0.0)
    n = 100
    wait = np.zeros(n, dtype=np.uint32)
    st = O.init(t, r, np.arange(n), wait=wait)
    assert np.all(wait == 0xFFFFFFFF)
    ph, nph, hist, tally = O.run(t, r, np.arange(n), st, 0, 200, capacity=16, wait=wait)
    assert nph == 0 and np.all(wait == 0xFFFFFFFF)


def test_null_collision_needs_wait_array():
    t, r = _frozen_run(1)
    with pytest.raises(ValueError):
        O.init(t, r, np.arange(4))


@pytest.mark.parametrize("target", ["Au", "Al"])
def test_null_collision_bunch_matches_direct_and_radiation_length(target):
    """Sec. 2.2 bunch (1 GeV, 5 mm, fields off): null collisions lose energy at the radiation-length
    rate like the direct method, and the two photon spectra agree (two-sample chi^2)."""
    from paper_1612_07592_gb300 import workloads as W
    c = W.bunch(1000.0, target, n=1500)
    X0_gcm2, rho = (6.46, 19.3) if target == "Au" else (24.01, 2.70)
    law = math.exp(-0.5 / (X0_gcm2 / rho))
    p = O.table_params(n_eta=2, n_y=4, n_E=96, n_s=64, gamma_min=2.0, gamma_max=1e5)
    t = O.Tables(p, [13.0, 79.0])
    ids = np.arange(c["n"])
    g0 = 1000.0 / 0.51099895 + 1.0
    spectra, ratios = [], []
    for method in (0, 1):
        run = dict(c["run"], iz=1 if target == "Au" else 0, brems_method=method)
        r = O.run_params(**run)
        wait = np.zeros(len(ids), dtype=np.uint32)
        st = O.init(t, r, ids, wait=wait)
        ph, n, hist, tally = O.run(t, r, ids, st, 0, c["steps"], capacity=1 << 21, wait=wait)
        g = np.sqrt(1 + (st[:, 2:5] ** 2).sum(1))
        ratios.append((g - 1).mean() / (g0 - 1))
        spectra.append(hist[O.HIST_E_BINS:2 * O.HIST_E_BINS].astype(np.float64))
        emitted = O.fixed_to_float(tally, O.T["E_BR_STORED"])
        assert abs(emitted / (g0 - g).sum() - 1) < 1e-9
    assert abs(ratios[1] / law - 1) < 0.06, (ratios, law)
    # per-electron energy spread is ~0.3 of the mean: the two means agree within 4 sigma
    assert abs(ratios[1] - ratios[0]) < 4 * 0.45 * ratios[0] * math.sqrt(2.0 / len(ids))
    a, b = spectra
    # merge bins to >= 20 counts each
    edges, acc_a, acc_b = [], 0.0, 0.0
    A, B = [], []
    for k in range(len(a)):
        acc_a += a[k]; acc_b += b[k]
        if acc_a >= 20 and acc_b >= 20:
            A.append(acc_a); B.append(acc_b); acc_a = acc_b = 0.0
    if acc_a or acc_b:
        A[-1] += acc_a; B[-1] += acc_b
    A, B = np.array(A), np.array(B)
    ka, kb = math.sqrt(B.sum() / A.sum()), math.sqrt(A.sum() / B.sum())
    chi2 = float((((ka * A - kb * B) ** 2) / (A + B)).sum())
    assert st_.chi2.sf(chi2, len(A) - 1) > 1e-3, chi2


# ------------------------------------------------------- reflected wave -----
def _refl(pol=0, r=0.7, a0=3.0):
    return O.run_params(a0=a0, polarisation=pol, geometry=0, reflect_r=r, mirror_x_m=3e-6, flat_s=10e-15,
                        ramp_periods=2.0)


KL = 2 * math.pi / 1e-6
XM = 3e-6 * KL


@pytest.mark.parametrize("pol", [0, 1])
def test_reflected_wave_mirror_node(pol):
    """r = 1: the transverse E vanishes on the mirror plane at all times; B doubles there."""
    run = _refl(pol, r=1.0)
    run0 = _refl(pol, r=0.0)
    for t in np.linspace(XM + 0.3, XM + 60.0, 41):
        E, B = O.fields(run, XM, 0.0, t)
        E0, B0 = O.fields(run0, XM, 0.0, t)
        assert abs(E[1]) < 1e-12 * 3 and abs(E[2]) < 1e-12 * 3
        np.testing.assert_allclose(B, 2 * B0, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("pol", [0, 1])
def test_reflected_wave_satisfies_maxwell(pol):
    """Vacuum Maxwell equations in 1D (c = 1), by central differences where incident and reflected
    pulses overlap, in their ramps and flat tops."""
    run = _refl(pol, r=0.7)
    h = 1e-4
    rng = np.random.default_rng(3)
    for _ in range(40):
        x = XM - rng.uniform(0.5, 30.0)
        t = XM + rng.uniform(0.0, 80.0)        # incident phase t - x and reflected t + x - 2 XM inside the pulse
        Ex1, Bx1 = O.fields(run, x + h, 0, t)
        Ex0, Bx0 = O.fields(run, x - h, 0, t)
        Et1, Bt1 = O.fields(run, x, 0, t + h)
        Et0, Bt0 = O.fields(run, x, 0, t - h)
        dxE, dxB = (Ex1 - Ex0) / (2 * h), (Bx1 - Bx0) / (2 * h)
        dtE, dtB = (Et1 - Et0) / (2 * h), (Bt1 - Bt0) / (2 * h)
        tol = 1e-6 * 3.0
        assert abs(dtE[1] + dxB[2]) < tol          # (curl B)_y = -d_x B_z = d_t E_y
        assert abs(dtB[2] + dxE[1]) < tol          # (curl E)_z =  d_x E_y = -d_t B_z
        assert abs(dtE[2] - dxB[1]) < tol          # (curl B)_z =  d_x B_y = d_t E_z
        assert abs(dtB[1] - dxE[2]) < tol          # (curl E)_y = -d_x E_z = -d_t B_y


@pytest.mark.parametrize("pol", [0, 1])
def test_reflected_wave_is_the_mirror_image_superposed(pol):
    """The reflected run's field is the incident pulse plus its mirror image -r e(t + x - 2 x_m)
    moving along -x: E = e(t - x) - r e(psi), B = x^ x e(t - x) + r x^ x e(psi) (B = -x^ x E_r),
    with e the r = 0 pulse, at r = 0.7 over random (t, x) on both sides of the mirror.  Maxwell's
    equations hold for any amplitude, so the amplitude is checked against this definition."""
    rr = 0.7
    k = 2 * math.pi / 1e-6
    r0 = O.run_params(a0=20.0, polarisation=pol, geometry=0)
    r1 = O.run_params(a0=20.0, polarisation=pol, geometry=0, reflect_r=rr, mirror_x_m=3e-6)
    xm = 3e-6 * k
    rng = np.random.default_rng(43)
    hit = 0
    for t, x in zip(rng.uniform(0.0, 150.0, 400), rng.uniform(-20.0, 60.0, 400)):
        ei = O.fields(r0, 0.0, 0.0, t - x)[0]                # e at the incident phase
        er = O.fields(r0, 0.0, 0.0, t + x - 2 * xm)[0]       # e at the reflected phase
        E, B = O.fields(r1, x, 0.0, t)
        want_E = (0.0, ei[1] - rr * er[1], ei[2] - rr * er[2])
        want_B = (0.0, -ei[2] - rr * er[2], ei[1] + rr * er[1])
        assert np.allclose(E, want_E, rtol=0, atol=1e-12) and np.allclose(B, want_B, rtol=0, atol=1e-12)
        hit += abs(er[1]) > 1.0
    assert hit > 50                                          # the mirror image is present at many points


def test_reflected_wave_zero_r_is_plane_wave():
    run, run0 = _refl(1, r=0.0), O.run_params(a0=3.0, polarisation=1, flat_s=10e-15, ramp_periods=2.0)
    for (x, t) in ((5.0, 30.0), (15.0, 50.0), (20.0, 90.0)):
        E, B = O.fields(run, x, 0, t)
        E0, B0 = O.fields(run0, x, 0, t)
        assert np.array_equal(E, E0) and np.array_equal(B, B0)


def test_reflected_wave_eta_light_front():
    """Where only the reflected pulse is present (the incident one has passed), eta of any electron
    is (gamma + u_x)|E|/E_S: the light-front form of a wave moving along -x.  Where only the incident
    pulse is present it is (gamma - u_x)|E|/E_S."""
    run = _refl(1, r=0.8, a0=50.0)
    E_S = O.schwinger_field(1e-6)
    pulse = 2 * 2 * math.pi * 2.0 + 2 * math.pi * 10e-15 * 299792458.0 / 1e-6
    rng = np.random.default_rng(4)
    x = XM - pulse - 5.0                   # the two pulses do not overlap here
    checked = [0, 0]
    for t in np.linspace(x, x + 2 * pulse + 30.0, 300):
        E, B = O.fields(run, x, 0, t)
        if not np.any(E):
            continue
        u = rng.normal(0, 30, 3)
        g = math.sqrt(1 + u @ u)
        phi, psi = t - x, t + x - 2 * XM
        inc = 0 < phi < pulse
        ref = 0 < psi < pulse
        assert inc != ref
        want = ((g + u[0]) if ref else (g - u[0])) * math.sqrt(E @ E) / E_S
        assert abs(O.eta(u, E, B, E_S) / want - 1) < 1e-9
        checked[int(ref)] += 1
    assert min(checked) > 20


def test_reflected_wave_dynamics_are_chaotic():
    """In the LP standing wave in front of a perfect mirror (a0 = 270, r = 1) nearby trajectories
    separate exponentially: a 2^-50 relative perturbation of the initial momenta grows by more than
    1e10 within 900 steps (it stays below 1e-11 in the plane wave alone).  Per-particle parity of two
    implementations with different rounding therefore has a horizon of a few hundred steps after the
    reflected pulse arrives; beyond it the comparison is statistical."""
    from paper_1612_07592_gb300 import workloads as W
    p = O.table_params(n_eta=48, n_y=48, n_E=48, n_s=48)
    t = O.Tables(p, [13.0, 79.0])
    worst = {}
    for name, refl in (("refl", 1.0), ("plane", 0.0)):
        run = W.base_run(a0=270.0, init_dist=1, T_mev=1.0, seed=2, reflect_r=refl, mirror_x_m=3e-6, **W.AU)
        run["iz"] = 1
        r = O.run_params(**run)
        ids = np.arange(200)
        a = O.init(t, r, ids)
        b = a.copy()
        b[:, 2:5] *= 1 + 2.0 ** -50
        O.run(t, r, ids, a, 0, 900, capacity=16)
        O.run(t, r, ids, b, 0, 900, capacity=16)
        scale = np.maximum(np.abs(a[:, 2:5]).max(1), 270.0)
        worst[name] = (np.abs(a[:, 2:5] - b[:, 2:5]).max(1) / scale).max()
    assert worst["plane"] < 1e-11
    assert worst["refl"] > 1e10 * 2.0 ** -50

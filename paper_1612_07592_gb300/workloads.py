"""Seeded synthetic workloads of the paper's setup (Sec. 3), shared by tests and the benchmark.

This module describes inputs only: run parameters (laser, target, step), particle
counts, arrival times.  It holds none of the method's arithmetic; the random
numbers the method itself draws (initial positions and momenta, optical depths,
emission decisions) come from the per-particle Philox streams inside the library
and inside the test oracle.

The paper's runs (Sec. 3): lambda = 1 um, LP along y, propagation along x,
30 fs flat top, Al or Au 1 um slab from x = 2 um, intensities 1e21..1e24 W/cm^2
(a0 = 0.86 sqrt(I_18)).  The prescribed-field workloads below keep that setup
and use the charge states and densities of the five configurations this
implementation is measured on.
"""
from __future__ import annotations

import numpy as np

LAMBDA = 1e-6
AL = dict(Z=13.0, charge_state=11.0)
AU = dict(Z=79.0, charge_state=51.0)


def a0_of(I_wcm2: float) -> float:
    """a0 = 0.855 lambda_um sqrt(I / 1e18 W/cm^2) (Sec. 3 quotes 0.86 at 1 um)."""
    return 0.855 * np.sqrt(I_wcm2 / 1e18)


def tables_small():
    """Tables of the 1D Al case: 128 x 128 (eta 1e-4..1e2)."""
    return dict(n_eta=128, n_y=128, eta_min=1e-4, eta_max=1e2, y_min=1e-6, y_max=1e2, n_E=128, n_s=128,
                gamma_min=2.0, gamma_max=1e6, photon_min_mc2=1.0)


def tables_large():
    """Tables of the Au and 2D cases: 256 x 256."""
    d = tables_small()
    d.update(n_eta=256, n_y=256, n_E=256, n_s=256)
    return d


def base_run(**kw) -> dict:
    d = dict(a0=27.0, lambda_m=LAMBDA, polarisation=0, geometry=0, w0_m=3e-6, focus_x_m=2e-6, flat_s=30e-15,
             ramp_periods=1.0, ne_over_nc=50.0, slab_x0_m=2e-6, slab_thick_m=1e-6, y_half_m=3e-6,
             dt_over_T=0.01, init_dist=0, T_mev=1.0, beam_gamma=1.0, seed=0, run_id=0, enable_ncs=1,
             enable_brems=1, box_enable=0)
    d.update(AL)
    d.update(kw)
    return d


def config1() -> dict:
    """1D LP plane wave, a0 = 27 (1e21 W/cm^2), Al 11+, 1 um slab, n_e = 50 n_c; 1e4 electrons at rest,
    dt = T/100, 2000 steps, FP64, 128 x 128 tables, seed 0."""
    return dict(name="1d-lp-a27-al11-1e4x2000", n=10_000, steps=2000, tables=tables_small(), Z=(13.0,),
                run=base_run(a0=27.0))


def config2() -> dict:
    """Same 1D setup on Au 51+, a0 = 270 (1e23 W/cm^2), 1e6 electrons with Maxwell-Juttner T = 1 MeV,
    4000 steps, 256 x 256 tables."""
    return dict(name="1d-lp-a270-au51-mj1mev-1e6x4000", n=1_000_000, steps=4000, tables=tables_large(),
                Z=(79.0,), run=base_run(a0=270.0, init_dist=1, T_mev=1.0, **AU))


def config3() -> dict:
    """2D paraxial Gaussian focus w0 = 3 lambda at the slab front, CP with a0 = 855 per component,
    Au 2 um slab (|y| <= 3 um), 3e7 electrons at rest, 2000 steps, photon buffer 2e8."""
    return dict(name="2d-gauss-cp-a855-au51-3e7x2000", n=30_000_000, steps=2000, tables=tables_large(),
                Z=(79.0,), capacity=200_000_000,
                run=base_run(a0=855.0, polarisation=1, geometry=1, w0_m=3e-6, focus_x_m=2e-6,
                             slab_thick_m=2e-6, y_half_m=3e-6, **AU))


def config4(seed: int = 0) -> dict:
    """64 runs: I_k = 10^(21 + 3k/63) W/cm^2 LP 1D, Al 11+ (even k) / Au 51+ (odd k), 1 um slabs,
    n_e = 50 n_c, N_k = clip(lognormal(median 2e5, sigma 1), 1e4, 4e6), 1000 steps."""
    rng = np.random.default_rng(seed)
    n = np.clip(np.round(np.exp(np.log(2e5) + rng.standard_normal(64))), 1e4, 4e6).astype(np.int64)
    runs = []
    for k in range(64):
        I = 10.0 ** (21 + 3 * k / 63)
        tgt = AL if k % 2 == 0 else AU
        runs.append(base_run(a0=a0_of(I), run_id=k, **tgt))
    return dict(name="batch64-lp-1e21..1e24-al/au-lognormal-x1000", n=n, steps=1000, tables=tables_large(),
                Z=(13.0, 79.0), runs=runs)


def config5(rate_hz: float = 50.0, n_requests: int = 600, seed: int = 5) -> dict:
    """Serving trace: Poisson arrivals; geometry of config 3, intensity and target drawn as in config 4;
    N log-uniform in [1e4, 1e7]; steps uniform in [500, 4000]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    reqs = []
    for i in range(n_requests):
        k = int(rng.integers(0, 64))
        I = 10.0 ** (21 + 3 * k / 63)
        tgt = AL if k % 2 == 0 else AU
        n = int(np.exp(rng.uniform(np.log(1e4), np.log(1e7))))
        steps = int(rng.integers(500, 4001))
        run = base_run(a0=a0_of(I / 2.0), polarisation=1, geometry=1, w0_m=3e-6, focus_x_m=2e-6,
                       slab_thick_m=2e-6, y_half_m=3e-6, run_id=i, seed=1000 + i, **tgt)
        reqs.append(dict(arrival_s=float(t[i]), n=n, steps=steps, run=run))
    return dict(name=f"serve-poisson{rate_hz:g}hz-{n_requests}req", requests=reqs, tables=tables_large(),
                Z=(13.0, 79.0))


def bunch(E0_mev: float, target: str, thickness_m: float = 5e-3, n: int = 100_000, dt_over_T: float = 1.0) -> dict:
    """The paper's own brems benchmark (Sec. 2.2): a mono-energetic electron bunch normally incident on
    5 mm of Au (19.3 g/cc) or Al (2.70 g/cc), fields off, pusher + bremsstrahlung only.  Fully ionised
    densities as in Sec. 3 (n_e ~ 4177 / 711 n_c).  Steps cover the slab at v ~ c."""
    if target == "Au":
        tgt = dict(Z=79.0, charge_state=79.0, ne_over_nc=4177.0)
    else:
        tgt = dict(Z=13.0, charge_state=13.0, ne_over_nc=711.0)
    gamma = E0_mev / 0.51099895 + 1.0
    steps = int(np.ceil(thickness_m / (LAMBDA * dt_over_T)))
    run = base_run(a0=0.0, geometry=2, init_dist=2, beam_gamma=gamma, slab_x0_m=0.0, slab_thick_m=thickness_m,
                   dt_over_T=dt_over_T, enable_ncs=0, seed=77, **tgt)
    return dict(name=f"bunch-{E0_mev:g}MeV-{target}-{thickness_m * 1e3:g}mm", n=n, steps=steps,
                tables=tables_small(), Z=(13.0, 79.0), run=run)


PHOTON_RECORD = np.dtype([("x", "<f4"), ("y", "<f4"), ("energy", "<f4"), ("kx", "<f4"), ("ky", "<f4"),
                          ("kz", "<f4"), ("step", "<u4"), ("id_mech", "<u4")])


def synthetic_photons(n: int, seed: int, x_range, k_range, step_range, theta_max: float = 0.3,
                      y_half: float = 0.0, mech_frac: float = 0.5) -> np.ndarray:
    """Seeded photon records (the 32-byte layout of the photon buffer) for the pair-production
    tests: emission points uniform in x_range (c/omega units) and, if y_half > 0, in |y| < y_half;
    energies log-uniform over k_range (m c^2); directions uniform in a cone of half-angle
    theta_max about +x (a fraction reversed to -x); emission steps uniform over step_range;
    distinct parent ids and a mechanism bit."""
    rng = np.random.default_rng(seed)
    p = np.zeros(n, dtype=PHOTON_RECORD)
    p["x"] = rng.uniform(x_range[0], x_range[1], n)
    p["y"] = rng.uniform(-y_half, y_half, n) if y_half > 0 else 0.0
    p["energy"] = np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1]), n))
    ct = rng.uniform(np.cos(theta_max), 1.0, n)
    st = np.sqrt(1.0 - ct * ct)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    back = rng.uniform(0.0, 1.0, n) < 0.1
    p["kx"] = np.where(back, -ct, ct)
    p["ky"] = st * np.cos(ph)
    p["kz"] = st * np.sin(ph)
    p["step"] = rng.integers(step_range[0], step_range[1], n)
    mech = (rng.uniform(0.0, 1.0, n) < mech_frac).astype(np.uint32)
    p["id_mech"] = rng.permutation(n).astype(np.uint32) | (mech << np.uint32(31))
    return p

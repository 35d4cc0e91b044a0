"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

FP64 path: identical event lists, per-particle state to 1e-9 relative (the two
sides build their tables with different quadrature rules; table values agree to
~1e-12 and interpolated rates to ~1e-10, the rest is rounding order).  FP32
path: per-particle state within the FP32 bound below on particles whose event
fingerprint matches the oracle's, a bounded fraction of legitimate event flips,
and the photon spectrum statistically equal (chi-square).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F64_RTOL = 1e-9
# FP32 state error where events match, relative to the trajectory's momentum scale
# max(|u|, a0) (the quiver amplitude; |u| itself passes near zero at the nodes of the
# vector potential).  Positions and optical depths are compensated float pairs, so the
# remaining error is the FP32 rounding of each step's momentum update (~1e-7).
F32_RTOL = 1e-5
# On the 1D Au a0 = 270 workload the time step T/100 does not resolve the passages
# through the nodes of the vector potential at gamma ~ 5, where one step changes u by
# ~8: the discrete map is ill-conditioned there (the FP64 oracle itself breaks the
# plane-wave invariant gamma - u_x by ~10 % in such a step; see the oracle pins).  For that
# workload the bound is the oracle's own response to FP32-sized rounding:
# tests/golden/fp32_error_model.txt holds, for the FP64 oracle whose momenta are perturbed by up
# to one FP32 ulp after every step, the event-match fraction and the fraction of matched
# electrons below each error threshold (momentum, position, optical depth).  The FP32 path
# must do no worse at any threshold, within 3 sigma of the two binomial estimates.
WELL_RESOLVED = {"1d-al-a27-rest", "2d-au-a855-cp"}
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fp32_error_model.txt")
THRESHOLDS = (1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2)


def fp32_model(case):
    rows = {}
    for ln in open(MODEL_PATH):
        if ln.startswith("#") or not ln.strip():
            continue
        p = ln.split()
        if p[0] == case:
            rows[p[1]] = dict(n=int(p[2]), match=float(p[3]), frac=np.array([float(v) for v in p[4:]]))
    return rows


def _sig(f, n):
    # binomial variance at (k + 1/2) / (n + 1), so that a fraction of 0 or 1 still carries sampling noise
    q = (f * n + 0.5) / (n + 1.0)
    return q * (1.0 - q) / max(n, 1)


def assert_no_worse_than_model(case, match, errs, n_total):
    """FP32 event-match fraction and error CDFs (u, x, tau over matched electrons) against the
    oracle's per-step one-ulp model of the same electrons, threshold by threshold."""
    model = fp32_model(case)
    n_model_total = round(model["u"]["n"] / model["u"]["match"])
    m = match.mean()
    sig = math.sqrt(_sig(model["u"]["match"], n_model_total) + _sig(m, n_total))
    assert m >= model["u"]["match"] - 3 * sig, ("event match", m, model["u"]["match"])
    for q, e in errs.items():
        for t, fm in zip(THRESHOLDS, model[q]["frac"]):
            fg = float(np.mean(e < t))
            sig = math.sqrt(_sig(fm, model[q]["n"]) + _sig(fg, len(e)))
            assert fg >= fm - 3 * sig, (q, t, fg, fm)


def state_errors(st, st_o, a0):
    """Relative FP32 errors per electron: momentum (scale max(|u|, a0)), position (max(|x|, 1)),
    optical depth (max(|tau|, 1)); the definitions of the model file."""
    eu = np.abs(st[:, 2:5] - st_o[:, 2:5]).max(1) / np.maximum(np.abs(st_o[:, 2:5]).max(1), a0)
    ex = np.abs(st[:, 0:2] - st_o[:, 0:2]).max(1) / np.maximum(np.abs(st_o[:, 0:2]).max(1), 1.0)
    et = np.abs(st[:, 5] - st_o[:, 5]) / np.maximum(np.abs(st_o[:, 5]), 1.0)
    return eu, ex, et


def assert_yields_within_flips(tal, tal_o, ev, ev_o):
    """Photon counts against the oracle's on the same electrons and draws: an electron whose event
    word matches emitted the same numbers of NCS and brems photons, so each total differs exactly
    by the emissions of the electrons whose words differ; the stored/below-cut split can further
    differ only for photons within FP32 rounding of the 1 m c^2 cut (at most 2 here)."""
    ev, ev_o = ev.astype(np.uint64), ev_o.astype(np.uint64)
    mis = ev != ev_o
    for mech, (st_k, bl_k) in enumerate((("N_NCS_STORED", "N_NCS_BELOW"), ("N_BR_STORED", "N_BR_BELOW"))):
        sh = np.uint64(16 * mech)
        cg = ((ev >> sh) & np.uint64(0xFFFF)).astype(np.int64)
        co = ((ev_o >> sh) & np.uint64(0xFFFF)).astype(np.int64)
        tot_g = int(tal[pe.T[st_k]]) + int(tal[pe.T[bl_k]])
        tot_o = int(tal_o[O.T[st_k]]) + int(tal_o[O.T[bl_k]])
        assert tot_g == int(cg.sum()) and tot_o == int(co.sum()), (st_k, "totals against event words")
        assert tot_g - tot_o == int((cg - co)[mis].sum()), st_k
        flips = int((cg + co)[mis].sum())
        assert abs(int(tal[pe.T[st_k]]) - int(tal_o[O.T[st_k]])) <= flips + 2, (st_k, flips)


_TAB = {}


def _tp(n=48, **kw):
    d = W.tables_small()
    d.update(n_eta=n, n_y=n, n_E=n, n_s=n)
    d.update(kw)
    return d


def tables(tp, Z):
    key = (tuple(sorted(tp.items())), tuple(Z))
    if key not in _TAB:
        lt = pe.pe_create_tables(tp, Z)
        op = {("photon_min" if k == "photon_min_mc2" else k): v for k, v in tp.items()}
        ot = O.Tables(O.table_params(**op), list(Z))
        _TAB[key] = (lt, ot)
    return _TAB[key]


def orun(run: dict, Z):
    d = dict(run)
    d.pop("precision", None)
    d.pop("id0", None)                  # the oracle takes the global ids themselves
    d["iz"] = list(Z).index(d["Z"])
    return O.run_params(**d)


def run_oracle(ot, run, Z, ids, steps, step0=0, state=None, wait=None):
    """Oracle run; for the null-collision method ``wait`` (uint32 per particle) carries the
    candidate waits (filled at init when ``state`` is None)."""
    rp = orun(run, Z)
    if wait is None and rp.brems_method == pe.PE_BREMS_NULL:
        wait = np.zeros(len(ids), dtype=np.uint32)
    st = O.init(ot, rp, ids, wait=wait) if state is None else state
    ev = np.zeros(len(ids), dtype=np.uint64)
    ph, nph, hist, tally = O.run(ot, rp, ids, st, step0, steps, capacity=1 << 22, events=ev, wait=wait)
    return st, ph, nph, hist, tally, ev


def run_gpu(lt, run, n, steps, precision, capacity=1 << 22, **launch):
    r = pe.Run(lt, pe.run_params(precision=precision, **run), n, capacity=capacity, events=True)
    if launch:
        pe.pe_step_ex([r.handle], steps, **launch)
    else:
        pe.pe_step([r.handle], steps)
    out = r.tally_out()
    return r, out


def photon_keys(ph):
    return np.sort(ph["id_mech"].astype(np.uint64) << np.uint64(32) | ph["step"].astype(np.uint64))


def sort_photons(ph):
    k = ph["id_mech"].astype(np.uint64) << np.uint64(32) | ph["step"].astype(np.uint64)
    return ph[np.argsort(k, kind="stable")]


def fx(t, k):
    return pe.fixed_to_float(np.asarray(t, dtype=np.uint64), pe.T[k])


# ------------------------------------------------------------------ tables ----
@pytest.mark.parametrize("n", [33, 128])
def test_tables_match_oracle(n):
    tp = _tp(n)
    lt, ot = tables(tp, (13.0, 79.0))
    np.testing.assert_allclose(pe.pe_tables_export(lt, 0), ot.export(0), rtol=1e-10)
    np.testing.assert_allclose(pe.pe_tables_export(lt, 1), ot.export(1).ravel(), rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(pe.pe_tables_export(lt, 2), ot.export(2), rtol=1e-9, atol=1e-13)
    for iz in (0, 1):
        np.testing.assert_allclose(pe.pe_tables_export(lt, 3, iz), ot.export(3, iz), rtol=1e-9, atol=1e-300)
        np.testing.assert_allclose(pe.pe_tables_export(lt, 4, iz), ot.export(4, iz).ravel(), rtol=1e-9, atol=1e-13)


# -------------------------------------------------------------------- init ----
@pytest.mark.parametrize("kind", ["rest", "mj", "beam", "2d"])
def test_init_matches_oracle(kind):
    tp = _tp(33)
    Z = (13.0, 79.0)
    lt, ot = tables(tp, Z)
    run = W.base_run(seed=17, run_id=3)
    if kind == "mj":
        run.update(init_dist=1, T_mev=1.0, **W.AU)
    if kind == "beam":
        run.update(init_dist=2, beam_gamma=200.0)
    if kind == "2d":
        run.update(geometry=1, polarisation=1, slab_thick_m=2e-6)
    n = 1000
    st_o = O.init(ot, orun(run, Z), np.arange(n))
    for prec in (pe.PE_F64, pe.PE_F32):
        r = pe.Run(lt, pe.run_params(precision=prec, **run), n)
        st = r.state()
        if prec == pe.PE_F64:
            # rounding order (FMA contraction) leaves ~1e-15 absolute on coordinates near zero
            np.testing.assert_allclose(st, st_o, rtol=1e-14, atol=1e-13)
        else:
            # positions and tau are float pairs (exact to ~2^-48), momenta plain floats
            np.testing.assert_allclose(st[:, [0, 1, 5]], st_o[:, [0, 1, 5]], rtol=1e-14, atol=1e-13)
            np.testing.assert_array_equal(st[:, 2:5], st_o[:, 2:5].astype(np.float32).astype(np.float64))
        r.close()


# ------------------------------------------------------------- FP64 parity ----
CASES = {
    # config 2 physics (Au 51+, a0 = 270, MJ 1 MeV) on a ragged particle count
    "1d-au-a270-mj": (dict(a0=270.0, init_dist=1, T_mev=1.0, seed=2, **W.AU), 1000, 1500),
    # config 1 physics (Al 11+, a0 = 27, at rest)
    "1d-al-a27-rest": (dict(a0=27.0, seed=0), 777, 2000),
    # config 3 physics (2D Gaussian focus, CP a0 = 855, Au 2 um slab)
    "2d-au-a855-cp": (dict(a0=855.0, polarisation=1, geometry=1, slab_thick_m=2e-6, seed=4, **W.AU), 600, 900),
    # dense fields-off target: brems-dominated (Sec. 2.2 benchmark mode)
    "beam-au-brems": (dict(a0=0.0, init_dist=2, beam_gamma=2000.0, ne_over_nc=2e4, slab_x0_m=-1e-3,
                           slab_thick_m=2e-3, enable_ncs=0, seed=9, **W.AU), 500, 800),
    # the paper's bunch benchmark: 100 MeV into 5 mm of fully ionised Au, fields off (Sec. 2.2)
    "bunch-100mev-au-5mm": (dict(W.bunch(100.0, "Au")["run"]), 300, 5000),
    # the same 1 GeV bunch with null-collision brems (majorant candidates, P/P_hat thinning)
    "bunch-1gev-au-5mm-null": (dict(W.bunch(1000.0, "Au")["run"], brems_method=1), 300, 5000),
    # null collisions in the dense fields-off target and under the 1D plane wave (paired kernel)
    "beam-au-brems-null": (dict(a0=0.0, init_dist=2, beam_gamma=2000.0, ne_over_nc=2e4, slab_x0_m=-1e-3,
                                slab_thick_m=2e-3, enable_ncs=0, seed=9, brems_method=1, **W.AU), 1000, 1000),
    "1d-au-a270-dense-null": (dict(a0=270.0, init_dist=1, T_mev=1.0, seed=12, brems_method=1, slab_thick_m=20e-6,
                                   **dict(W.AU, ne_over_nc=2e4)), 1000, 1500),
    # reflected wave: the a0 = 270 pulse reflected by a mirror at the slab's rear face (eta ~ 1).  The
    # standing wave is chaotic (the oracle pin: in LP a 2^-50 perturbation reaches O(1) by step ~900),
    # so per-particle parity runs to the horizon where a 1e-15 perturbation stays below ~1e-11
    # (LP 400 steps, CP r = 0.8 700 steps); the FP32 statistics run longer (test_gpu_variants)
    "1d-au-a270-refl-lp": (dict(a0=270.0, init_dist=1, T_mev=1.0, seed=2, reflect_r=1.0, mirror_x_m=3e-6,
                                **W.AU), 1000, 400),
    "1d-au-a270-refl-cp": (dict(a0=270.0, polarisation=1, init_dist=1, T_mev=1.0, seed=3, reflect_r=0.8,
                                mirror_x_m=3e-6, **W.AU), 700, 700),
}


@pytest.mark.parametrize("case", list(CASES))
def test_f64_parity(case):
    runkw, n, steps = CASES[case]
    run = W.base_run(**runkw)
    Z = (13.0, 79.0)
    lt, ot = tables(_tp(48), Z)
    wait_o = np.zeros(n, dtype=np.uint32) if run.get("brems_method") else None
    st_o, ph_o, nph_o, hist_o, tal_o, ev_o = run_oracle(ot, run, Z, np.arange(n), steps, wait=wait_o)
    r, out = run_gpu(lt, run, n, steps, pe.PE_F64)
    st = r.state()
    ev = r.event_words()
    assert np.array_equal(ev, ev_o), f"{np.sum(ev != ev_o)} particles with different event lists"
    np.testing.assert_allclose(st[:, [0, 1, 5]], st_o[:, [0, 1, 5]], rtol=F64_RTOL, atol=1e-9)
    # momenta relative to each electron's momentum scale (a small component of a large u carries
    # the rounding of |u|)
    scale_u = np.maximum(np.abs(st_o[:, 2:5]).max(1), 1.0)
    assert (np.abs(st[:, 2:5] - st_o[:, 2:5]).max(1) / scale_u).max() < F64_RTOL
    if wait_o is not None:
        np.testing.assert_array_equal(r.wait_words(), wait_o)
    tal = np.frombuffer(bytes(out.tally), dtype=np.uint64)
    for k in ("N_NCS_STORED", "N_NCS_BELOW", "N_BR_STORED", "N_BR_BELOW", "N_PHOTONS", "N_ETA_ABOVE",
              "N_ETA_BELOW", "N_GAMMA_ABOVE", "N_CLAMP"):
        assert tal[pe.T[k]] == tal_o[O.T[k]], k
    for k in ("E_NCS_STORED", "E_NCS_BELOW", "E_BR_STORED", "E_RECOIL_NCS", "E_RECOIL_BR"):
        a, b = fx(tal, k), O.fixed_to_float(tal_o, O.T[k])
        assert abs(a - b) <= 1e-9 * max(abs(b), 1e-300), k
    ph = sort_photons(r.photon_records())
    pho = sort_photons(ph_o)
    assert len(ph) == len(pho) == nph_o
    np.testing.assert_array_equal(ph["id_mech"], pho["id_mech"])
    np.testing.assert_array_equal(ph["step"], pho["step"])
    for f in ("x", "y", "energy", "kx", "ky", "kz"):
        np.testing.assert_allclose(ph[f], pho[f], rtol=1e-6, atol=1e-6)
    hist = np.frombuffer(bytes(out.hist), dtype=np.uint64)
    assert np.abs(hist.astype(np.int64) - hist_o.astype(np.int64)).sum() <= 2   # bin-edge ties only
    # energy bookkeeping: electron recoil energy = photon energy emitted (1e-12)
    emitted = sum(fx(tal, k) for k in ("E_NCS_STORED", "E_NCS_BELOW", "E_BR_STORED", "E_BR_BELOW"))
    recoil = fx(tal, "E_RECOIL_NCS") + fx(tal, "E_RECOIL_BR")
    if emitted > 0:
        assert abs(recoil / emitted - 1) < 1e-12
    r.close()


@pytest.mark.parametrize("case", ["1d-au-a270-mj", "2d-au-a855-cp", "1d-au-a270-refl-cp", "beam-au-brems-null"])
def test_f64_persistent_equals_plain(case):
    """The FP64 plain kernel (one step per launch, global atomics) and the FP64 persistent kernel
    (K steps per launch in registers, shared-memory accumulators) round every operation alike
    (their translation unit contracts no multiply-add), so they agree bit for bit: state, event
    words, every tally word, histograms and photon records."""
    runkw, n, steps = CASES[case]
    run = W.base_run(**runkw)
    lt, _ = tables(_tp(48), (13.0, 79.0))
    a = pe.Run(lt, pe.run_params(precision=pe.PE_F64, **run), n, events=True)
    b = pe.Run(lt, pe.run_params(precision=pe.PE_F64, **run), n, events=True)
    pe.pe_step([a.handle], steps)
    pe.pe_step_ex([b.handle], steps, block=128, steps_per_launch=37)
    np.testing.assert_array_equal(a.state(), b.state())
    np.testing.assert_array_equal(a.event_words(), b.event_words())
    if a.wait is not None:
        np.testing.assert_array_equal(a.wait_words(), b.wait_words())
    ta, tb = a.tally_out(), b.tally_out()
    assert bytes(ta.tally) == bytes(tb.tally) and bytes(ta.hist) == bytes(tb.hist)
    np.testing.assert_array_equal(sort_photons(a.photon_records()), sort_photons(b.photon_records()))


# ------------------------------------------------------------- FP32 parity ----
@pytest.mark.parametrize("case", ["1d-au-a270-mj", "1d-al-a27-rest", "2d-au-a855-cp"])
def test_f32_parity(case):
    runkw, n, steps = CASES[case]
    run = W.base_run(**runkw)
    Z = (13.0, 79.0)
    lt, ot = tables(_tp(48), Z)
    st_o, ph_o, nph_o, hist_o, tal_o, ev_o = run_oracle(ot, run, Z, np.arange(n), steps)
    r, out = run_gpu(lt, run, n, steps, pe.PE_F32)
    st = r.state()
    ev = r.event_words()
    match = ev == ev_o
    frac = match.mean()
    eu, ex, et = state_errors(st, st_o, max(run["a0"], 1.0))
    err_u, err_x, err_t = eu[match], ex[match], et[match]
    print(f"{case}: event match {frac:.4f}, max rel err u {err_u.max():.2e} x {err_x.max():.2e} tau {err_t.max():.2e}, "
          f"within {F32_RTOL:g}: u {np.mean(err_u < F32_RTOL):.3f} x {np.mean(err_x < F32_RTOL):.3f} "
          f"tau {np.mean(err_t < F32_RTOL):.3f}, median u {np.median(err_u):.2e}")
    if case in WELL_RESOLVED:
        assert frac > 0.9
        assert err_u.max() < F32_RTOL and err_x.max() < F32_RTOL
    else:
        assert_no_worse_than_model("small", match, dict(u=err_u, x=err_x, tau=err_t), n)
    assert_yields_within_flips(np.frombuffer(bytes(out.tally), dtype=np.uint64), tal_o, ev, ev_o)
    r.close()


def test_f32_spectrum_chi2():
    # NCS photon spectra of FP32 GPU and FP64 oracle from independent seeds agree (chi-square)
    from scipy.stats import chi2
    run = W.base_run(a0=270.0, init_dist=1, T_mev=1.0, **W.AU)
    Z = (13.0, 79.0)
    lt, ot = tables(_tp(48), Z)
    n, steps = 24000, 1200
    _, _, _, hist_o, _, _ = run_oracle(ot, dict(run, seed=101), Z, np.arange(n), steps)
    r, out = run_gpu(lt, dict(run, seed=202), n, steps, pe.PE_F32)
    h1 = np.frombuffer(bytes(out.hist), dtype=np.uint64)[:512].astype(float)
    h2 = hist_o[:512].astype(float)
    # merge sparse bins from the top so every merged bin holds >= 10 counts in the sum
    m1, m2, a, b = [], [], 0.0, 0.0
    for x, y in zip(h1, h2):
        a += x; b += y
        if a + b >= 20:
            m1.append(a); m2.append(b); a = b = 0.0
    if a + b > 0 and m1:
        m1[-1] += a; m2[-1] += b
    m1, m2 = np.array(m1), np.array(m2)
    assert m1.sum() > 1000 and m2.sum() > 1000
    k1, k2 = math.sqrt(m2.sum() / m1.sum()), math.sqrt(m1.sum() / m2.sum())
    stat = np.sum((k1 * m1 - k2 * m2) ** 2 / (m1 + m2))
    p = chi2.sf(stat, len(m1) - 1)
    print(f"chi2 {stat:.1f} dof {len(m1) - 1} p {p:.3g}")
    assert p > 1e-3
    r.close()


# ---------------------------------------------------- batching invariance ----
def test_f32_batch_equals_alone():
    Z = (13.0, 79.0)
    lt, _ = tables(_tp(48), Z)
    runs = [W.base_run(a0=270.0, init_dist=1, seed=1, run_id=0, **W.AU),
            W.base_run(a0=27.0, seed=2, run_id=1),
            W.base_run(a0=855.0, polarisation=1, geometry=1, slab_thick_m=2e-6, seed=3, run_id=2, **W.AU)]
    sizes = [1000, 77, 513]
    alone = []
    for run, n in zip(runs, sizes):
        r = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **run), n, events=True)
        pe.pe_step([r.handle], 400)
        alone.append(r)
    mix = [pe.Run(lt, pe.run_params(precision=pe.PE_F32, **run), n, events=True) for run, n in zip(runs, sizes)]
    pe.pe_step_ex([m.handle for m in mix], 400, block=128, steps_per_launch=100)
    for a, m in zip(alone, mix):
        np.testing.assert_array_equal(a.state(), m.state())
        np.testing.assert_array_equal(a.event_words(), m.event_words())
        ta, tm = a.tally_out(), m.tally_out()
        assert bytes(ta.tally) == bytes(tm.tally)
        assert bytes(ta.hist) == bytes(tm.hist)
        np.testing.assert_array_equal(photon_keys(a.photon_records()), photon_keys(m.photon_records()))


@pytest.mark.parametrize("case", ["1d-au-a270-mj", "1d-au-a270-refl-lp", "1d-au-a270-refl-cp", "2d-au-a855-cp"])
def test_f32_step_split_invariance(case):
    """The paired kernel's state is exact across launch boundaries and tile shapes: K = 600, 1 and 7
    (tiles of 64 electrons) give the same state, events and tallies, for every kind it steps (the
    plane wave, the reflected wave with its one emission site per lane, the 2D focus).  K = 1 on a
    single plane-wave run takes the one-step streaming form."""
    lt, _ = tables(_tp(48), (13.0, 79.0))
    runkw = dict(a0=270.0, init_dist=1, seed=8, **W.AU) if case == "1d-au-a270-mj" else CASES[case][0]
    run = W.base_run(**runkw)
    outs = []
    for cfg in (dict(steps_per_launch=600), dict(steps_per_launch=1), dict(steps_per_launch=7, block=64)):
        r = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **run), 900, events=True)
        pe.pe_step_ex([r.handle], 300, **cfg)
        pe.pe_step_ex([r.handle], 300, **cfg)
        outs.append((r.state(), r.event_words(), bytes(r.tally_out().tally)))
    assert int(np.sum(outs[0][1] != 0)) > 0          # emissions happened
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
        assert o[2] == outs[0][2]


@pytest.mark.parametrize("ctas_per_sm", [1, None])
def test_f32_streaming_form_many_tiles(ctas_per_sm):
    """The streaming one-step form (launches of <= 4 steps on one run: each CTA stages its
    256-electron tiles through shared memory with bulk copies, the next tile in flight) walks
    many tiles per CTA, with a ragged last one: its result equals the register-resident
    kernel's bit for bit, photons included."""
    lt, _ = tables(_tp(48), (13.0, 79.0))
    run = W.base_run(a0=270.0, init_dist=1, seed=12, **W.AU)
    n = 300_007
    outs = []
    for cfg in (dict(steps_per_launch=12), dict(steps_per_launch=1, ctas_per_sm=ctas_per_sm),
                dict(steps_per_launch=3, ctas_per_sm=ctas_per_sm)):
        cfg = {k: v for k, v in cfg.items() if v is not None}
        r = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **run), n, capacity=1 << 22)
        pe.pe_step_ex([r.handle], 12, **cfg)
        out = r.tally_out()
        outs.append((r.state(), photon_keys(r.photon_records()), bytes(out.tally), bytes(out.hist)))
        r.close()
    assert np.isfinite(outs[0][0]).all() and len(outs[0][1]) > 0
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
        assert o[2] == outs[0][2] and o[3] == outs[0][3]


# -------------------------------------------------------------- edge cases ----
def test_edge_cases():
    Z = (13.0, 79.0)
    lt, ot = tables(_tp(33), Z)
    run = W.base_run(a0=270.0, init_dist=1, seed=3, **W.AU)
    # empty run
    for prec in (pe.PE_F64, pe.PE_F32):
        r = pe.Run(lt, pe.run_params(precision=prec, **run), 0)
        pe.pe_step([r.handle], 10)
        out = r.tally_out()
        assert out.steps_done == 10 and out.tally[pe.T["N_PHOTONS"]] == 0
        r.close()
    # one particle
    st_o, *_ = run_oracle(ot, run, Z, np.arange(1), 300)
    r, _ = run_gpu(lt, run, 1, 300, pe.PE_F64)
    np.testing.assert_allclose(r.state(), st_o, rtol=F64_RTOL, atol=1e-9)
    # photon buffer overflow: status, exact counts, nothing written past capacity
    big, ob = run_gpu(lt, run, 800, 600, pe.PE_F32)
    small = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **run), 800, capacity=3)
    pe.pe_step([small.handle], 600)
    os_ = small.tally_out()
    assert ob.tally[pe.T["N_PHOTONS"]] > 3
    assert os_.status == pe.PE_ERR_BUFFER_FULL
    assert bytes(os_.tally) == bytes(ob.tally)
    assert os_.photons_stored == 3
    assert np.all(small.photons[3 * 8:].cpu().numpy() == 0)
    for cap in (0, 1):                                   # no room, or room for one record
        tiny = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **run), 800, capacity=cap)
        pe.pe_step([tiny.handle], 600)
        ot_ = tiny.tally_out()
        assert ot_.status == pe.PE_ERR_BUFFER_FULL and bytes(ot_.tally) == bytes(ob.tally)
        assert ot_.photons_stored == cap
        assert np.all(tiny.photons[cap * 8:].cpu().numpy() == 0)
        tiny.close()
    # a device wait that ran out (injected on the host as the tally word the kernel would set)
    # makes pe_tally report PE_ERR_TIMEOUT
    small.tally[pe.T["N_WAIT_TIMEOUT"]] = 1
    with pytest.raises(pe.PeError) as e:
        small.tally_out()
    assert e.value.status == pe.PE_ERR_TIMEOUT
    # bad arguments
    with pytest.raises(pe.PeError) as e:
        pe.Run(lt, pe.run_params(precision=7, **run), 10)
    assert e.value.status == pe.PE_ERR_ARG
    with pytest.raises(pe.PeError) as e:
        pe.Run(lt, pe.run_params(precision=pe.PE_F32, **dict(run, Z=26.0)), 10)
    assert e.value.status == pe.PE_ERR_ARG
    a = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **run), 10)
    b = pe.Run(lt, pe.run_params(precision=pe.PE_F64, **run), 10)
    with pytest.raises(pe.PeError) as e:
        pe.pe_step([a.handle, b.handle], 1)
    assert e.value.status == pe.PE_ERR_STATE
    with pytest.raises(pe.PeError) as e:
        pe.pe_create_tables(dict(_tp(33), n_eta=1), Z)
    assert e.value.status == pe.PE_ERR_ARG


def test_absorbing_box_accounting():
    Z = (13.0, 79.0)
    lt, ot = tables(_tp(33), Z)
    run = W.base_run(a0=100.0, seed=6, box_enable=1, box_x_m=(1.9e-6, 3.5e-6))
    n, steps = 500, 600
    st_o, ph_o, nph_o, hist_o, tal_o, ev_o = run_oracle(ot, run, Z, np.arange(n), steps)
    r, out = run_gpu(lt, run, n, steps, pe.PE_F64)
    assert out.tally[pe.T["N_KILLED"]] == tal_o[O.T["N_KILLED"]] > 0
    assert out.tally[pe.T["KILLED_STEPS"]] == tal_o[O.T["KILLED_STEPS"]]
    alive = ~np.isnan(st_o[:, 0])
    assert np.array_equal(alive, ~np.isnan(r.state()[:, 0]))
    assert out.live_particle_steps == alive.sum() * steps + int(tal_o[O.T["KILLED_STEPS"]])


# ------------------------------------------------------ full-size sampled ----
def test_config2_full_size_sampled():
    """Config 2 at full size (1e6 electrons, 256x256 tables, the whole 4000-step job) in the
    benchmark's launch shape; 256 sampled electrons advanced one by one by the oracle; momenta,
    positions and optical depths against the oracle's per-step one-ulp model of the same
    electrons."""
    c = W.config2()
    Z = c["Z"]
    lt, ot = tables(c["tables"], Z)
    steps = c["steps"]
    r, out = run_gpu(lt, c["run"], c["n"], steps, pe.PE_F32, capacity=1 << 24)
    st = r.state()
    ev = r.event_words()
    assert np.all(np.isfinite(st))
    tal = np.frombuffer(bytes(out.tally), dtype=np.uint64)
    hist = np.frombuffer(bytes(out.hist), dtype=np.uint64)
    assert hist[:512].sum() == tal[pe.T["N_NCS_STORED"]] and hist[512:1024].sum() == tal[pe.T["N_BR_STORED"]]
    ids = np.random.default_rng(0).choice(c["n"], 256, replace=False)
    st_o, _, _, _, _, ev_o = run_oracle(ot, c["run"], Z, ids, steps)
    match = ev[ids] == ev_o
    eu, ex, et = state_errors(st[ids], st_o, c["run"]["a0"])
    print(f"config 2 full size: event match {match.mean():.4f}, u median {np.median(eu[match]):.2e} "
          f"within {F32_RTOL:g}: u {np.mean(eu[match] < F32_RTOL):.3f} x {np.mean(ex[match] < F32_RTOL):.3f} "
          f"tau {np.mean(et[match] < F32_RTOL):.3f}")
    assert_no_worse_than_model("full", match, dict(u=eu[match], x=ex[match], tau=et[match]), len(ids))
    r.close()


def test_config3_full_size_sampled():
    """Config 3 at full size (3e7 electrons, 2D Gaussian focus, CP a0 = 855, 2000 steps) in the
    benchmark's launch shape; 128 sampled electrons advanced one by one by the oracle.  The 2D
    case is well resolved at dt = T/100: every electron whose events match is within F32_RTOL."""
    c = W.config3()
    Z = c["Z"]
    lt, ot = tables(c["tables"], Z)
    r, out = run_gpu(lt, c["run"], c["n"], c["steps"], pe.PE_F32, capacity=1 << 22)
    ids = np.random.default_rng(3).choice(c["n"], 128, replace=False)
    st = r.state()[ids]
    ev = r.event_words()[ids]
    r.close()
    st_o, _, _, _, _, ev_o = run_oracle(ot, c["run"], Z, ids, c["steps"])
    match = ev == ev_o
    scale = np.maximum(np.abs(st_o[:, 2:5]).max(1), c["run"]["a0"])
    err = (np.abs(st[:, 2:5] - st_o[:, 2:5]).max(1) / scale)[match]
    err_x = (np.abs(st[:, 0:2] - st_o[:, 0:2]).max(1) / np.maximum(np.abs(st_o[:, 0:2]).max(1), 1.0))[match]
    print(f"config 3 full size: event match {match.mean():.4f}, max {err.max():.2e}, x {err_x.max():.2e}")
    assert match.mean() > 0.95
    assert err.max() < F32_RTOL and err_x.max() < F32_RTOL


def test_config4_full_size_sampled():
    """Config 4 at full size (64 runs, 2.05e7 electrons, 1000 steps) advanced by one CUDA graph of
    batched launches; four sampled electrons per run advanced one by one by the oracle.  The
    batch spans a0 = 27..855 in 1D at dt = T/100, so the FP32 bound is the distributional one."""
    c = W.config4()
    Z = c["Z"]
    lt, ot = tables(c["tables"], Z)
    runs = [pe.Run(lt, pe.run_params(precision=pe.PE_F32, **rk), int(n), capacity=int(min(2 * n, 1 << 23)),
                   events=True) for rk, n in zip(c["runs"], c["n"])]
    g = pe.pe_graph_create([r.handle for r in runs], c["steps"], block=256, ctas_per_sm=15, steps_per_launch=500)
    pe.pe_graph_launch(g)
    pe.pe_graph_destroy(g)
    rng = np.random.default_rng(4)
    errs, matches = [], []
    for rk, n, r in zip(c["runs"], c["n"], runs):
        ids = rng.choice(int(n), 4, replace=False)
        st = r.state()[ids]
        ev = r.event_words()[ids]
        st_o, _, _, _, _, ev_o = run_oracle(ot, rk, Z, ids, c["steps"])
        m = ev == ev_o
        scale = np.maximum(np.abs(st_o[:, 2:5]).max(1), rk["a0"])
        errs.append((np.abs(st[:, 2:5] - st_o[:, 2:5]).max(1) / scale)[m])
        matches.append(m)
        r.close()
    err = np.concatenate(errs)
    match = np.concatenate(matches)
    print(f"config 4 full size: event match {match.mean():.4f}, median {np.median(err):.2e}, "
          f"within {F32_RTOL:g}: {np.mean(err < F32_RTOL):.3f}, p95 {np.quantile(err, 0.95):.2e}, max {err.max():.2e}")
    # the batch's runs take 1000 steps: bounded by the model of the 1500-step a0 = 270 Au case
    model = fp32_model("small")["u"]
    assert match.mean() >= model["match"] - 3 * math.sqrt(_sig(model["match"], 1000) + _sig(match.mean(), len(match)))
    for t, fm in zip(THRESHOLDS, model["frac"]):
        fg = float(np.mean(err < t))
        assert fg >= fm - 3 * math.sqrt(_sig(fm, model["n"]) + _sig(fg, len(err))), (t, fg, fm)


# ------------------------------------------------------- graph, autotune ----

def test_graph_equals_direct_steps():
    Z = (13.0, 79.0)
    lt, _ = tables(_tp(48), Z)
    runs = [W.base_run(a0=270.0, init_dist=1, seed=1, run_id=0, **W.AU),
            W.base_run(a0=27.0, seed=2, run_id=1),
            W.base_run(a0=855.0, polarisation=1, geometry=1, slab_thick_m=2e-6, seed=3, run_id=2, **W.AU)]
    sizes = [700, 300, 400]
    direct = [pe.Run(lt, pe.run_params(precision=pe.PE_F32, **rk), n, events=True) for rk, n in zip(runs, sizes)]
    pe.pe_step_ex([d.handle for d in direct], 400, block=128, steps_per_launch=50)
    graphed = [pe.Run(lt, pe.run_params(precision=pe.PE_F32, **rk), n, events=True) for rk, n in zip(runs, sizes)]
    g = pe.pe_graph_create([r.handle for r in graphed], 100, block=128, steps_per_launch=50)
    for _ in range(4):
        pe.pe_graph_launch(g)
    pe.pe_graph_destroy(g)
    for a, b in zip(direct, graphed):
        np.testing.assert_array_equal(a.state(), b.state())
        np.testing.assert_array_equal(a.event_words(), b.event_words())
        ta, tb = a.tally_out(), b.tally_out()
        assert bytes(ta.tally) == bytes(tb.tally) and bytes(ta.hist) == bytes(tb.hist)
        assert tb.steps_done == 400


def test_autotune_picks_a_shape():
    from paper_1612_07592_gb300 import autotune
    lt, _ = tables(_tp(48), (13.0, 79.0))
    rs = [pe.Run(lt, pe.run_params(precision=pe.PE_F32, **W.base_run(a0=270.0, init_dist=1, seed=9, **W.AU)), 5000)]
    space = dict(block=(128, 256), ctas_per_sm=(2, 4), steps_per_launch=(50, 200))
    cfg, res = autotune.tune(lt, rs, 200, space=space, use_cache=False)
    assert len(res) == 8 and all(ms > 0 for _, ms in res)
    assert cfg in [c for c, _ in res]
    # the runs are restored: stepping them now equals a fresh run
    fresh = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **W.base_run(a0=270.0, init_dist=1, seed=9, **W.AU)), 5000)
    pe.pe_step([rs[0].handle], 100)
    pe.pe_step([fresh.handle], 100)
    np.testing.assert_array_equal(rs[0].state(), fresh.state())


# ----------------------------------------------------------------- serving ----
def test_serving_alone_equals_mix():
    """Continuous batching: requests arrive while others are on the GPU and are admitted mid-run
    (a simulated clock of 1 ms per step makes the admission points reproducible); every iteration
    ends when the first resident run is done, so the runs share launches with changing company and
    their launch boundaries fall at different steps of their own.  Each result equals the same run
    stepped alone, bit for bit."""
    from paper_1612_07592_gb300.serve import Request, Server
    Z = (13.0, 79.0)
    lt, _ = tables(_tp(48), Z)
    kinds = [W.base_run(a0=270.0, init_dist=1, seed=11, run_id=0, **W.AU),
             W.base_run(a0=100.0, seed=12, run_id=1),
             W.base_run(a0=855.0, polarisation=1, geometry=1, slab_thick_m=2e-6, seed=13, run_id=2, **W.AU),
             W.base_run(a0=60.0, seed=14, run_id=3, **W.AU),
             W.base_run(a0=270.0, polarisation=1, init_dist=1, seed=15, run_id=4, **W.AU)]
    sizes, steps = [900, 300, 500, 257, 611], [700, 450, 333, 600, 3]
    arrivals = [0.0, 0.3, 0.55, 0.9, 1.0]
    alone = []
    for rk, n, st in zip(kinds, sizes, steps):
        r = pe.Run(lt, pe.run_params(precision=pe.PE_F32, **rk), n, capacity=1 << 16, events=True)
        pe.pe_step([r.handle], st)
        alone.append((r.state(), r.event_words(), bytes(r.tally_out().tally), bytes(r.tally_out().hist)))
        r.close()
    reqs = [Request(arrival_s=t, n=n, steps=st, run=rk, capacity=1 << 16)
            for t, rk, n, st in zip(arrivals, kinds, sizes, steps)]
    srv = Server(lt, steps_per_iteration=128, keep_results=True)
    stats = srv.run_trace(reqs, realtime=False, virtual_step_s=1e-3)
    assert stats.summary()["requests"] == len(reqs) and stats.max_resident >= 3
    mid = [q for q in reqs if q.resident_at_admission > 0 and q.admitted_iteration > 0]
    assert len(mid) >= 3, [(q.admitted_iteration, q.resident_at_admission) for q in reqs]
    offsets = {tuple(b % 128 for b in q.boundaries) for q in reqs}
    assert len(offsets) >= 3, [q.boundaries for q in reqs]
    for q, (st, ev, tal, hist) in zip(reqs, alone):
        assert q.boundaries[-1] == q.steps
        np.testing.assert_array_equal(q.state, st)
        np.testing.assert_array_equal(q.events, ev)
        assert bytes(q.tally.tally) == tal and bytes(q.tally.hist) == hist


def test_serving_admits_by_memory():
    from paper_1612_07592_gb300.serve import Request, Server
    lt, _ = tables(_tp(33), (13.0, 79.0))
    reqs = [Request(arrival_s=0.0, n=1000, steps=200, run=W.base_run(a0=50.0, seed=k, run_id=k)) for k in range(5)]
    need = Server.bytes_needed(reqs[0])
    budget = 2 * need + (1 << 20) + 1                    # room for two requests above the reserve
    srv = Server(lt, steps_per_iteration=100, memory_reserve_bytes=1 << 20,
                 mem_get_info=lambda: (budget - srv.resident_bytes, 1 << 40))
    stats = srv.run_trace(reqs, realtime=False)
    s = stats.summary()
    assert s["requests"] == 5 and stats.max_resident == 2
    assert s["particle_steps"] == 5 * 1000 * 200

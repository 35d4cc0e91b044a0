"""FP64 CPU oracle for the photon-emission step of arXiv:1612.07592 (Wan et al.).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It is plain C
(``oracle/*.c``) compiled with gcc and wrapped here with ctypes; it shares no
code with the CUDA library in ``paper_1612_07592_gb300``.

What it computes, step by step, is stated in ``oracle/step.c`` and
``oracle/tables.c`` with the paper section or equation each part follows.

The environment variable ``ORACLE_MUTANT`` (set only by tests/test_oracle_mutants.py,
in a child process) builds and loads the oracle with one planted mistake from
``MUTANTS`` instead, so that a test can show that the pins catch it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["tables.c", "step.c"]
# the planted mistakes step.c and tables.c know (OR_MUTANT_<name>)
MUTANTS = ("PHILOX_MULT", "BORIS_SIGN", "ETA_UE", "PHOTON_BACKWARD", "NCS_NO_GAMMA", "NCS_LAG",
           "RECOIL_TALLY", "BREMS_NO_BETA", "NCS_F_QUANTUM", "NCS_H_JACOBIAN", "BREMS_COULOMB", "BW_NORM",
           "MIRROR_SIGN", "INCIDENT_SIGN", "POSITION_NO_GAMMA", "PIC_CURRENT_SIGN", "NCS_SAMPLE_FLIP",
           "BREMS_SAMPLE_FLIP", "NULL_THINNING", "ENVELOPE_FALL", "GOUY_SIGN", "MJ_TEMPERATURE", "BH_SECOND_TERM",
           "DELTA_MAP", "WAIT_SCALE", "HIST_SHIFT", "INIT_SPREAD", "PIC_INJECT_HALF", "BW_PHOTON_STILL",
           "CHI_KE", "Y_UPDATE", "BOX_ONE_SIDED", "CURVATURE_SIGN", "AMPLITUDE", "TAU_NO_RESET", "CLAMP_GAMMA",
           "TARGET_Y", "ETA_GM", "BH_FREE_PATH", "ROW_WEIGHT", "BW_X_NODES", "REFL_SQUARED", "PIC_EX_SIGN",
           "PIC_JY_WEIGHT", "PIC_GATHER_NODE", "PIC_BY_SIGN")


def _mutant() -> str:
    m = os.environ.get("ORACLE_MUTANT", "")
    if m and m not in MUTANTS:
        raise ValueError(f"unknown ORACLE_MUTANT {m!r}")
    return m
_lock = threading.Lock()
_lib = None

HIST_E_BINS = 512
HIST_T_BINS = 180
HIST_WORDS = 2 * HIST_E_BINS + 2 * HIST_T_BINS
TALLY_WORDS = 32
T = dict(N_NCS_STORED=0, N_NCS_BELOW=1, N_BR_STORED=2, N_BR_BELOW=3, N_PHOTONS=4,
         N_ETA_ABOVE=5, N_ETA_BELOW=6, N_GAMMA_ABOVE=7, N_KILLED=8, KILLED_STEPS=9,
         N_CLAMP=10, N_HIST_OVER=11, E_NCS_STORED=16, E_NCS_BELOW=18, E_BR_STORED=20,
         E_BR_BELOW=22, E_RECOIL_NCS=24, E_RECOIL_BR=26)

PHOTON_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("energy", "<f4"), ("kx", "<f4"),
                         ("ky", "<f4"), ("kz", "<f4"), ("step", "<u4"), ("id_mech", "<u4")])
PAIR_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("e_minus", "<f4"), ("e_plus", "<f4"), ("kx", "<f4"),
                       ("ky", "<f4"), ("kz", "<f4"), ("step", "<u4"), ("photon", "<u4"), ("id_mech", "<u4")])
PAIR_TALLY_WORDS = 8
PT = dict(N_PAIRS=0, N_ENTERED=1, N_K_ABOVE=2, N_TESTS=3, E_PAIRS=4, E_POSITRONS=6)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so`` (with ORACLE_MUTANT
    set, the mutant into ``liboracle_<mutant>.so``)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "oracle.h")
    m = _mutant()
    path = os.path.join(_BUILD, f"liboracle_{m.lower()}.so") if m else _LIB_PATH
    if not force and os.path.exists(path):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(path) >= newest:
            return path
    tmp = path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c99", "-D_DEFAULT_SOURCE",
           "-ffp-contract=off", "-o", tmp] + ([f"-DOR_MUTANT_{m}"] if m else []) + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class TableParams(C.Structure):
    _fields_ = [("n_eta", C.c_int), ("n_y", C.c_int), ("eta_min", C.c_double), ("eta_max", C.c_double),
                ("y_min", C.c_double), ("y_max", C.c_double), ("n_E", C.c_int), ("n_s", C.c_int),
                ("gamma_min", C.c_double), ("gamma_max", C.c_double), ("photon_min", C.c_double)]


class RunParams(C.Structure):
    _fields_ = [("a0", C.c_double), ("lambda_m", C.c_double), ("polarisation", C.c_int),
                ("geometry", C.c_int), ("w0_m", C.c_double), ("focus_x_m", C.c_double),
                ("flat_s", C.c_double), ("ramp_periods", C.c_double),
                ("E_const", C.c_double * 3), ("B_const", C.c_double * 3),
                ("Z", C.c_double), ("charge_state", C.c_double), ("ne_over_nc", C.c_double),
                ("slab_x0_m", C.c_double), ("slab_thick_m", C.c_double), ("y_half_m", C.c_double),
                ("dt_over_T", C.c_double), ("init_dist", C.c_int), ("T_mev", C.c_double),
                ("beam_gamma", C.c_double), ("seed", C.c_uint64), ("run_id", C.c_uint32),
                ("enable_ncs", C.c_int), ("enable_brems", C.c_int), ("box_enable", C.c_int),
                ("box_x_m", C.c_double * 2), ("iz", C.c_int), ("reflect_r", C.c_double),
                ("mirror_x_m", C.c_double), ("brems_method", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            for name in ("or_bessel_k",):
                getattr(L, name).argtypes = [C.c_double, C.c_double]
                getattr(L, name).restype = C.c_double
            for name in ("or_int_k53", "or_ncs_power_integral", "or_ncs_h_direct", "or_coulomb_f",
                         "or_schwinger_field", "or_critical_density", "or_int_k13", "or_bw_T_direct"):
                getattr(L, name).argtypes = [C.c_double]
                getattr(L, name).restype = C.c_double
            L.or_bw_G.argtypes = [C.c_double, C.c_double]
            L.or_bw_G.restype = C.c_double
            L.or_chi_photon.argtypes = [dp, dp, dp, C.c_double]
            L.or_chi_photon.restype = C.c_double
            L.or_bw_tables_build.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int]
            L.or_bw_tables_build.restype = C.c_void_p
            L.or_bw_tables_free.argtypes = [C.c_void_p]
            L.or_bw_tables_export.argtypes = [C.c_void_p, C.c_int, dp, C.c_int64]
            L.or_bw_tables_export.restype = C.c_int64
            L.or_bw_T_interp.argtypes = [C.c_void_p, C.c_double, C.POINTER(C.c_int)]
            L.or_bw_T_interp.restype = C.c_double
            L.or_bw_sample_x.argtypes = [C.c_void_p, C.c_double, C.c_double]
            L.or_bw_sample_x.restype = C.c_double
            L.or_bw_transport.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(RunParams), C.c_void_p, C.c_int64,
                                          C.c_int64, C.c_void_p, C.c_int64, C.POINTER(C.c_uint64)]
            L.or_bw_transport.restype = C.c_int
            L.or_ncs_F.argtypes = [C.c_double, C.c_double]
            L.or_ncs_F.restype = C.c_double
            L.or_brems_dcs_raw.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
            L.or_brems_dcs_raw.restype = C.c_double
            L.or_brems_sigma_direct.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_brems_sigma_direct.restype = C.c_double
            L.or_bh_dcs_raw.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
            L.or_bh_dcs_raw.restype = C.c_double
            L.or_bh_sigma_direct.argtypes = [C.c_double, C.c_double]
            L.or_bh_sigma_direct.restype = C.c_double
            L.or_bh_sigma_interp.argtypes = [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_int)]
            L.or_bh_sigma_interp.restype = C.c_double
            L.or_sample_bh_x.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
            L.or_sample_bh_x.restype = C.c_double
            L.or_pair_transport.argtypes = [C.c_void_p, C.POINTER(RunParams), C.c_void_p, C.c_int64, C.c_int64,
                                            C.c_void_p, C.c_int64, C.POINTER(C.c_uint64), C.c_int]
            L.or_pair_transport.restype = C.c_int
            L.or_tables_build.argtypes = [C.POINTER(TableParams), C.c_int, dp]
            L.or_tables_build.restype = C.c_void_p
            L.or_tables_free.argtypes = [C.c_void_p]
            L.or_tables_export.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.c_int64]
            L.or_tables_export.restype = C.c_int64
            L.or_tables_classical_total.argtypes = [C.c_void_p]
            L.or_tables_classical_total.restype = C.c_double
            L.or_sample_ncs_delta.argtypes = [C.c_void_p, C.c_double, C.c_double, C.POINTER(C.c_int)]
            L.or_sample_ncs_delta.restype = C.c_double
            L.or_sample_brems_y.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
            L.or_sample_brems_y.restype = C.c_double
            L.or_ncs_h_interp.argtypes = [C.c_void_p, C.c_double, C.POINTER(C.c_int)]
            L.or_ncs_h_interp.restype = C.c_double
            L.or_brems_sigma_interp.argtypes = [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_int)]
            L.or_brems_sigma_interp.restype = C.c_double
            u32p = C.POINTER(C.c_uint32)
            L.or_init.argtypes = [C.c_void_p, C.POINTER(RunParams), C.POINTER(C.c_int64), C.c_int64, dp, u32p]
            L.or_init.restype = C.c_int
            L.or_run.argtypes = [C.c_void_p, C.POINTER(RunParams), C.POINTER(C.c_int64), C.c_int64,
                                 C.c_int64, C.c_int64, dp, u32p, C.c_void_p, C.c_int64,
                                 C.POINTER(C.c_int64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                 C.POINTER(C.c_uint64), C.c_int]
            L.or_run.restype = C.c_int
            L.or_fields.argtypes = [C.POINTER(RunParams), C.c_double, C.c_double, C.c_double, dp, dp]
            L.or_eta.argtypes = [dp, dp, dp, C.c_double]
            L.or_eta.restype = C.c_double
            L.or_boris.argtypes = [dp, dp, dp, C.c_double]
            L.or_null_x_hat.argtypes = [C.c_void_p, C.POINTER(RunParams)]
            L.or_null_x_hat.restype = C.c_double
            L.or_pic_init.argtypes = [C.POINTER(RunParams), C.c_int, C.c_double, dp, C.c_int64, dp]
            L.or_pic_init.restype = C.c_int
            L.or_pic_run.argtypes = [C.c_void_p, C.POINTER(RunParams), C.c_int, C.c_double, C.POINTER(C.c_int64),
                                     C.c_int64, C.c_int64, C.c_int64, dp, u32p, dp, C.c_void_p, C.c_int64,
                                     C.POINTER(C.c_int64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                     C.POINTER(C.c_uint64), C.c_int]
            L.or_pic_run.restype = C.c_int
            L.or_pic_gather.argtypes = [C.c_int, C.c_double, dp, C.c_double, dp, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def table_params(**kw) -> TableParams:
    d = dict(n_eta=128, n_y=128, eta_min=1e-4, eta_max=1e2, y_min=1e-6, y_max=1e2,
             n_E=128, n_s=128, gamma_min=2.0, gamma_max=1e6, photon_min=1.0)
    d.update(kw)
    return TableParams(**d)


def run_params(**kw) -> RunParams:
    """Run description with the paper's setup as defaults (Sec. 3)."""
    d = dict(a0=27.0, lambda_m=1e-6, polarisation=0, geometry=0, w0_m=3e-6, focus_x_m=2e-6,
             flat_s=30e-15, ramp_periods=1.0, Z=13.0, charge_state=11.0, ne_over_nc=50.0,
             slab_x0_m=2e-6, slab_thick_m=1e-6, y_half_m=3e-6, dt_over_T=0.01, init_dist=0,
             T_mev=1.0, beam_gamma=1.0, seed=0, run_id=0, enable_ncs=1, enable_brems=1,
             box_enable=0, iz=0)
    E = kw.pop("E_const", (0.0, 0.0, 0.0))
    B = kw.pop("B_const", (0.0, 0.0, 0.0))
    box = kw.pop("box_x_m", (0.0, 0.0))
    d.update(kw)
    r = RunParams(**d)
    r.E_const = (C.c_double * 3)(*E)
    r.B_const = (C.c_double * 3)(*B)
    r.box_x_m = (C.c_double * 2)(*box)
    return r


class Tables:
    """Oracle tables (FP64) for one table-parameter set and a list of Z."""

    def __init__(self, params: TableParams, Z_list):
        self.params = params
        self.Z = np.asarray(Z_list, dtype=np.float64)
        self._h = lib().or_tables_build(C.byref(params), len(self.Z), _dp(self.Z))
        if not self._h:
            raise RuntimeError("oracle table build failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_tables_free(h)
            self._h = None

    def export(self, which: int, iz: int = 0) -> np.ndarray:
        p = self.params
        n = {0: p.n_eta, 1: p.n_eta * p.n_y, 2: p.n_y, 3: p.n_E, 4: p.n_E * p.n_s, 5: p.n_E,
             6: p.n_E * p.n_s}[which]
        out = np.empty(n, dtype=np.float64)
        got = lib().or_tables_export(self._h, which, iz, _dp(out), n)
        if got != n:
            raise RuntimeError("export failed")
        if which == 1:
            out = out.reshape(p.n_eta, p.n_y)
        if which in (4, 6):
            out = out.reshape(p.n_E, p.n_s)
        return out

    def classical_total(self) -> float:
        return lib().or_tables_classical_total(self._h)

    def sample_ncs_delta(self, eta: float, R: float):
        b = C.c_int(0)
        d = lib().or_sample_ncs_delta(self._h, eta, R, C.byref(b))
        return d, b.value

    def sample_brems_y(self, iz: int, gamma: float, R: float) -> float:
        return lib().or_sample_brems_y(self._h, iz, gamma, R)

    def h_interp(self, eta: float):
        f = C.c_int(0)
        v = lib().or_ncs_h_interp(self._h, eta, C.byref(f))
        return v, f.value

    def sigma_interp(self, iz: int, gamma: float):
        f = C.c_int(0)
        v = lib().or_brems_sigma_interp(self._h, iz, gamma, C.byref(f))
        return v, f.value

    def bh_sigma_interp(self, iz: int, k: float):
        f = C.c_int(0)
        v = lib().or_bh_sigma_interp(self._h, iz, k, C.byref(f))
        return v, f.value

    def sample_bh_x(self, iz: int, k: float, R: float) -> float:
        return lib().or_sample_bh_x(self._h, iz, k, R)


def _wait_ptr(run: RunParams, wait, n: int):
    if wait is None:
        if run.brems_method == 1 and n > 0:
            raise ValueError("the null-collision method needs a wait array (uint32, one per particle)")
        return None
    assert wait.dtype == np.uint32 and wait.flags.c_contiguous and wait.shape == (n,)
    return wait.ctypes.data_as(C.POINTER(C.c_uint32))


def init(tables: Tables, run: RunParams, ids, wait=None) -> np.ndarray:
    """Initial state (n x 6).  For the null-collision brems method ``wait`` (uint32,
    one per particle) receives the steps to each particle's first candidate."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    st = np.zeros((len(ids), 6), dtype=np.float64)
    rc = lib().or_init(tables._h, C.byref(run), ids.ctypes.data_as(C.POINTER(C.c_int64)), len(ids), _dp(st),
                       _wait_ptr(run, wait, len(ids)))
    if rc != 0:
        raise RuntimeError("or_init failed")
    return st


def run(tables: Tables, run: RunParams, ids, state, step0: int, n_steps: int,
        capacity: int = 1 << 20, threads: int | None = None, events=None, wait=None):
    """Advance ``state`` (n x 6, in place); return (photons, true photon count, hist, tally).

    ``events`` (optional uint64 array, one per particle) accumulates each particle's
    event fingerprint (see oracle.h); ``wait`` is the null-collision wait array (in/out)."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    assert state.dtype == np.float64 and state.flags.c_contiguous and state.shape == (len(ids), 6)
    photons = np.zeros(capacity, dtype=PHOTON_DTYPE)
    hist = np.zeros(HIST_WORDS, dtype=np.uint64)
    tally = np.zeros(TALLY_WORDS, dtype=np.uint64)
    n_ph = C.c_int64(0)
    nt = threads if threads else (os.cpu_count() or 1)
    rc = lib().or_run(tables._h, C.byref(run), ids.ctypes.data_as(C.POINTER(C.c_int64)), len(ids),
                      step0, n_steps, _dp(state), _wait_ptr(run, wait, len(ids)),
                      photons.ctypes.data_as(C.c_void_p), capacity,
                      C.byref(n_ph), hist.ctypes.data_as(C.POINTER(C.c_uint64)),
                      tally.ctypes.data_as(C.POINTER(C.c_uint64)),
                      events.ctypes.data_as(C.POINTER(C.c_uint64)) if events is not None else None, nt)
    if rc != 0:
        raise RuntimeError("or_run failed")
    return photons[:min(n_ph.value, capacity)], n_ph.value, hist, tally


PAIR_DIRECT, PAIR_FREE_PATH = 0, 1


def pair_transport(tables: Tables, run: RunParams, photons, step_end: int, capacity: int = 1 << 20,
                   method: int = PAIR_DIRECT):
    """Bethe-Heitler conversion of the photon records (PHOTON_DTYPE) in the target up to
    step_end (see oracle.h); returns (pairs, true pair count, tally)."""
    ph = np.ascontiguousarray(photons, dtype=PHOTON_DTYPE)
    pairs = np.zeros(capacity, dtype=PAIR_DTYPE)
    tally = np.zeros(PAIR_TALLY_WORDS, dtype=np.uint64)
    rc = lib().or_pair_transport(tables._h, C.byref(run), ph.ctypes.data_as(C.c_void_p), len(ph), int(step_end),
                                 pairs.ctypes.data_as(C.c_void_p), capacity,
                                 tally.ctypes.data_as(C.POINTER(C.c_uint64)), int(method))
    if rc != 0:
        raise RuntimeError("or_pair_transport failed")
    n = int(tally[PT["N_PAIRS"]])
    return pairs[:min(n, capacity)], n, tally


class BWTables:
    """Breit-Wheeler tables (see oracle.h): T(chi) on n_chi log-spaced chi in [chi_min, chi_max]
    and the CDF of the pair spectrum over the positron fraction x at n_x nodes."""

    def __init__(self, n_chi: int = 64, chi_min: float = 1e-2, chi_max: float = 1e3, n_x: int = 128):
        self.n_chi, self.n_x, self.chi_min, self.chi_max = n_chi, n_x, chi_min, chi_max
        self._h = lib().or_bw_tables_build(n_chi, chi_min, chi_max, n_x)
        if not self._h:
            raise ValueError("bad Breit-Wheeler table parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_bw_tables_free(h)
            self._h = None

    def export(self, which: int) -> np.ndarray:
        n = self.n_chi if which == 0 else self.n_chi * self.n_x
        out = np.zeros(n)
        if lib().or_bw_tables_export(self._h, which, _dp(out), n) != n:
            raise ValueError(which)
        return out if which == 0 else out.reshape(self.n_chi, self.n_x)

    def T_interp(self, chi: float):
        fl = C.c_int(0)
        v = lib().or_bw_T_interp(self._h, chi, C.byref(fl))
        return v, fl.value

    def sample_x(self, chi: float, R: float) -> float:
        return lib().or_bw_sample_x(self._h, chi, R)


def bw_transport(bw: BWTables, tables: Tables, run: RunParams, photons, step_end: int, capacity: int = 1 << 20):
    """Breit-Wheeler conversion of the photon records (PHOTON_DTYPE) in the run's prescribed fields up
    to step_end (see oracle.h); returns (pairs, true pair count, tally)."""
    ph = np.ascontiguousarray(photons, dtype=PHOTON_DTYPE)
    pairs = np.zeros(capacity, dtype=PAIR_DTYPE)
    tally = np.zeros(PAIR_TALLY_WORDS, dtype=np.uint64)
    rc = lib().or_bw_transport(bw._h, tables._h, C.byref(run), ph.ctypes.data_as(C.c_void_p), len(ph),
                               int(step_end), pairs.ctypes.data_as(C.c_void_p), capacity,
                               tally.ctypes.data_as(C.POINTER(C.c_uint64)))
    if rc != 0:
        raise RuntimeError("or_bw_transport failed")
    n = int(tally[PT["N_PAIRS"]])
    return pairs[:min(n, capacity)], n, tally


def chi_photon(kvec, E, B, E_S: float) -> float:
    kvec = np.ascontiguousarray(kvec, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    return lib().or_chi_photon(_dp(kvec), _dp(E), _dp(B), E_S)


def fixed_to_float(tally: np.ndarray, idx: int) -> float:
    """Value of a 128-bit fixed-point tally pair (lo, hi) in m c^2."""
    return float(int(tally[idx + 1])) + float(int(tally[idx])) / 2.0 ** 64


# ---------------------------------------------------------------- 1D PIC ----
def pic_grid_words(n_cells: int) -> int:
    return 6 * n_cells + 5


def pic_weight(run: RunParams, n_total: int) -> float:
    """Areal density of one macro-electron: n_e (n_c) x slab thickness (c/omega) / electrons."""
    kl = 2 * np.pi / run.lambda_m
    return run.ne_over_nc * run.slab_thick_m * kl / n_total


def pic_init(run: RunParams, n_cells: int, weight: float, state: np.ndarray) -> np.ndarray:
    grid = np.zeros(pic_grid_words(n_cells))
    st = np.ascontiguousarray(state, dtype=np.float64)
    rc = lib().or_pic_init(C.byref(run), n_cells, weight, _dp(st), len(st), _dp(grid))
    if rc != 0:
        raise RuntimeError("or_pic_init failed")
    return grid


def pic_run(tables: "Tables", run: RunParams, n_cells: int, weight: float, ids, state, grid, step0: int,
            n_steps: int, capacity: int = 1 << 20, threads: int | None = None, events=None, wait=None):
    """Advance particles (n x 6, in place) and grid (in place) together; returns
    (photons, true photon count, hist, tally)."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    assert state.dtype == np.float64 and state.flags.c_contiguous and state.shape == (len(ids), 6)
    assert grid.dtype == np.float64 and grid.shape == (pic_grid_words(n_cells),)
    photons = np.zeros(capacity, dtype=PHOTON_DTYPE)
    hist = np.zeros(HIST_WORDS, dtype=np.uint64)
    tally = np.zeros(TALLY_WORDS, dtype=np.uint64)
    n_ph = C.c_int64(0)
    nt = threads if threads else (os.cpu_count() or 1)
    rc = lib().or_pic_run(tables._h, C.byref(run), n_cells, weight, ids.ctypes.data_as(C.POINTER(C.c_int64)),
                          len(ids), step0, n_steps, _dp(state), _wait_ptr(run, wait, len(ids)), _dp(grid),
                          photons.ctypes.data_as(C.c_void_p), capacity, C.byref(n_ph),
                          hist.ctypes.data_as(C.POINTER(C.c_uint64)), tally.ctypes.data_as(C.POINTER(C.c_uint64)),
                          events.ctypes.data_as(C.POINTER(C.c_uint64)) if events is not None else None, nt)
    if rc != 0:
        raise RuntimeError("or_pic_run failed")
    return photons[:min(n_ph.value, capacity)], n_ph.value, hist, tally


def pic_fields(grid, n_cells: int):
    """(ex at half nodes, ey, ez, by, bz at nodes, rho_ion at nodes) from a grid array."""
    n = n_cells
    ex = grid[:n]
    fp, fm, gp, gm, rho = (grid[n + k * (n + 1): n + (k + 1) * (n + 1)] for k in range(5))
    return ex, 0.5 * (fp + fm), 0.5 * (gp + gm), 0.5 * (gm - gp), 0.5 * (fp - fm), rho


def pic_gather(grid, n_cells: int, dx: float, x: float):
    E = np.zeros(3)
    B = np.zeros(3)
    lib().or_pic_gather(n_cells, dx, _dp(grid), x, _dp(E), _dp(B))
    return E, B


def null_x_hat(tables: Tables, run: RunParams) -> float:
    """Majorant optical depth per step of the null-collision method."""
    return lib().or_null_x_hat(tables._h, C.byref(run))


def fields(run: RunParams, x: float, y: float, t: float):
    E = np.zeros(3)
    B = np.zeros(3)
    lib().or_fields(C.byref(run), x, y, t, _dp(E), _dp(B))
    return E, B


def eta(u, E, B, E_S: float) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    return lib().or_eta(_dp(u), _dp(E), _dp(B), E_S)


def boris(u, E, B, dt: float) -> np.ndarray:
    u = np.array(u, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lib().or_boris(_dp(u), _dp(E), _dp(B), dt)
    return u


def __getattr__(name):
    # thin scalar passthroughs: bessel_k, int_k53, ncs_F, ...
    m = {"bessel_k": "or_bessel_k", "int_k53": "or_int_k53", "ncs_F": "or_ncs_F",
         "ncs_power_integral": "or_ncs_power_integral", "ncs_h_direct": "or_ncs_h_direct",
         "coulomb_f": "or_coulomb_f", "brems_dcs_raw": "or_brems_dcs_raw",
         "brems_sigma_direct": "or_brems_sigma_direct", "schwinger_field": "or_schwinger_field",
         "bh_dcs_raw": "or_bh_dcs_raw", "bh_sigma_direct": "or_bh_sigma_direct",
         "critical_density": "or_critical_density", "int_k13": "or_int_k13", "bw_G": "or_bw_G",
         "bw_T_direct": "or_bw_T_direct"}
    if name in m:
        return getattr(lib(), m[name])
    raise AttributeError(name)

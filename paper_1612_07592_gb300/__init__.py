"""GB300 photon-emission step (arXiv:1612.07592, Wan et al.) -- Python binding.

A thin ctypes layer over ``libpe.so`` (the C ABI in ``include/pe.h``): the same
entry points with the same names, plus a small ``Run`` helper that allocates
the caller-owned buffers as torch CUDA tensors.  Every step of the physics runs
in the library's CUDA kernels; this module only marshals arguments.  Importing
it needs no GPU; calling into the library needs the compiled ``libpe.so`` and a
CUDA device, and fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PE_LIB_PATH selects another build of the same library (e.g. a variant compiled with other flags)
LIB_PATH = os.environ.get("PE_LIB_PATH") or os.path.join(HERE, "libpe.so")

PE_OK, PE_ERR_ARG, PE_ERR_CUDA, PE_ERR_NOMEM, PE_ERR_BUFFER_FULL, PE_ERR_TABLE_RANGE, PE_ERR_TIMEOUT, PE_ERR_STATE = range(8)
PE_LP_Y, PE_CP = 0, 1
PE_PLANE_1D, PE_GAUSS_2D, PE_CONST, PE_PIC_1D = 0, 1, 2, 3
PE_F64, PE_F32 = 0, 1
PE_REST, PE_MAXWELL_JUTTNER, PE_BEAM, PE_CALLER = 0, 1, 2, 3
PE_BREMS_DIRECT, PE_BREMS_NULL = 0, 1
PE_WAIT_NEVER = 0xFFFFFFFF
PE_PIC_MAX_CELLS = 4096
HIST_E_BINS, HIST_T_BINS = 512, 180
HIST_WORDS = 2 * HIST_E_BINS + 2 * HIST_T_BINS
TALLY_WORDS = 32
MAX_BATCH = 64
T = dict(N_NCS_STORED=0, N_NCS_BELOW=1, N_BR_STORED=2, N_BR_BELOW=3, N_PHOTONS=4, N_ETA_ABOVE=5,
         N_ETA_BELOW=6, N_GAMMA_ABOVE=7, N_KILLED=8, KILLED_STEPS=9, N_CLAMP=10, N_HIST_OVER=11, N_WAIT_TIMEOUT=12,
         N_NONFINITE=13, E_NCS_STORED=16, E_NCS_BELOW=18, E_BR_STORED=20, E_BR_BELOW=22, E_RECOIL_NCS=24, E_RECOIL_BR=26)
PHOTON_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("energy", "<f4"), ("kx", "<f4"),
                         ("ky", "<f4"), ("kz", "<f4"), ("step", "<u4"), ("id_mech", "<u4")])
# Bethe-Heitler pair records (pe_pair) and the pair tally words
PAIR_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("e_minus", "<f4"), ("e_plus", "<f4"), ("kx", "<f4"),
                       ("ky", "<f4"), ("kz", "<f4"), ("step", "<u4"), ("photon", "<u4"), ("id_mech", "<u4")])
PAIR_TALLY_WORDS = 8
PT = dict(N_PAIRS=0, N_ENTERED=1, N_K_ABOVE=2, N_TESTS=3, E_PAIRS=4, E_POSITRONS=6)
PE_PAIR_DIRECT, PE_PAIR_FREE_PATH = 0, 1
EXPORTED = ["pe_create_tables", "pe_destroy_tables", "pe_tables_export", "pe_init_particles", "pe_step",
            "pe_step_ex", "pe_tally", "pe_destroy", "pe_graph_create", "pe_graph_launch", "pe_graph_destroy",
            "pe_a0_from_intensity", "pe_launch_count", "pe_last_error", "pe_pair_transport", "pe_resume_particles",
            "pe_bw_tables_host"]


class PeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pe status {status}: {msg}")
        self.status = status


class TableParams(C.Structure):
    _fields_ = [("n_eta", C.c_int), ("n_y", C.c_int), ("eta_min", C.c_double), ("eta_max", C.c_double),
                ("y_min", C.c_double), ("y_max", C.c_double), ("n_E", C.c_int), ("n_s", C.c_int),
                ("gamma_min", C.c_double), ("gamma_max", C.c_double), ("photon_min_mc2", C.c_double),
                ("n_Z", C.c_int), ("Z", C.POINTER(C.c_double))]


class RunParams(C.Structure):
    _fields_ = [("a0", C.c_double), ("lambda_m", C.c_double), ("polarisation", C.c_int), ("geometry", C.c_int),
                ("w0_m", C.c_double), ("focus_x_m", C.c_double), ("flat_s", C.c_double),
                ("ramp_periods", C.c_double), ("E_const", C.c_double * 3), ("B_const", C.c_double * 3),
                ("Z", C.c_double), ("charge_state", C.c_double), ("ne_over_nc", C.c_double),
                ("slab_x0_m", C.c_double), ("slab_thick_m", C.c_double), ("y_half_m", C.c_double),
                ("dt_over_T", C.c_double), ("precision", C.c_int), ("init_dist", C.c_int),
                ("T_mev", C.c_double), ("beam_gamma", C.c_double), ("seed", C.c_uint64),
                ("run_id", C.c_uint32), ("enable_ncs", C.c_int), ("enable_brems", C.c_int),
                ("box_enable", C.c_int), ("box_x_m", C.c_double * 2), ("reflect_r", C.c_double),
                ("mirror_x_m", C.c_double), ("brems_method", C.c_int), ("n_cells", C.c_int),
                ("id0", C.c_uint32)]


class Buffers(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("ux", C.c_void_p), ("uy", C.c_void_p),
                ("uz", C.c_void_p), ("tau", C.c_void_p), ("photons", C.c_void_p),
                ("photon_capacity", C.c_int64), ("hist", C.c_void_p), ("tally", C.c_void_p),
                ("events", C.c_void_p), ("brems_wait", C.c_void_p), ("grid", C.c_void_p)]


class LaunchConfig(C.Structure):
    _fields_ = [("block", C.c_int), ("ctas_per_sm", C.c_int), ("steps_per_launch", C.c_int)]


class TallyOut(C.Structure):
    _fields_ = [("tally", C.c_uint64 * TALLY_WORDS), ("hist", C.c_uint64 * HIST_WORDS),
                ("n_particles", C.c_int64), ("steps_done", C.c_int64), ("photons_stored", C.c_int64),
                ("live_particle_steps", C.c_double), ("e_ncs_stored", C.c_double), ("e_ncs_below", C.c_double),
                ("e_br_stored", C.c_double), ("e_br_below", C.c_double), ("e_recoil_ncs", C.c_double),
                ("e_recoil_br", C.c_double)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libpe.so.  Raises if the library has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            vp = C.c_void_p
            L.pe_create_tables.argtypes = [C.POINTER(TableParams), C.POINTER(vp)]
            L.pe_destroy_tables.argtypes = [vp]
            L.pe_tables_export.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int64,
                                           C.POINTER(C.c_int64)]
            L.pe_init_particles.argtypes = [vp, C.POINTER(RunParams), C.c_int64, C.POINTER(Buffers), vp,
                                            C.POINTER(vp)]
            L.pe_step.argtypes = [C.POINTER(vp), C.c_int, C.c_int64]
            L.pe_step_ex.argtypes = [C.POINTER(vp), C.c_int, C.c_int64, C.POINTER(LaunchConfig)]
            L.pe_tally.argtypes = [vp, C.POINTER(TallyOut)]
            L.pe_graph_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int64, C.POINTER(LaunchConfig), C.POINTER(vp)]
            L.pe_graph_launch.argtypes = [vp]
            L.pe_graph_destroy.argtypes = [vp]
            L.pe_destroy.argtypes = [vp]
            L.pe_pic_step_noalloc.argtypes = [vp, C.POINTER(RunParams), C.c_int64, C.POINTER(Buffers), C.c_int64,
                                              C.c_int64, vp]
            L.pe_electron_spectrum.argtypes = [vp, C.c_int, C.c_double, C.c_double, vp]
            L.pe_photon_map.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, vp]
            L.pe_pair_transport.argtypes = [vp, vp, C.c_int64, C.c_int64, vp, C.c_int64, vp, C.c_int]
            L.pe_resume_particles.argtypes = [vp, C.POINTER(RunParams), C.c_int64, C.POINTER(Buffers), C.c_int64, vp,
                                              C.POINTER(vp)]
            L.pe_bw_tables_host.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
            L.pe_bw_tables_create.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(vp)]
            L.pe_bw_tables_destroy.argtypes = [vp]
            L.pe_bw_transport.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, vp, C.c_int64, vp]
            L.pe_math_probe.argtypes = [C.c_int, vp, vp, C.c_int64, vp]
            L.pe_debug_count.argtypes = [vp, vp, C.POINTER(C.c_uint64)]
            L.pe_debug_build.restype = C.c_int
            L.pe_fma_peak.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, C.POINTER(C.c_int)]
            L.pe_a0_from_intensity.argtypes = [C.c_double, C.c_double, C.c_int]
            L.pe_a0_from_intensity.restype = C.c_double
            L.pe_launch_count.restype = C.c_int64
            L.pe_last_error.restype = C.c_char_p
            for name in ("pe_create_tables", "pe_destroy_tables", "pe_tables_export", "pe_init_particles",
                         "pe_step", "pe_step_ex", "pe_tally", "pe_destroy", "pe_graph_create", "pe_graph_launch",
                         "pe_graph_destroy", "pe_pic_step_noalloc", "pe_electron_spectrum", "pe_photon_map",
                         "pe_pair_transport", "pe_resume_particles", "pe_bw_tables_host", "pe_math_probe",
                         "pe_fma_peak", "pe_bw_tables_create", "pe_bw_tables_destroy", "pe_bw_transport",
                         "pe_debug_count"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(status: int, allow=()):
    if status != PE_OK and status not in allow:
        raise PeError(status, lib().pe_last_error().decode())
    return status


# ---------------------------------------------------------------- C ABI ----
def table_params(**kw):
    d = dict(n_eta=128, n_y=128, eta_min=1e-4, eta_max=1e2, y_min=1e-6, y_max=1e2, n_E=128, n_s=128,
             gamma_min=2.0, gamma_max=1e6, photon_min_mc2=1.0)
    Z = kw.pop("Z", (13.0, 79.0))
    d.update(kw)
    return d, tuple(float(z) for z in Z)


def pe_create_tables(params: dict, Z) -> int:
    z = (C.c_double * len(Z))(*Z)
    p = TableParams(**params, n_Z=len(Z), Z=z)
    h = C.c_void_p()
    _check(lib().pe_create_tables(C.byref(p), C.byref(h)))
    return h.value


def pe_destroy_tables(h: int):
    _check(lib().pe_destroy_tables(h))


def pe_tables_export(h: int, which: int, iz: int = 0) -> np.ndarray:
    n = C.c_int64(0)
    dummy = (C.c_double * 1)()
    lib().pe_tables_export(h, which, iz, dummy, 0, C.byref(n))
    out = np.empty(max(n.value, 1), dtype=np.float64)
    _check(lib().pe_tables_export(h, which, iz, out.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n)))
    return out[:n.value]


def pic_grid_words(n_cells: int) -> int:
    """Words of the field grid of a PE_PIC_1D run (PE_PIC_GRID_WORDS)."""
    return 6 * int(n_cells) + 5


def run_params(**kw) -> RunParams:
    d = dict(a0=27.0, lambda_m=1e-6, polarisation=0, geometry=0, w0_m=3e-6, focus_x_m=2e-6, flat_s=30e-15,
             ramp_periods=1.0, Z=13.0, charge_state=11.0, ne_over_nc=50.0, slab_x0_m=2e-6, slab_thick_m=1e-6,
             y_half_m=3e-6, dt_over_T=0.01, precision=PE_F64, init_dist=PE_REST, T_mev=1.0, beam_gamma=1.0,
             seed=0, run_id=0, enable_ncs=1, enable_brems=1, box_enable=0)
    E = kw.pop("E_const", (0.0, 0.0, 0.0))
    B = kw.pop("B_const", (0.0, 0.0, 0.0))
    box = kw.pop("box_x_m", (0.0, 0.0))
    kw.pop("iz", None)
    d.update(kw)
    r = RunParams(**d)
    r.E_const = (C.c_double * 3)(*E)
    r.B_const = (C.c_double * 3)(*B)
    r.box_x_m = (C.c_double * 2)(*box)
    return r


def pe_init_particles(tables: int, params: RunParams, n: int, buffers: Buffers, stream: int) -> int:
    h = C.c_void_p()
    _check(lib().pe_init_particles(tables, C.byref(params), n, C.byref(buffers), stream, C.byref(h)))
    return h.value


def pe_resume_particles(tables: int, params: RunParams, n: int, buffers: Buffers, step0: int, stream: int) -> int:
    h = C.c_void_p()
    _check(lib().pe_resume_particles(tables, C.byref(params), n, C.byref(buffers), int(step0), stream, C.byref(h)))
    return h.value


def pe_step(runs, n_steps: int):
    arr = (C.c_void_p * len(runs))(*runs)
    _check(lib().pe_step(arr, len(runs), n_steps))


def pe_step_ex(runs, n_steps: int, block: int = 0, ctas_per_sm: int = 0, steps_per_launch: int = 0):
    arr = (C.c_void_p * len(runs))(*runs)
    cfg = LaunchConfig(block, ctas_per_sm, steps_per_launch)
    _check(lib().pe_step_ex(arr, len(runs), n_steps, C.byref(cfg)))


def pe_graph_create(runs, steps_per_replay: int, block: int = 0, ctas_per_sm: int = 0,
                    steps_per_launch: int = 0) -> int:
    arr = (C.c_void_p * len(runs))(*runs)
    cfg = LaunchConfig(block, ctas_per_sm, steps_per_launch)
    h = C.c_void_p()
    _check(lib().pe_graph_create(arr, len(runs), steps_per_replay, C.byref(cfg), C.byref(h)))
    return h.value


def pe_graph_launch(graph: int):
    _check(lib().pe_graph_launch(graph))


def pe_graph_destroy(graph: int):
    _check(lib().pe_graph_destroy(graph))


def pe_tally(run: int) -> TallyOut:
    out = TallyOut()
    st = _check(lib().pe_tally(run, C.byref(out)), allow=(PE_ERR_BUFFER_FULL,))
    out.status = st
    return out


def pe_pic_step_noalloc(tables: int, params: RunParams, n: int, buffers: Buffers, step0: int, n_steps: int,
                        stream) -> None:
    """PIC steps on caller-owned buffers with the library's fixed scratch array (no device
    allocation); see pe.h.  ``stream`` is a cudaStream_t value (e.g. torch's ``cuda_stream``)."""
    _check(lib().pe_pic_step_noalloc(tables, C.byref(params), int(n), C.byref(buffers), int(step0), int(n_steps),
                                     stream))


def pe_electron_spectrum(run: int, n_bins: int, e_min_mev: float, e_max_mev: float, counts_ptr: int) -> None:
    _check(lib().pe_electron_spectrum(run, int(n_bins), float(e_min_mev), float(e_max_mev), counts_ptr))


def pe_photon_map(run: int, nx: int, x_min_m: float, x_max_m: float, ne: int, e_min_mev: float, e_max_mev: float,
                  counts_ptr: int) -> None:
    _check(lib().pe_photon_map(run, int(nx), float(x_min_m), float(x_max_m), int(ne), float(e_min_mev),
                               float(e_max_mev), counts_ptr))


def pe_pair_transport(run: int, photons_ptr: int, n_photons: int, step_end: int, pairs_ptr: int, capacity: int,
                      tally_ptr: int, method: int = PE_PAIR_DIRECT) -> None:
    _check(lib().pe_pair_transport(run, photons_ptr, int(n_photons), int(step_end), pairs_ptr, int(capacity),
                                   tally_ptr, int(method)))


def pe_bw_tables_host(n_chi: int, chi_min: float, chi_max: float, n_x: int):
    """Breit-Wheeler tables built on the host: (T [n_chi], CDF [n_chi, n_x]); see pe.h."""
    T = np.zeros(n_chi)
    cdf = np.zeros(n_chi * n_x)
    _check(lib().pe_bw_tables_host(int(n_chi), float(chi_min), float(chi_max), int(n_x),
                                   T.ctypes.data_as(C.POINTER(C.c_double)), cdf.ctypes.data_as(C.POINTER(C.c_double))))
    return T, cdf.reshape(n_chi, n_x)


def pe_bw_tables_create(n_chi: int = 64, chi_min: float = 1e-2, chi_max: float = 1e3, n_x: int = 128) -> int:
    """Breit-Wheeler tables on the current device (see pe.h)."""
    h = C.c_void_p()
    _check(lib().pe_bw_tables_create(int(n_chi), float(chi_min), float(chi_max), int(n_x), C.byref(h)))
    return h.value


def pe_bw_tables_destroy(h: int) -> None:
    _check(lib().pe_bw_tables_destroy(h))


def pe_bw_transport(run: int, bw: int, photons_ptr: int, n_photons: int, step_end: int, pairs_ptr: int,
                    capacity: int, tally_ptr: int) -> None:
    _check(lib().pe_bw_transport(run, bw, photons_ptr, int(n_photons), int(step_end), pairs_ptr, int(capacity),
                                 tally_ptr))


def pe_debug_build() -> bool:
    """True for a library compiled with PE_DEBUG (range checks of table indices; see pe.h)."""
    return bool(lib().pe_debug_build())


def pe_debug_count(tables: int | None = None, bw: int | None = None) -> int:
    """Table indices found out of range so far (synchronises the device; 0 in a release build)."""
    out = C.c_uint64(0)
    _check(lib().pe_debug_count(tables, bw, C.byref(out)))
    return out.value


PE_MATH = dict(RCP=0, SIN=1, COS=2, SIN1=3, COS1=4, BREMS_P=5, BREMS_P1=6, CUDA_RCP=7, CUDA_SIN=8, CUDA_COS=9,
               CUDA_EXPM1=10, GOUY_C=11, GOUY_S=12, EXP_NEG=13, TAU=14)
PE_FMA_F32, PE_FMA_F32X2, PE_FMA_F64 = 0, 1, 2


def pe_math_probe(fn: int, in_ptr: int, out_ptr: int, n: int, stream) -> None:
    """One of the library's FP32 device forms on n device floats (see pe.h)."""
    _check(lib().pe_math_probe(int(fn), in_ptr, out_ptr, int(n), stream))


def pe_fma_peak(kind: int, blocks: int, threads: int, iters: int, out_ptr: int, stream) -> int:
    """Launch the FMA-loop kernel of one pipe (see pe.h); returns the chains per thread."""
    ch = C.c_int(0)
    _check(lib().pe_fma_peak(int(kind), int(blocks), int(threads), int(iters), out_ptr, stream, C.byref(ch)))
    return ch.value


def pe_destroy(run: int):
    _check(lib().pe_destroy(run))


def pe_a0_from_intensity(I_wcm2: float, lambda_m: float = 1e-6, polarisation: int = PE_LP_Y) -> float:
    return lib().pe_a0_from_intensity(I_wcm2, lambda_m, polarisation)


def pe_launch_count() -> int:
    return lib().pe_launch_count()


# ------------------------------------------------------- torch-side helper ----
class Run:
    """One run with caller-owned buffers allocated as torch CUDA tensors."""

    def __init__(self, tables: int, params: RunParams, n: int, capacity: int = 1 << 20, stream=None,
                 device="cuda", events: bool = False, _resume_step: int | None = None, _arrays=None):
        import torch
        self.torch = torch
        dt = torch.float32 if params.precision == PE_F32 else torch.float64
        dev = torch.device(device)
        m = max(int(n), 1)
        self.n = int(n)
        # positions and optical depths take 8 bytes per particle in both precisions
        # (FP32 runs store float pairs hi + lo there)
        self.x = torch.zeros(m, dtype=torch.float64, device=dev)
        self.y = torch.zeros(m, dtype=torch.float64, device=dev)
        self.ux = torch.zeros(m, dtype=dt, device=dev)
        self.uy = torch.zeros(m, dtype=dt, device=dev)
        self.uz = torch.zeros(m, dtype=dt, device=dev)
        self.tau = torch.zeros(m, dtype=torch.float64, device=dev)
        self.capacity = int(capacity)
        self.photons = torch.zeros(max(self.capacity, 1) * 8, dtype=torch.int32, device=dev)
        self.hist = torch.zeros(HIST_WORDS, dtype=torch.int64, device=dev)
        self.tally = torch.zeros(TALLY_WORDS, dtype=torch.int64, device=dev)
        self.events = torch.zeros(m, dtype=torch.int64, device=dev) if events else None
        # null-collision brems: steps to each particle's next candidate (uint32 words)
        self.wait = torch.zeros(m, dtype=torch.int32, device=dev) if params.brems_method == PE_BREMS_NULL else None
        # 1D PIC: the field grid (E_x at half nodes; F+, F-, G+, G-, ion charge at nodes)
        self.grid = (torch.zeros(pic_grid_words(params.n_cells), dtype=dt, device=dev)
                     if params.geometry == PE_PIC_1D else None)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.params = params
        if _resume_step is None:
            self.handle = pe_init_particles(tables, params, self.n, self._buffers(), self.stream.cuda_stream)
        else:
            with torch.cuda.stream(self.stream):
                for name, arr in _arrays.items():
                    dst = getattr(self, name)
                    src = torch.from_numpy(np.ascontiguousarray(arr)).view(dst.dtype).reshape(-1)
                    dst[: src.numel()].copy_(src.to(dev))
            self.handle = pe_resume_particles(tables, params, self.n, self._buffers(), _resume_step,
                                              self.stream.cuda_stream)

    # ------------------------------------------------------------ checkpoint ----
    def checkpoint(self) -> dict:
        """Host copy of everything the run's next steps depend on: the state arrays, the stored
        photons, histograms, tallies, event and wait words, the PIC grid, and the step index."""
        out = self.tally_out()
        arrays = {}
        for name in ("x", "y", "ux", "uy", "uz", "tau", "hist", "tally", "events", "wait", "grid"):
            t = getattr(self, name)
            if t is not None:
                arrays[name] = t.cpu().numpy().copy()
        arrays["photons"] = self.photons[: out.photons_stored * 8].cpu().numpy().copy()
        return {"step": int(out.steps_done), "n": self.n, "capacity": self.capacity,
                "events": self.events is not None, "arrays": arrays}

    @classmethod
    def resume(cls, tables: int, params: RunParams, ckpt: dict, stream=None, device="cuda"):
        """A run continuing from a checkpoint (pe_resume_particles): the next pe_step gives the
        results the checkpointed run would have given."""
        return cls(tables, params, ckpt["n"], capacity=ckpt["capacity"], stream=stream, device=device,
                   events=ckpt["events"], _resume_step=ckpt["step"], _arrays=ckpt["arrays"])

    def save(self, path: str):
        """Write a checkpoint to an .npz file."""
        c = self.checkpoint()
        np.savez(path, _step=c["step"], _n=c["n"], _capacity=c["capacity"], _events=c["events"], **c["arrays"])

    @classmethod
    def load(cls, tables: int, params: RunParams, path: str, stream=None, device="cuda"):
        """Resume from an .npz checkpoint written by save()."""
        z = np.load(path)
        arrays = {k: z[k] for k in z.files if not k.startswith("_")}
        ckpt = {"step": int(z["_step"]), "n": int(z["_n"]), "capacity": int(z["_capacity"]),
                "events": bool(z["_events"]), "arrays": arrays}
        return cls.resume(tables, params, ckpt, stream=stream, device=device)

    def _buffers(self) -> Buffers:
        return Buffers(self.x.data_ptr(), self.y.data_ptr(), self.ux.data_ptr(), self.uy.data_ptr(),
                       self.uz.data_ptr(), self.tau.data_ptr(), self.photons.data_ptr(), self.capacity,
                       self.hist.data_ptr(), self.tally.data_ptr(),
                       self.events.data_ptr() if self.events is not None else None,
                       self.wait.data_ptr() if self.wait is not None else None,
                       self.grid.data_ptr() if self.grid is not None else None)

    def rebind(self, tables: int, precision_params: RunParams | None = None):
        """Replace the run handle by a fresh one on the same buffers (caller-provided state,
        optical depths redrawn, step index 0, tallies cleared)."""
        p = precision_params if precision_params is not None else self.params
        q = RunParams.from_buffer_copy(p)
        q.init_dist = PE_CALLER
        old = self.handle
        self.handle = pe_init_particles(tables, q, self.n, self._buffers(), self.stream.cuda_stream)
        if old:
            pe_destroy(old)

    def _state_tensors(self):
        ts = [self.x, self.y, self.ux, self.uy, self.uz, self.tau]
        return ts + [t for t in (self.wait, self.grid) if t is not None]

    def snapshot(self):
        return [t.clone() for t in self._state_tensors()]

    def restore(self, snap):
        for dst, src in zip(self._state_tensors(), snap):
            dst.copy_(src)

    def state(self) -> np.ndarray:
        """Host copy (n x 6, float64): x, y, ux, uy, uz, tau.

        In FP32 runs positions and optical depths are stored as float pairs (hi, lo)
        whose sum is the value."""
        def pair(t):
            if self.params.precision == PE_F32:
                p = t[:self.n].view(self.torch.float32).reshape(-1, 2).double().cpu().numpy()
                return p[:, 0] + p[:, 1]
            return t[:self.n].cpu().numpy()
        cols = [pair(self.x), pair(self.y)]
        cols += [c[:self.n].double().cpu().numpy() for c in (self.ux, self.uy, self.uz)]
        return np.stack(cols + [pair(self.tau)], axis=1)

    def photon_records(self, count: int | None = None) -> np.ndarray:
        out = self.tally_out() if count is None else None
        k = count if count is not None else out.photons_stored
        raw = self.photons[: k * 8].cpu().numpy()
        return raw.view(PHOTON_DTYPE)

    def event_words(self) -> np.ndarray:
        return self.events[:self.n].cpu().numpy().view(np.uint64)

    def pic_fields(self):
        """1D PIC grid as float64 arrays (ex at half nodes; ey, ez, by, bz, ion charge at nodes)."""
        g = self.grid.double().cpu().numpy()
        n = self.params.n_cells
        ex = g[:n]
        fp, fm, gp, gm, rho = (g[n + k * (n + 1): n + (k + 1) * (n + 1)] for k in range(5))
        return ex, 0.5 * (fp + fm), 0.5 * (gp + gm), 0.5 * (gm - gp), 0.5 * (fp - fm), rho

    def electron_spectrum(self, n_bins: int = 200, e_min_mev: float = 0.01, e_max_mev: float = 1e4) -> np.ndarray:
        """Counts of live electrons in log bins of kinetic energy (MeV), computed on the device."""
        out = self.torch.zeros(n_bins, dtype=self.torch.int64, device=self.x.device)
        pe_electron_spectrum(self.handle, n_bins, e_min_mev, e_max_mev, out.data_ptr())
        return out.cpu().numpy().view(np.uint64)

    def photon_map(self, nx: int, x_min_m: float, x_max_m: float, ne: int = 64, e_min_mev: float = 0.511,
                   e_max_mev: float = 1e4) -> np.ndarray:
        """Counts of stored photons over (emission x, log energy), computed on the device (nx x ne)."""
        out = self.torch.zeros(nx * ne, dtype=self.torch.int64, device=self.x.device)
        pe_photon_map(self.handle, nx, x_min_m, x_max_m, ne, e_min_mev, e_max_mev, out.data_ptr())
        return out.cpu().numpy().view(np.uint64).reshape(nx, ne)

    def pair_transport(self, photons=None, n_photons: int | None = None, step_end: int = -1,
                       capacity: int | None = None, method: int = PE_PAIR_DIRECT):
        """Bethe-Heitler conversion, computed on the device, of photon records in this run's target up
        to step_end (-1: the steps done).  photons: a CUDA uint8/int32 tensor of records or a
        PHOTON_DTYPE numpy array (copied to the device); default the run's own stored photons.
        method: PE_PAIR_DIRECT (per-step tests) or PE_PAIR_FREE_PATH (one geometric draw per photon).
        Returns (pairs as PAIR_DTYPE, true pair count, tally words)."""
        torch = self.torch
        if photons is None:
            n = self.tally_out().photons_stored if n_photons is None else n_photons
        else:
            n = (len(photons) if isinstance(photons, np.ndarray) else 0) if n_photons is None else n_photons
        cap = max(int(n), 1) if capacity is None else int(capacity)
        with torch.cuda.stream(self.stream):
            if photons is None:
                dev_ph = self.photons
            elif isinstance(photons, np.ndarray):
                host = torch.from_numpy(np.ascontiguousarray(photons).view(np.int32).reshape(-1))
                dev_ph = host.to(self.x.device)
            else:
                dev_ph = photons
            pairs = torch.zeros(max(cap, 1) * 10, dtype=torch.int32, device=self.x.device)
            tally = torch.zeros(PAIR_TALLY_WORDS, dtype=torch.int64, device=self.x.device)
        pe_pair_transport(self.handle, dev_ph.data_ptr(), int(n), step_end, pairs.data_ptr(), cap, tally.data_ptr(),
                          method)
        self.stream.synchronize()
        t = tally.cpu().numpy().view(np.uint64)
        k = int(min(t[PT["N_PAIRS"]], cap))
        return pairs[: k * 10].cpu().numpy().view(PAIR_DTYPE), int(t[PT["N_PAIRS"]]), t

    def bw_transport(self, bw: int, photons=None, n_photons: int | None = None, step_end: int = -1,
                     capacity: int | None = None):
        """Breit-Wheeler conversion, computed on the device, of photon records in this run's fields up
        to step_end (-1: the steps done); photons as for pair_transport (default: the run's own).
        Returns (pairs as PAIR_DTYPE, true pair count, tally words)."""
        torch = self.torch
        if photons is None:
            n = self.tally_out().photons_stored if n_photons is None else n_photons
        else:
            n = (len(photons) if isinstance(photons, np.ndarray) else 0) if n_photons is None else n_photons
        cap = max(int(n), 1) if capacity is None else int(capacity)
        with torch.cuda.stream(self.stream):
            if photons is None:
                dev_ph = self.photons
            elif isinstance(photons, np.ndarray):
                dev_ph = torch.from_numpy(np.ascontiguousarray(photons).view(np.int32).reshape(-1)).to(self.x.device)
            else:
                dev_ph = photons
            pairs = torch.zeros(max(cap, 1) * 10, dtype=torch.int32, device=self.x.device)
            tally = torch.zeros(PAIR_TALLY_WORDS, dtype=torch.int64, device=self.x.device)
        pe_bw_transport(self.handle, bw, dev_ph.data_ptr(), int(n), step_end, pairs.data_ptr(), cap, tally.data_ptr())
        self.stream.synchronize()
        t = tally.cpu().numpy().view(np.uint64)
        k = int(min(t[PT["N_PAIRS"]], cap))
        return pairs[: k * 10].cpu().numpy().view(PAIR_DTYPE), int(t[PT["N_PAIRS"]]), t

    def wait_words(self) -> np.ndarray:
        """Null-collision waits (uint32, PE_WAIT_NEVER = no further candidate)."""
        return self.wait[:self.n].cpu().numpy().view(np.uint32)

    def tally_out(self) -> TallyOut:
        return pe_tally(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            pe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fixed_to_float(tally, idx: int) -> float:
    return float(int(tally[idx + 1]) & 0xFFFFFFFFFFFFFFFF) + float(int(tally[idx]) & 0xFFFFFFFFFFFFFFFF) / 2.0 ** 64

"""CPU checks of the library boundary: it builds, loads, exports every symbol the
header declares, the ctypes mirrors match the C struct layouts, the product
path never reaches the oracle, and compute calls fail loudly without a GPU."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1612_07592_gb300 as pe
from paper_1612_07592_gb300 import build as pe_build
from paper_1612_07592_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pe.h")


@pytest.fixture(scope="module")
def libpath():
    return pe_build.build()


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[a-z_0-9]+\s+\*?\s*|const char\*\s+)(pe_[a-z0-9_]+)\s*\(", src, re.M)))


def test_header_symbols_exported(libpath):
    names = _declared()
    assert "pe_step" in names and "pe_init_particles" in names and "pe_launch_count" in names and len(names) >= 27
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pe_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = C.CDLL(libpath)
    for n in names:
        getattr(L, n)


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pe.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(pe_table_params),'
                    ' sizeof(pe_run_params), sizeof(pe_buffers), sizeof(pe_launch_config), sizeof(pe_tally_out),'
                    ' offsetof(pe_run_params, seed), offsetof(pe_tally_out, live_particle_steps), sizeof(pe_pair),'
                    ' offsetof(pe_pair, step));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()))
    want = [C.sizeof(pe.TableParams), C.sizeof(pe.RunParams), C.sizeof(pe.Buffers), C.sizeof(pe.LaunchConfig),
            C.sizeof(pe.TallyOut), pe.RunParams.seed.offset, pe.TallyOut.live_particle_steps.offset,
            pe.PAIR_DTYPE.itemsize, pe.PAIR_DTYPE.fields["step"][1]]
    assert got == want


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_1612_07592_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b|oracle/|liboracle|\bor_[a-z_]+\(", txt, re.M), f


def test_compute_fails_loudly_without_gpu(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    tp, Z = pe.table_params(n_eta=4, n_y=4, n_E=4, n_s=4, Z=(13.0,))
    with pytest.raises(pe.PeError) as e:
        pe.pe_create_tables(tp, Z)
    assert e.value.status in (pe.PE_ERR_NOMEM, pe.PE_ERR_CUDA)


def test_argument_errors_are_reported(libpath):
    tp, Z = pe.table_params(n_eta=1, Z=(13.0,))
    with pytest.raises(pe.PeError) as e:
        pe.pe_create_tables(tp, Z)
    assert e.value.status == pe.PE_ERR_ARG
    assert pe.pe_a0_from_intensity(1e21) == pytest.approx(0.855 * 1000 ** 0.5)
    assert pe.pe_a0_from_intensity(1e24) == pytest.approx(855.0, rel=1e-3)
    with pytest.raises(pe.PeError) as e:                 # pair transport without a run
        pe.pe_pair_transport(0, 0, 1, -1, 0, 0, 0)
    assert e.value.status == pe.PE_ERR_ARG
    last = max(pe.PE_MATH.values())                       # the probe checks fn and n before any launch
    for fn, n in ((last + 1, 0), (-1, 0), (pe.PE_MATH["TAU"], -1)):
        with pytest.raises(pe.PeError) as e:
            pe.pe_math_probe(fn, 0, 0, n, None)
        assert e.value.status == pe.PE_ERR_ARG
    pe.pe_math_probe(pe.PE_MATH["TAU"], 0, 0, 0, None)    # nothing to do: no launch, PE_OK


def test_workloads():
    c4 = W.config4()
    n = c4["n"]
    assert len(n) == 64 and n.min() >= 1e4 and n.max() <= 4e6
    assert 1.5e7 < n.sum() < 2.6e7
    assert abs(W.a0_of(1e21) - 27.04) < 0.01 and abs(W.a0_of(1e24) - 855.0) < 0.1
    c5 = W.config5(n_requests=50)
    arr = [q["arrival_s"] for q in c5["requests"]]
    assert np.all(np.diff(arr) > 0)
    assert W.config2()["n"] == 1_000_000 and W.config3()["n"] == 30_000_000
    ph = W.synthetic_photons(2000, 1, (0.0, 10.0), (1.0, 1e4), (0, 100), theta_max=0.3, y_half=2.0)
    assert ph.dtype.itemsize == 32 and len(ph) == 2000
    k = np.sqrt(ph["kx"].astype(np.float64) ** 2 + ph["ky"] ** 2 + ph["kz"] ** 2)
    assert np.abs(k - 1).max() < 1e-6
    assert 0.05 < np.mean(ph["kx"] < 0) < 0.15 and np.all(np.abs(ph["kx"]) >= np.cos(0.3) - 1e-6)
    assert ph["energy"].min() >= 1.0 and ph["energy"].max() <= 1e4 and np.all(np.abs(ph["y"]) <= 2.0)
    assert len(np.unique(ph["id_mech"] & 0x7FFFFFFF)) == 2000


def test_constants_match_header(tmp_path):
    """Every constant the binding passes across the boundary (status codes, enums, tally word
    indices, sizes) equals the header's value, read by compiling the header."""
    names = {"PE_OK": pe.PE_OK, "PE_ERR_ARG": pe.PE_ERR_ARG, "PE_ERR_CUDA": pe.PE_ERR_CUDA,
             "PE_ERR_NOMEM": pe.PE_ERR_NOMEM, "PE_ERR_BUFFER_FULL": pe.PE_ERR_BUFFER_FULL,
             "PE_ERR_TABLE_RANGE": pe.PE_ERR_TABLE_RANGE, "PE_ERR_TIMEOUT": pe.PE_ERR_TIMEOUT,
             "PE_ERR_STATE": pe.PE_ERR_STATE, "PE_LP_Y": pe.PE_LP_Y, "PE_CP": pe.PE_CP,
             "PE_PLANE_1D": pe.PE_PLANE_1D, "PE_GAUSS_2D": pe.PE_GAUSS_2D, "PE_CONST": pe.PE_CONST,
             "PE_PIC_1D": pe.PE_PIC_1D, "PE_F64": pe.PE_F64, "PE_F32": pe.PE_F32, "PE_REST": pe.PE_REST,
             "PE_MAXWELL_JUTTNER": pe.PE_MAXWELL_JUTTNER, "PE_BEAM": pe.PE_BEAM, "PE_CALLER": pe.PE_CALLER,
             "PE_BREMS_DIRECT": pe.PE_BREMS_DIRECT, "PE_BREMS_NULL": pe.PE_BREMS_NULL,
             "PE_WAIT_NEVER": pe.PE_WAIT_NEVER, "PE_PIC_MAX_CELLS": pe.PE_PIC_MAX_CELLS,
             "PE_PAIR_DIRECT": pe.PE_PAIR_DIRECT, "PE_PAIR_FREE_PATH": pe.PE_PAIR_FREE_PATH,
             "PE_PAIR_TALLY_WORDS": pe.PAIR_TALLY_WORDS}
    names.update({"PE_T_" + k: v for k, v in pe.T.items()})
    names.update({"PE_PT_" + k: v for k, v in pe.PT.items()})
    names.update({"PE_MATH_" + k: v for k, v in pe.PE_MATH.items()})
    prog = tmp_path / "consts.c"
    body = "".join(f'printf("{n} %lld\\n", (long long)({n}));' for n in names)
    prog.write_text('#include <stdio.h>\n#include "pe.h"\nint main(void){' + body + "return 0;}\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    bad = {n: (int(got[n]), v) for n, v in names.items() if int(got[n]) != int(v)}
    assert not bad, bad


def test_bw_tables_host_match_oracle(libpath):
    """The library's Breit-Wheeler tables (its own Bessel trapezoid and Gauss panels, built on the
    host) equal the oracle's (adaptive Gauss-Kronrod Bessel functions): T to 1e-8, the CDF to 1e-9."""
    import oracle as O
    T, cdf = pe.pe_bw_tables_host(24, 1e-2, 1e3, 64)
    bw = O.BWTables(24, 1e-2, 1e3, 64)
    np.testing.assert_allclose(T, bw.export(0), rtol=1e-8)
    np.testing.assert_allclose(cdf, bw.export(1), rtol=0, atol=1e-9)
    for bad in ((1, 1e-2, 1e3, 64), (24, 0.0, 1e3, 64), (24, 1e-2, 1e-3, 64), (24, 1e-2, 1e3, 5000)):
        with pytest.raises(pe.PeError) as e:
            pe.pe_bw_tables_host(*bad)
        assert e.value.status == pe.PE_ERR_ARG

"""Planted mistakes in the oracle, each caught by a pin (CPU only).

Each mutant in ``oracle.MUTANTS`` is step.c compiled with ``OR_MUTANT_<name>``: one plausible
mistake -- a dropped term, a wrong sign, a missing factor, a one-step lag, a wrong constant.
The pin named beside it runs in a child process against that build and must fail with a test
failure (pytest exit status 1, not a crash or a collection error); the same pins pass on the
oracle itself in the normal suite.
"""
import os
import subprocess
import sys

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = "tests/test_oracle_pins.py::"
CAUGHT_BY = {
    "PHILOX_MULT": PINS + "test_philox_known_answers",               # a wrong round multiplier
    "BORIS_SIGN": PINS + "test_ncs_first_emission_follows_the_rate",  # rotation the wrong way
    "ETA_UE": PINS + "test_eta_identity_exact",                       # the 2 V_x (u.E) term dropped
    "PHOTON_BACKWARD": PINS + "test_ncs_first_emission_follows_the_rate",   # photon against the velocity
    "NCS_NO_GAMMA": PINS + "test_ncs_first_emission_follows_the_rate",      # rate without 1/gamma
    "NCS_LAG": PINS + "test_ncs_first_emission_follows_the_rate",     # crossing tested before the decrement
    "RECOIL_TALLY": PINS + "test_energy_bookkeeping",                 # recoil energy tallied with its sign flipped
    "BREMS_NO_BETA": PINS + "test_brems_probability_carries_beta",    # Eq. 4 without beta
    "NCS_F_QUANTUM": PINS + "test_ncs_F_vs_scipy_pointwise",          # the emissivity's delta^2 y K_2/3 term dropped
    "NCS_H_JACOBIAN": PINS + "test_ncs_table_vs_brute_force",         # h integrated without dchi/chi's Jacobian
    "BREMS_COULOMB": PINS + "test_brems_complete_screening_closed_form",     # Eq. 1 without f(Z)
    "INCIDENT_SIGN": PINS + "test_plane_wave_orbit_from_rest",        # the laser's E_y with the wrong sign
    "POSITION_NO_GAMMA": PINS + "test_plane_wave_orbit_from_rest",    # x advanced by u dt instead of v dt
    "MIRROR_SIGN": "tests/test_oracle_pins_variants.py::test_reflected_wave_mirror_node",   # mirror image not inverted
    "BW_NORM": "tests/test_oracle_bw.py::test_small_chi_limit",       # T(chi) with a stray factor 2
    "PIC_CURRENT_SIGN": "tests/test_oracle_pic.py::test_pic_gauss_law",     # J_x deposited with the wrong sign
    "NCS_SAMPLE_FLIP": PINS + "test_ncs_sampler_inverts_table",       # the NCS CDF inverted at 1 - R
    "BREMS_SAMPLE_FLIP": PINS + "test_brems_sampler_range_and_inversion",   # the brems CDF inverted at 1 - R
    "NULL_THINNING": "tests/test_oracle_pins_variants.py::test_null_collision_first_event_has_direct_probability",
    "ENVELOPE_FALL": PINS + "test_plane_wave_fields_from_the_vector_potential",  # g' of the falling ramp signed wrong
    "GOUY_SIGN": PINS + "test_gaussian_focus_satisfies_the_paraxial_equation",  # Gouy phase against the curvature
    "MJ_TEMPERATURE": PINS + "test_maxwell_juttner_mean_energy",      # theta = T / 2 m c^2
    "BH_SECOND_TERM": "tests/test_oracle_pairs.py::test_bh_complete_screening_limit",  # Tsai's x(1-x) term dropped
    "DELTA_MAP": PINS + "test_ncs_sampler_inverts_table",             # delta from y with 1 for 2
    "WAIT_SCALE": "tests/test_oracle_pins_variants.py::test_null_collision_waits_are_geometric",  # waits at twice the rate
    "HIST_SHIFT": PINS + "test_histograms_bin_the_photon_records",    # energy bins one over
    "INIT_SPREAD": PINS + "test_initial_positions_uniform_in_the_slab",     # electrons over twice the slab
    "PIC_INJECT_HALF": "tests/test_oracle_pic.py::test_pic_vacuum_injection_is_exact",  # the laser entering at half amplitude
    "BW_PHOTON_STILL": "tests/test_oracle_bw.py::test_transport_in_the_plane_wave",     # photons that never move
    "CHI_KE": "tests/test_oracle_bw.py::test_photon_chi_special_cases",  # chi without the (k.E) term
    "Y_UPDATE": PINS + "test_free_streaming_and_the_absorbing_box",   # 2D y advanced with u_z
    "BOX_ONE_SIDED": PINS + "test_free_streaming_and_the_absorbing_box",    # the box's rear face only
    "CURVATURE_SIGN": PINS + "test_gaussian_focus_satisfies_the_paraxial_equation",  # wavefront curvature sign
    "AMPLITUDE": PINS + "test_gaussian_focus_satisfies_the_paraxial_equation",       # w0 / w for sqrt(w0 / w)
    "TAU_NO_RESET": PINS + "test_ncs_optical_depth_resets_after_emission",  # no fresh tau after an emission
    "CLAMP_GAMMA": PINS + "test_photon_energy_clamp_conserves_energy",      # the photon clamped to gamma
    "TARGET_Y": PINS + "test_brems_only_inside_the_target",           # the 2D target unbounded in y
    "ETA_GM": PINS + "test_eta_identity_exact",                       # gamma - u_x without its 1
    "BH_FREE_PATH": "tests/test_oracle_pairs.py::test_pair_free_path_conversion_law",  # free path at twice the rate
    "ROW_WEIGHT": PINS + "test_ncs_sampler_inverts_table",            # interpolation weight on the wrong row
    "BW_X_NODES": "tests/test_oracle_bw.py::test_sampler_follows_the_spectrum",   # uniform x nodes for (1 - cos)/2
    "REFL_SQUARED": "tests/test_oracle_pins_variants.py::test_reflected_wave_is_the_mirror_image_superposed",  # r^2 for r
    "PIC_EX_SIGN": "tests/test_oracle_pic.py::test_pic_gauss_law",    # E_x driven up by J_x
    "PIC_JY_WEIGHT": "tests/test_oracle_pic.py::test_pic_transverse_current_is_time_centred",  # J_y at x^{n+1} only
    "PIC_GATHER_NODE": "tests/test_oracle_pic.py::test_pic_plasma_frequency",    # E_x gathered as if at nodes
    "PIC_BY_SIGN": "tests/test_oracle_pic.py::test_pic_gather_decodes_the_waves",  # B_y read from G with the wrong sign
}


def _run_pin(mutant):
    env = dict(os.environ, ORACLE_MUTANT=mutant, OMP_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", CAUGHT_BY[mutant]],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def pin_runs():
    """Every mutant's pin, run in child processes side by side."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        return dict(zip(sorted(CAUGHT_BY), ex.map(_run_pin, sorted(CAUGHT_BY))))


def test_every_mutant_has_a_pin():
    assert set(CAUGHT_BY) == set(O.MUTANTS)


@pytest.mark.parametrize("mutant", sorted(CAUGHT_BY))
def test_pin_catches_mutant(mutant, pin_runs):
    p = pin_runs[mutant]
    assert p.returncode == 1, (p.returncode, p.stdout[-3000:], p.stderr[-2000:])
